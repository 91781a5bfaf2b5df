"""Small shared helpers for the tests (input construction and error norms only)."""
import numpy as np

import synth


def rel_fro(a, b):
    """||a - b||_F / ||b||_F."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))


def small_system(n, n_v, n_c, n_mu=None, seed_index=50, n_pw=None):
    """A small seeded system; `n` an int or (n1, n2, n3).  With n_mu None the
    points are all QRCP pivots up to min(N_r, 2 * pairs)."""
    if isinstance(n, int):
        n = (n, n, n)
    n = tuple(int(v) for v in n)
    n_r = int(np.prod(n))
    n_e = n_v + n_c
    if n_pw is None:
        n_pw = min(max(2 * n_e, 24), n_r - 8)
    phi = synth.make_orbitals(n, n_e, 1000 + seed_index, n_pw=n_pw)
    energies = synth.make_energies(n_v, n_c, 2000 + seed_index)
    if n_mu is None:
        n_mu = min(n_r, 2 * n_v * n_c)
    mu = synth.qrcp_points(phi, n_v, n_mu)
    cell = tuple(v * synth.GRID_SPACING_BOHR for v in n)
    return synth.System(n=n, cell=cell, n_v=n_v, n_c=n_c, phi=phi, energies=energies,
                        mu_idx=mu, name=f"small{n}")
