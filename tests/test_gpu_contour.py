"""GPU parity of the contour-integral polarizability (Algorithm 2,
build_polarizability_contour): D against the oracle's contour quadrature at
the same number of nodes (the same sum, so FP64 agreement), against the
direct pair sum within the quadrature error, and eps^-1 X against the
oracle.  Tolerances: 1e-10 (FP64) / 1e-6 (mixed) on eps^-1 X with enough
nodes that the quadrature error is below 1e-13 (Eq. rel_err_Cauchy,
empirically reached at 20 nodes for these spectra)."""
import numpy as np
import pytest

import oracle as O
import synth
from oracle import cauchy as OC
from helpers import rel_fro, small_system

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2403_12340_gb300 as pkg

    pkg.load_library()


def _whitened_oracle_d(s, theta_rank, piv, L, b):
    """D = L_r^-1 (-2 B_rr) L_r^-T in the GPU's pivot basis."""
    r = theta_rank
    p = piv[:r]
    brr = b[np.ix_(p, p)]
    lr = L[:r, :r]
    x = np.linalg.solve(lr, -2.0 * brr)
    return np.linalg.solve(lr, x.T).T


@pytest.mark.parametrize("n_nodes", [6, 12, 24])
def test_contour_D_matches_oracle_quadrature(n_nodes):
    import torch
    import paper_2403_12340_gb300 as pkg

    s = small_system(12, 3, 13, n_mu=30, seed_index=95)
    mu = np.asarray(s.mu_idx)
    with pkg.IsdfSmw(s.n, s.cell) as sol:
        _, rank = sol.fit(pkg.to_fortran(s.phi), s.n_v, s.n_c, mu)
        D, _ = sol.polarizability_contour(s.energies, n_nodes, want_D=True)
        piv, L = sol.factor(want_L=True)
        torch.cuda.synchronize()
        d_gpu = D[0].cpu().numpy()[:rank, :rank]
        L = L.cpu().numpy()
    pm = s.phi[mu]
    d_quad = _whitened_oracle_d(s, rank, piv, L, OC.polarizability_contour(pm, s.energies, s.n_v, n_nodes))
    d_sum = _whitened_oracle_d(s, rank, piv, L, OC.polarizability_direct(pm, s.energies, s.n_v))
    assert rel_fro(d_gpu, d_quad) < 1e-12
    assert rel_fro(d_gpu, d_sum) < 50 * OC.contour_error_bound(s.energies, s.n_v, n_nodes) + 1e-13


CASES = [(12, 3, 13, 30, 96), ((10, 12, 9), 2, 10, 16, 97), (16, 4, 28, 128, 98)]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}-{c[1]}-{c[2]}-{c[3]}" for c in CASES])
def test_contour_eps_inv_matches_oracle(case, prec):
    import torch
    import paper_2403_12340_gb300 as pkg

    n, n_v, n_c, n_mu, seed = case
    s = small_system(n, n_v, n_c, n_mu=n_mu, seed_index=seed)
    x = synth.probe_block(s.n_r, 5)
    with pkg.IsdfSmw(s.n, s.cell) as sol:
        sol.fit(pkg.to_fortran(s.phi), s.n_v, s.n_c, s.mu_idx, prec=prec)
        sol.polarizability_contour(s.energies, 24)
        sol.smw(0)
        y = sol.apply(pkg.to_fortran(x), 0).cpu().numpy()
        torch.cuda.synchronize()
    ref = O.isdf_smw_solve(s.phi, s.energies, s.n_v, s.mu_idx, s.n, s.cell, x)
    assert rel_fro(y, ref.y) < (1e-10 if prec == 0 else 1e-6)


def test_contour_at_48():
    """48^3 / N_mu = 1536, FP64: the contour D with the nodes the bound asks
    for 1e-13 against the pair-sum D of the same context."""
    import torch
    import paper_2403_12340_gb300 as pkg

    s = synth.workload("isdf48")
    n_nodes = pkg.isdf_contour_nodes(s.energies, s.n_v, s.n_c, 1e-13)
    assert 10 <= n_nodes <= 64
    with pkg.IsdfSmw(s.n, s.cell) as sol:
        sol.fit(pkg.to_fortran(s.phi), s.n_v, s.n_c, s.mu_idx)
        Dd, _ = sol.polarizability(s.energies, [0.0], want_D=True)
        Dc, _ = sol.polarizability_contour(s.energies, n_nodes, want_D=True)
        torch.cuda.synchronize()
        assert rel_fro(Dc.cpu().numpy(), Dd.cpu().numpy()) < 1e-11


def test_contour_arguments():
    import paper_2403_12340_gb300 as pkg

    s = small_system(12, 3, 9, n_mu=20, seed_index=99)
    with pkg.IsdfSmw(s.n, s.cell) as sol:
        sol.fit(pkg.to_fortran(s.phi), s.n_v, s.n_c, s.mu_idx)
        with pytest.raises(pkg.IsdfError) as ei:
            sol.polarizability_contour(s.energies, 0)
        assert ei.value.code == -1
        bad = s.energies.copy()
        bad[0] = bad[-1] + 1.0  # no gap
        with pytest.raises(pkg.IsdfError) as ei:
            sol.polarizability_contour(bad, 16)
        assert ei.value.code == -5
