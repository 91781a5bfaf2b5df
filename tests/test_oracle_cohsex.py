"""Pins of the COHSEX oracle (oracle/cohsex.py): the ISDF form (Algorithm 3
steps 1-7 with the Hadamard identity) against the exact dense form when
every pair set is fitted at full rank, and the sum-over-states Coulomb hole
against the local form of Eq. Sigma_G0W0 for a complete orbital set."""
import numpy as np

import oracle as O
import synth
from oracle import cohsex as X
from helpers import rel_fro, small_system


def _full_rank_points(phi, n_v_pairs_left, rows):
    """QRCP points of a pair set, as many as its numerical rank."""
    n_r = phi.shape[0]
    return synth.qrcp_points(phi, n_v_pairs_left, min(n_r, rows))


def test_isdf_sigma_equals_exact_at_full_rank():
    s = small_system(8, 2, 3, n_mu=6, seed_index=120)
    phi, n_v, n_e = s.phi, s.n_v, s.n_e
    # every pair set fitted with at least as many points as its rank
    mu_vc = synth.qrcp_points(phi, n_v, n_v * (n_e - n_v))
    mu_vn = synth.qrcp_points(X.pair_phi_vn(phi, n_v), n_v, n_v * n_e)
    mu_nn = synth.qrcp_points(X.pair_phi_nn(phi), n_e, n_e * (n_e + 1) // 2)
    ex = X.sigma_exact(phi, s.energies, n_v, s.n, s.cell)
    iz = X.sigma_isdf(phi, s.energies, n_v, mu_vc, mu_vn, mu_nn, s.n, s.cell)
    for a, b in zip(iz, ex):
        assert rel_fro(a, b) < 1e-9


def test_coh_sum_over_states_equals_local_form_for_a_complete_set():
    """With all N_r orthonormal orbitals, sum_m psi_m(r) psi_m(r') = delta(r, r'),
    so 1/2 sum_m (psi_n .* psi_m)^T (W - V) (psi_n .* psi_m) = 1/2 sum_r psi_n(r)^2 (W - V)(r, r)."""
    n = (4, 4, 4)
    n_r = 64
    rng = np.random.default_rng(5)
    q, _ = np.linalg.qr(rng.standard_normal((n_r, n_r)))
    phi = np.asfortranarray(q)
    n_v = 10
    energies = np.concatenate([np.sort(rng.uniform(-0.4, -0.1, n_v)), np.sort(rng.uniform(0.0, 0.8, n_r - n_v))])
    cell = (2.0, 2.0, 2.0)
    _, _, coh = X.sigma_exact(phi, energies, n_v, n, cell)
    wmv = (O.eps_inv_dense(phi, energies, n_v, n, cell) - np.eye(n_r)) @ O.coulomb_dense(n, cell)
    local = 0.5 * (phi ** 2).T @ np.diag(wmv)
    assert rel_fro(coh, local) < 1e-11


def test_sigma_signs_and_exchange_is_negative():
    """Sigma_X is minus a sum of Coulomb energies (V positive semidefinite): <= 0;
    W - V is negative semidefinite in the static limit (eps^-1 V <= V), so
    Sigma_SEX_X >= 0 and Sigma_COH <= 0."""
    s = small_system(8, 2, 4, n_mu=8, seed_index=121)
    sex_x, x, coh = X.sigma_exact(s.phi, s.energies, s.n_v, s.n, s.cell)
    assert np.all(x <= 1e-14) and np.all(sex_x >= -1e-14) and np.all(coh <= 1e-14)
