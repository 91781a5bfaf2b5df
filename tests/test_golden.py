"""The oracle against the worked example of tests/golden/plane_wave_two_pairs.txt,
whose eps^-1 and W = eps^-1 V are known in closed form (two plane-wave pairs
on a 16^3 grid).  The expected values are the fixture's hand-derived
expressions; no program, oracle or CUDA path wrote them.  CPU only."""
import numpy as np
import pytest

import oracle as O
import synth
from oracle import cohsex as X
from helpers import eval_expr, load_golden, plane_wave_golden, plane_wave_golden_eps_inv, rel_fro


def test_fixture_is_consistent():
    g = load_golden("plane_wave_two_pairs.txt")
    for i in ("c1", "c2"):
        assert eval_expr(g[f"lambda {i} at w = 0"]) == pytest.approx(eval_expr(g[f"lambda {i}"], w=0.0), rel=1e-15)
        for w in (0.0, 0.7):
            lam = eval_expr(g[f"lambda {i}"], w=w)
            assert 1.0 < lam < 1.2  # eps >= 1 on the pair directions, weak screening at this cell size
            assert eval_expr(g[f"w_eigen {i}"], w=w) > 0
    with pytest.raises(ValueError):
        eval_expr("__import__('os')")


def test_oracle_eps_on_pair_directions():
    """eps u_i = lambda_i u_i and eps v = v for the constant (G = 0) direction."""
    s, u, g = plane_wave_golden(2)
    eps = O.eps_dense(s.phi, s.energies, 1, s.n, s.cell)
    for k, i in enumerate(("c1", "c2")):
        assert rel_fro(eps @ u[:, k], eval_expr(g[f"lambda {i}"], w=0.0) * u[:, k]) < 1e-13
    one = np.full(s.n_r, 1.0)
    assert rel_fro(eps @ one, one) < 1e-13


@pytest.mark.parametrize("n_mu", [2, 6])
def test_oracle_isdf_smw_equals_closed_form(n_mu):
    """ISDF-SMW at pair rank 2, with 2 points and with 6 (rank-deficient
    C C^T), equals the closed form eps^-1 X and W u_i at every frequency."""
    s, u, g = plane_wave_golden(n_mu)
    x = synth.probe_block(s.n_r, 4)
    vu = O.apply_coulomb(u, s.n, s.cell)
    for w in (float(t) for t in g["frequencies"].split()):
        ref = O.isdf_smw_solve(s.phi, s.energies, 1, s.mu_idx, s.n, s.cell, x, omega=w)
        assert ref.rank == 2
        closed = plane_wave_golden_eps_inv(u, g, x, w)
        assert rel_fro(ref.y, closed) < 1e-12, w
        # eps^-1 is close to I here: the correction on its own, too
        assert rel_fro(ref.y - x, closed - x) < 1e-10, w
        wu = O.apply_eps_inv(ref.theta, ref.k, vu, s.n, s.cell)  # W u = eps^-1 (V u)
        for k, i in enumerate(("c1", "c2")):
            assert rel_fro(wu[:, k], eval_expr(g[f"w_eigen {i}"], w=w) * u[:, k]) < 1e-12, (w, i)


def _sigma_closed(g):
    bands = ("v", "c1", "c2")
    return [np.array([eval_expr(g[f"{kind} {b}"]) for b in bands]) for kind in ("sigma_sex_x", "sigma_x", "sigma_coh")]


def test_fixture_sigma_uses_the_fixture_lambdas():
    """The COHSEX expressions carry lambda_i(0) and v_Gi / Omega_cell of the
    fixture's own definitions."""
    g = load_golden("plane_wave_two_pairs.txt")
    lam = [eval_expr(g["lambda c1 at w = 0"]), eval_expr(g["lambda c2 at w = 0"])]
    vo = [1 / (8 * np.pi), 1 / (16 * np.pi)]  # v_Gi / Omega_cell = (64 / pi) / 512, (32 / pi) / 512
    sex, x, coh = _sigma_closed(g)
    assert np.allclose(x[1:], [-v for v in vo], rtol=1e-15)
    assert np.allclose(sex[1:], [(1 - 1 / l) * v for l, v in zip(lam, vo)], rtol=1e-15)
    assert np.allclose(coh, [-0.5 * sum((1 - 1 / l) * v for l, v in zip(lam, vo)),
                             -0.5 * (1 - 1 / lam[0]) * vo[0], -0.5 * (1 - 1 / lam[1]) * vo[1]], rtol=1e-15)


def test_oracle_sigma_isdf_equals_closed_form():
    """Algorithm 3 steps 1-7 with the three pair sets fitted at full rank
    (the dense route equals this one at full rank, tests/test_oracle_cohsex.py;
    its explicit Coulomb double sum is too slow on 16^3 for the CPU suite)."""
    s, _, g = plane_wave_golden(2)
    mu_vn = synth.qrcp_points(X.pair_phi_vn(s.phi, 1), 1, 5)
    mu_nn = synth.qrcp_points(X.pair_phi_nn(s.phi), 3, 12)
    got = X.sigma_isdf(s.phi, s.energies, 1, s.mu_idx, mu_vn, mu_nn, s.n, s.cell)
    for a, b, name in zip(got, _sigma_closed(g), ("SEX_X", "X", "COH")):
        assert np.abs(a - b).max() < 1e-11 * np.abs(b).max(), (name, a, b)
