"""GPU parity of the static COHSEX self-energies (isdf_cohsex, Algorithm 3
steps 4-7) against the FP64 oracle (oracle/cohsex.py): the ISDF form with
the same points, and the exact dense form when every pair set is fitted at
full rank.  Tolerance 1e-10 relative (FP64 path); the self-energies are
basis-invariant (they depend on the span of each fit, not on its basis)."""
import numpy as np
import pytest

import synth
from oracle import cohsex as X
from helpers import rel_fro, small_system

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2403_12340_gb300 as pkg

    pkg.load_library()


def _gpu_sigma(s, mu_vc, mu_vn, mu_nn):
    import torch
    import paper_2403_12340_gb300 as pkg

    n_v, n_e = s.n_v, s.n_e
    with pkg.IsdfSmw(s.n, s.cell) as vc, pkg.IsdfSmw(s.n, s.cell) as vn, pkg.IsdfSmw(s.n, s.cell) as nn:
        vc.fit(pkg.to_fortran(s.phi), n_v, s.n_c, mu_vc)
        vc.polarizability(s.energies, [0.0])
        vc.smw(0)
        vn.fit(pkg.to_fortran(X.pair_phi_vn(s.phi, n_v)), n_v, n_e, mu_vn)
        nn.fit(pkg.to_fortran(X.pair_phi_nn(s.phi)), n_e, n_e, mu_nn)
        out = pkg.isdf_cohsex(vc.ctx, vn.ctx, nn.ctx, n_e)
        torch.cuda.synchronize()
        return [t.cpu().numpy() for t in out]


CASES = [  # grid, n_v, n_c, points of the vc, vn and nn fits
    (10, 2, 5, 8, 12, 24),
    ((12, 10, 9), 3, 6, 14, 20, 40),
    (16, 4, 10, 40, 48, 96),
]


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}-{c[1]}-{c[2]}" for c in CASES])
def test_cohsex_matches_oracle_isdf(case):
    n, n_v, n_c, k_vc, k_vn, k_nn = case
    s = small_system(n, n_v, n_c, n_mu=k_vc, seed_index=130 + n_v)
    mu_vc = np.asarray(s.mu_idx)
    mu_vn = synth.qrcp_points(X.pair_phi_vn(s.phi, n_v), n_v, k_vn)
    mu_nn = synth.qrcp_points(X.pair_phi_nn(s.phi), s.n_e, k_nn)
    g = _gpu_sigma(s, mu_vc, mu_vn, mu_nn)
    o = X.sigma_isdf(s.phi, s.energies, n_v, mu_vc, mu_vn, mu_nn, s.n, s.cell)
    for a, b in zip(g, o):
        assert rel_fro(a, b) < 1e-10


def test_cohsex_equals_exact_at_full_rank():
    s = small_system(8, 2, 3, n_mu=6, seed_index=140)
    n_v, n_e = s.n_v, s.n_e
    mu_vc = synth.qrcp_points(s.phi, n_v, n_v * (n_e - n_v))
    mu_vn = synth.qrcp_points(X.pair_phi_vn(s.phi, n_v), n_v, n_v * n_e)
    mu_nn = synth.qrcp_points(X.pair_phi_nn(s.phi), n_e, n_e * (n_e + 1) // 2)
    g = _gpu_sigma(s, mu_vc, mu_vn, mu_nn)
    e = X.sigma_exact(s.phi, s.energies, n_v, s.n, s.cell)
    for a, b in zip(g, e):
        assert rel_fro(a, b) < 1e-9


def test_cohsex_errors():
    import paper_2403_12340_gb300 as pkg

    s = small_system(10, 2, 5, n_mu=8, seed_index=141)
    n_v, n_e = s.n_v, s.n_e
    mu_vn = synth.qrcp_points(X.pair_phi_vn(s.phi, n_v), n_v, 12)
    with pkg.IsdfSmw(s.n, s.cell) as vc, pkg.IsdfSmw(s.n, s.cell) as vn:
        vc.fit(pkg.to_fortran(s.phi), n_v, s.n_c, s.mu_idx)
        vn.fit(pkg.to_fortran(X.pair_phi_vn(s.phi, n_v)), n_v, n_e, mu_vn)
        with pytest.raises(pkg.IsdfError) as ei:
            pkg.isdf_cohsex(vc.ctx, vn.ctx, vn.ctx, n_e)  # no smw_inverse yet
        assert ei.value.code == -9
        vc.polarizability(s.energies, [0.0])
        vc.smw(0)
        with pytest.raises(pkg.IsdfError) as ei:
            pkg.isdf_cohsex(vc.ctx, vn.ctx, vn.ctx, n_e)  # vn passed as the nn fit
        assert ei.value.code == -2
