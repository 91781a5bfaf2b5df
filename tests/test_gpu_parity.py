"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerance: relative Frobenius error <= 1e-10 on the basis-invariant outputs
(eps^-1 X, and the dense inverse where it exists), as the FP64 target states.
Basis-dependent intermediates (theta, G, D, K) are compared after mapping
the oracle's least-squares P into the whitened pivot basis (full-rank cases).
"""
import numpy as np
import pytest

import oracle as O
import synth
from gpu_helpers import run_gpu
from helpers import rel_fro, small_system

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2403_12340_gb300 as pkg

    pkg.load_library()


SMALL = [
    # (grid, N_v, N_c, N_mu): cubic / non-cubic / odd axes, ragged tiles,
    # N_mu above, at and below the pair count
    ((6, 6, 6), 2, 5, 10),
    ((8, 10, 6), 3, 7, 19),
    ((9, 9, 9), 3, 6, 18),
    ((5, 6, 7), 2, 4, 8),
    ((12, 10, 14), 4, 9, 30),
    ((8, 8, 8), 2, 3, 9),        # 9 points > 6 pairs: rank-deficient C C^T
    ((4, 4, 4), 3, 10, 64),      # every grid point is an interpolation point
    ((10, 10, 10), 1, 1, 1),     # one pair, one point (Sherman-Morrison)
    ((16, 12, 10), 6, 20, 70),   # N_mu crosses a 64-wide tile
]


@pytest.mark.parametrize("grid,nv,nc,nmu", SMALL)
def test_small_systems_match_oracle(grid, nv, nc, nmu):
    s = small_system(grid, nv, nc, nmu, seed_index=hash((grid, nv, nc)) % 97)
    x = synth.probe_block(s.n_r, 5)
    omegas = (0.0, 0.37, 4.0)
    g = run_gpu(s, x, omegas)
    for k, w in enumerate(omegas):
        ref = O.isdf_smw_solve(s.phi, s.energies, s.n_v, s.mu_idx, s.n, s.cell, x, omega=w)
        assert g["rank"] == ref.rank
        assert rel_fro(g["y"][k], ref.y) < TOL, (k, rel_fro(g["y"][k], ref.y))


def test_isdf16_equals_dense_inverse():
    """4096-point grid, 112 pairs, 128 points: ISDF-SMW is exact, so the GPU
    result matches the dense 4096 x 4096 inverse of eps."""
    s = synth.workload("isdf16")
    x = synth.probe_block(s.n_r)
    g = run_gpu(s, x)
    assert g["rank"] == 112
    einv = O.eps_inv_dense(s.phi, s.energies, s.n_v, s.n, s.cell)
    assert rel_fro(g["y"][0], einv @ x) < TOL
    ref = O.isdf_smw_solve(s.phi, s.energies, s.n_v, s.mu_idx, s.n, s.cell, x)
    assert rel_fro(g["y"][0], ref.y) < TOL
    # W = eps^-1 V is symmetric: X^T eps^-1 (V X) is a symmetric 16 x 16 matrix
    vx = O.apply_coulomb(x, s.n, s.cell)
    g2 = run_gpu(s, vx)
    wx = x.T @ g2["y"][0]
    assert np.abs(wx - wx.T).max() < 1e-10 * np.abs(wx).max()


def test_whitened_basis_intermediates_full_rank():
    """theta = P_p L, G = L^T (P^T V P)_pp L, D = L^-1 (-2 B_pp) L^-T,
    K_pp = L K L^T, with P, B, G, K from the oracle; theta at the pivot
    points equals L; L is the Cholesky factor of C C^T in pivot order."""
    s = small_system((12, 10, 14), 4, 9, 30, seed_index=5)
    x = synth.probe_block(s.n_r, 3)
    g = run_gpu(s, x, want=True)
    r = g["rank"]
    assert r == 30
    piv = g["piv"][:r]
    L = g["L"][:r, :r]
    c = O.isdf_coefficients(s.phi, s.n_v, s.mu_idx)
    a = (c @ c.T)[np.ix_(piv, piv)]
    assert rel_fro(L, np.linalg.cholesky(a)) < 1e-12
    theta = g["theta"][:, :r]
    assert rel_fro(theta[s.mu_idx[piv], :], L) < 1e-12
    ref = O.isdf_smw_solve(s.phi, s.energies, s.n_v, s.mu_idx, s.n, s.cell, x)
    P = ref.theta[:, piv]
    assert rel_fro(theta, P @ L) < 1e-11
    assert rel_fro(g["G"][:r, :r], L.T @ ref.g[np.ix_(piv, piv)] @ L) < 1e-11
    Linv = np.linalg.inv(L)
    assert rel_fro(g["D"][0][:r, :r], Linv @ (-2.0 * ref.b[np.ix_(piv, piv)]) @ Linv.T) < 1e-11
    assert rel_fro(L @ g["K"][0][:r, :r] @ L.T, ref.k[np.ix_(piv, piv)]) < 1e-10


def test_rank_deficient_projector_invariant():
    """At 128 points and 112 pairs theta is not unique, but theta theta^T =
    M_hat M_hat^T (the projection of M onto the row space of C) is."""
    s = synth.workload("isdf16")
    x = synth.probe_block(s.n_r, 4)
    g = run_gpu(s, x, want=True)
    th = g["theta"][:, : g["rank"]]
    ref_th, _ = O.isdf_fit(s.phi, s.n_v, s.mu_idx)
    mh = ref_th @ O.isdf_coefficients(s.phi, s.n_v, s.mu_idx)
    assert rel_fro(th @ (th.T @ x), mh @ (mh.T @ x)) < TOL
    assert np.all(g["theta"][:, g["rank"]:] == 0.0)


def test_degenerate_zero_pairs_at_points_gives_identity():
    """Orbitals that all vanish at the chosen points: C = 0, rank 0, and
    eps_hat^-1 = I (no screening is captured)."""
    s = small_system((6, 6, 6), 2, 4, 6)
    s.phi[s.mu_idx, :] = 0.0
    x = synth.probe_block(s.n_r, 2)
    g = run_gpu(s, x)
    assert g["rank"] == 0
    assert np.array_equal(g["y"][0], x)


def test_apply_many_rhs_and_in_place():
    s = small_system((8, 8, 8), 3, 7, 21)
    x = synth.probe_block(s.n_r, 70)     # more columns than one 64-column chunk
    ref = O.isdf_smw_solve(s.phi, s.energies, s.n_v, s.mu_idx, s.n, s.cell, x)
    g = run_gpu(s, x)
    assert rel_fro(g["y"][0], ref.y) < TOL
    g2 = run_gpu(s, x, in_place=True)
    assert rel_fro(g2["y"][0], ref.y) < TOL


def test_error_codes():
    import torch

    import paper_2403_12340_gb300 as pkg

    s = small_system((6, 6, 6), 2, 5, 10)
    phi = pkg.to_fortran(s.phi)
    with pkg.IsdfSmw(s.n, s.cell) as ctx:
        X = pkg.to_fortran(synth.probe_block(s.n_r, 2))
        with pytest.raises(pkg.IsdfError, match="ISDF_ERR_STATE"):
            ctx.smw(0)
        bad = s.mu_idx.copy()
        bad[1] = bad[0]
        with pytest.raises(pkg.IsdfError, match="ISDF_ERR_INDEX"):
            ctx.fit(phi, s.n_v, s.n_c, bad)
        bad[1] = s.n_r
        with pytest.raises(pkg.IsdfError, match="ISDF_ERR_INDEX"):
            ctx.fit(phi, s.n_v, s.n_c, bad)
        nanphi = pkg.to_fortran(phi)
        nanphi[3, 1] = float("nan")
        with pytest.raises(pkg.IsdfError, match="ISDF_ERR_NONFINITE"):
            ctx.fit(nanphi, s.n_v, s.n_c, s.mu_idx)
        ctx.fit(phi, s.n_v, s.n_c, s.mu_idx)
        e = s.energies.copy()
        e[0], e[-1] = e[-1], e[0]
        with pytest.raises(pkg.IsdfError, match="ISDF_ERR_ORDER"):
            ctx.polarizability(e, [0.0])
        with pytest.raises(pkg.IsdfError, match="ISDF_ERR_ARG"):
            ctx.polarizability(s.energies, [-1.0])
        ctx.polarizability(s.energies, [0.0])
        with pytest.raises(pkg.IsdfError, match="ISDF_ERR_STATE"):
            ctx.apply(X, 0)
        with pytest.raises(pkg.IsdfError, match="ISDF_ERR_ARG"):
            ctx.smw(3)
        ctx.smw(0)
        Y = ctx.apply(X, 0)
        ref = O.isdf_smw_solve(s.phi, s.energies, s.n_v, s.mu_idx, s.n, s.cell, synth.probe_block(s.n_r, 2))
        assert rel_fro(Y.cpu().numpy(), ref.y) < TOL
    with pytest.raises(pkg.IsdfError, match="ISDF_ERR_SHAPE"):
        pkg.IsdfSmw((17, 8, 8), (8.5, 4.0, 4.0))


def test_context_reuse_across_systems():
    """One context, two fits of different sizes: same answers as fresh ones."""
    import paper_2403_12340_gb300 as pkg

    a = small_system((8, 8, 8), 3, 7, 21, seed_index=3)
    b = small_system((8, 8, 8), 2, 9, 12, seed_index=4)
    xa = synth.probe_block(a.n_r, 2)
    with pkg.IsdfSmw(a.n, a.cell) as ctx:
        ys = []
        for sysm in (a, b, a):
            ctx.fit(pkg.to_fortran(sysm.phi), sysm.n_v, sysm.n_c, sysm.mu_idx)
            ctx.polarizability(sysm.energies, [0.0])
            ctx.smw(0)
            ys.append(ctx.apply(pkg.to_fortran(xa), 0).cpu().numpy())
    for sysm, y in zip((a, b, a), ys):
        ref = O.isdf_smw_solve(sysm.phi, sysm.energies, sysm.n_v, sysm.mu_idx, sysm.n, sysm.cell, xa)
        assert rel_fro(y, ref.y) < TOL


def test_points_from_device_memory():
    """Interpolation points passed as an int64 device array give the same
    fit and eps^-1 X as the same points in host memory; a bad index in
    device memory is refused like one in host memory."""
    import torch

    import paper_2403_12340_gb300 as pkg

    s = small_system((12, 10, 14), 4, 9, 30, seed_index=6)
    x = synth.probe_block(s.n_r, 3)
    ref = O.isdf_smw_solve(s.phi, s.energies, s.n_v, s.mu_idx, s.n, s.cell, x)
    ys = []
    for on_device in (False, True):
        with pkg.IsdfSmw(s.n, s.cell) as ctx:
            mu = torch.as_tensor(s.mu_idx, dtype=torch.int64, device="cuda") if on_device else s.mu_idx
            _, rank = ctx.fit(pkg.to_fortran(s.phi), s.n_v, s.n_c, mu)
            assert rank == ref.rank
            ctx.polarizability(s.energies, [0.0])
            ctx.smw(0)
            ys.append(ctx.apply(pkg.to_fortran(x), 0).cpu().numpy())
            if on_device:
                bad = mu.clone()
                bad[2] = s.n_r
                with pytest.raises(pkg.IsdfError, match="ISDF_ERR_INDEX"):
                    ctx.fit(pkg.to_fortran(s.phi), s.n_v, s.n_c, bad)
    assert np.array_equal(ys[0], ys[1])
    assert rel_fro(ys[1], ref.y) < TOL
