"""GPU parity of the mixed-precision path (ISDF_PREC_MIXED: split-BF16
tensor-core contractions, FP64 factorisations) against the FP64 oracle.
Tolerance 1e-6 relative Frobenius on eps^-1 X, the stated bound of the
mixed path."""
import numpy as np
import pytest

import oracle as O
import synth
from gpu_helpers import run_gpu
from helpers import rel_fro, small_system

pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-6
MIXED = 1


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


CASES = [
    ((6, 6, 6), 2, 5, 10),
    ((8, 10, 6), 3, 7, 19),
    ((9, 9, 9), 3, 6, 18),
    ((12, 10, 14), 4, 9, 30),
    ((8, 8, 8), 2, 3, 9),        # rank-deficient C C^T
    ((16, 12, 10), 6, 20, 70),
    ((24, 24, 24), 8, 40, 200),  # several 128-row tiles of points
]


@pytest.mark.parametrize("grid,nv,nc,nmu", CASES)
def test_mixed_small_systems_match_oracle(grid, nv, nc, nmu):
    s = small_system(grid, nv, nc, nmu, seed_index=hash((grid, nv, nc)) % 97)
    x = synth.probe_block(s.n_r, 5)
    omegas = (0.0, 0.37)
    g = run_gpu(s, x, omegas, prec=MIXED)
    for k, w in enumerate(omegas):
        ref = O.isdf_smw_solve(s.phi, s.energies, s.n_v, s.mu_idx, s.n, s.cell, x, omega=w)
        assert g["rank"] == ref.rank
        err = rel_fro(g["y"][k], ref.y)
        assert err < TOL_MIXED, (k, err)


def test_mixed_isdf16_against_dense_inverse():
    s = synth.workload("isdf16")
    x = synth.probe_block(s.n_r)
    g = run_gpu(s, x, prec=MIXED)
    assert g["rank"] == 112
    einv = O.eps_inv_dense(s.phi, s.energies, s.n_v, s.n, s.cell)
    assert rel_fro(g["y"][0], einv @ x) < TOL_MIXED


def test_mixed_intermediates_close_to_fp64():
    """theta, G, D, K of the mixed path against the FP64 path on the same
    context inputs (same pivots, same basis)."""
    s = small_system((12, 10, 14), 4, 9, 30, seed_index=5)
    x = synth.probe_block(s.n_r, 3)
    a = run_gpu(s, x, want=True, prec=0)
    b = run_gpu(s, x, want=True, prec=MIXED)
    assert np.array_equal(a["piv"], b["piv"])
    # theta: FP32-grade products; G also carries the FP32 FFT (~1e-6 relative)
    assert rel_fro(b["theta"], a["theta"]) < 1e-6
    assert rel_fro(b["G"], a["G"]) < 1e-5
    # D is whitened with L^-1 on both sides: its error grows with kappa(L)^2
    assert rel_fro(b["D"][0], a["D"][0]) < 1e-5
    assert rel_fro(b["K"][0], a["K"][0]) < 1e-5


@pytest.mark.parametrize("grid,nv,nc,nmu", CASES[:4] + CASES[5:])
def test_mixed_pair_space_whitening_matches_oracle(grid, nv, nc, nmu):
    """ISDF_PREC_MIXED_PAIRS: D whitened in pair space (S = L^-1 C_r diag,
    D = S S^T) on the same systems, two frequencies (the frequency batch)."""
    s = small_system(grid, nv, nc, nmu, seed_index=hash((grid, nv, nc)) % 97)
    x = synth.probe_block(s.n_r, 5)
    omegas = (0.0, 0.37)
    g = run_gpu(s, x, omegas, prec=2)
    for k, w in enumerate(omegas):
        ref = O.isdf_smw_solve(s.phi, s.energies, s.n_v, s.mu_idx, s.n, s.cell, x, omega=w)
        assert rel_fro(g["y"][k], ref.y) < TOL_MIXED, k


def test_mixed_ill_conditioned_points():
    """Uniformly random points give cond(C C^T) in the hundreds: the mixed
    path then whitens in pair space by itself and stays within 1e-6."""
    s = small_system((20, 20, 20), 8, 40, 160, seed_index=33)
    s.mu_idx = synth.random_points(s.n_r, 160, 77)
    x = synth.probe_block(s.n_r, 5)
    g = run_gpu(s, x, prec=MIXED)
    ref = O.isdf_smw_solve(s.phi, s.energies, s.n_v, s.mu_idx, s.n, s.cell, x)
    assert g["rank"] == ref.rank
    assert rel_fro(g["y"][0], ref.y) < TOL_MIXED


def test_mixed_smw_refinement():
    """isdf_set_refinement: rounds of FP64 residual correction of the SMW
    solve in the mixed single-frequency apply.  With 1 and 2 rounds eps^-1 X
    stays within the mixed bound of the oracle and within 1e-6 of the
    unrefined result (the Newton-Schulz K is already close to the exact
    solve with the same D and G); 65 probe vectors cover two apply chunks.
    Out-of-range round counts are refused."""
    import torch
    import paper_2403_12340_gb300 as pkg

    s = small_system(24, 8, 40, n_mu=200, seed_index=61)
    x = synth.probe_block(s.n_r, 65)
    ref = O.isdf_smw_solve(s.phi, s.energies, s.n_v, s.mu_idx, s.n, s.cell, x)
    ys = {}
    with pkg.IsdfSmw(s.n, s.cell) as sol:
        sol.fit(pkg.to_fortran(s.phi), s.n_v, s.n_c, s.mu_idx, prec=MIXED)
        sol.polarizability(s.energies, [0.0])
        sol.smw(0)
        X = pkg.to_fortran(x)
        for steps in (0, 1, 2):
            pkg.isdf_set_refinement(sol.ctx, steps)
            ys[steps] = sol.apply(X, 0).cpu().numpy()
        for bad in (-1, 9):
            with pytest.raises(pkg.IsdfError) as ei:
                pkg.isdf_set_refinement(sol.ctx, bad)
            assert ei.value.code == -1
        torch.cuda.synchronize()
    for steps, y in ys.items():
        assert rel_fro(y, ref.y) < TOL_MIXED, steps
    assert rel_fro(ys[1], ys[0]) < 1e-6
    assert rel_fro(ys[2], ys[1]) < 1e-6
