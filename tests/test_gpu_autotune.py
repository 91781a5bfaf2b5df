"""The tile autotuner of the tensor-core GEMMs (isdf_set_autotune): timed
choices and the forced narrow tiles (64 wide, 16 for a B of at most 16
columns) both keep the mixed path within its
bound against the FP64 oracle, the table records valid choices, and a tuned
shape gives the same result on every later call.  The table is process-wide,
so every test leaves the tuner off and the table empty."""
import numpy as np
import pytest

import oracle as O
import synth
from gpu_helpers import run_gpu
from helpers import rel_fro, small_system

pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-6


@pytest.fixture()
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2403_12340_gb300 as p

    p.load_library()
    p.isdf_autotune_clear()
    yield p
    p.isdf_set_autotune(0)
    p.isdf_autotune_clear()


def _check_table(table, forced):
    assert table
    for t in table:
        assert t["bn"] in (16, 64, 128)
        if t["bn"] == 16:  # 128 x 16 tiles only for a B of at most 16 columns
            assert t["N"] <= 16 and not t["lower"]
        assert 1 <= t["splits"] <= max(1, t["max_split"])
        # the accumulation-length minimum holds for every choice that may split
        if t["max_split"] > 1:
            assert t["splits"] >= min(t["max_split"], -(-t["Kp"] // 64 // 128))
        if t["lower"]:
            assert t["bn"] == 128
        if forced:
            assert t["bn"] == (128 if t["lower"] else (16 if t["N"] <= 16 else 64))
        else:
            assert t["ms_best"] <= t["ms_heuristic"] + 1e-6


@pytest.mark.parametrize("mode", [1, 2])
def test_autotuned_mixed_solve_matches_oracle(pkg, mode):
    s = small_system((24, 24, 24), 8, 40, 200, seed_index=93)
    x = synth.probe_block(s.n_r, 4)
    omegas = (0.0, 0.5)
    pkg.isdf_set_autotune(mode)
    g1 = run_gpu(s, x, omegas, prec=1)
    table = pkg.isdf_autotune_table()
    _check_table(table, forced=(mode == 2))
    if mode == 2:
        assert any(t["bn"] == 64 for t in table)
    g2 = run_gpu(s, x, omegas, prec=1)  # every shape now from the table
    assert len(pkg.isdf_autotune_table()) == len(table)
    for k, w in enumerate(omegas):
        ref = O.isdf_smw_solve(s.phi, s.energies, s.n_v, s.mu_idx, s.n, s.cell, x, omega=w)
        assert rel_fro(g1["y"][k], ref.y) < TOL_MIXED, (k, mode)
        assert np.array_equal(g1["y"][k], g2["y"][k]), (k, mode)


@pytest.mark.parametrize("M,N,K", [(200, 130, 100), (1000, 600, 4096), (257, 129, 20000), (300, 7, 513)])
def test_narrow_tiles_dgemm_split(pkg, M, N, K):
    """isdf_dgemm_split with the narrow tiles forced (64 wide; 16 for N <= 16),
    against float64."""
    import torch

    pkg.isdf_set_autotune(2)
    rng = np.random.default_rng(M + 3 * N + 7 * K)
    a = rng.standard_normal((M, K))
    b = rng.standard_normal((N, K))
    c0 = rng.standard_normal((M, N))
    A, B, C = pkg.to_fortran(a), pkg.to_fortran(b), pkg.to_fortran(c0)
    pkg.isdf_dgemm_split(A, B, C, alpha=0.75, beta=-0.5, nslices=3)
    torch.cuda.synchronize()
    ref = 0.75 * a @ b.T - 0.5 * c0
    scale = 0.75 * np.abs(a) @ np.abs(b).T + 0.5 * np.abs(c0)
    assert (np.abs(C.cpu().numpy() - ref) / scale).max() < 2e-6
    assert any(t["bn"] == (16 if N <= 16 else 64) for t in pkg.isdf_autotune_table())


def test_autotune_off_records_nothing(pkg):
    s = small_system((12, 10, 14), 4, 9, 30, seed_index=94)
    x = synth.probe_block(s.n_r, 2)
    assert pkg.isdf_set_autotune(0) == 0
    run_gpu(s, x, (0.0,), prec=1)
    assert pkg.isdf_autotune_table() == []
