"""The solid-sized case (72^3 grid, N_r = 373248, N_v = 256, N_c = 1792,
N_mu = 6144): the mixed path against an FP64 run of the CUDA path on the
same GPU, which is the reference at this size (the FP64 path itself is
checked against the oracle on the smaller systems).  About 7e13 algorithmic
flops per solve; the FP64 run takes about 50 s.

Tolerance: 1e-6 relative Frobenius on eps^-1 X (16 probes), the stated
bound of the mixed path.  The points are QRCP pivots of the Gaussian
face-split sketch over 2 N_mu seeded candidate points (cond(C C^T) = 9.4);
the fit's FP32-grade face-split Gram enters theta through L_r^-1, so the
error of the mixed path grows with cond(L_r) and uniformly random points
(cond(C C^T) = 531) would not meet the bound."""
import time

import numpy as np
import pytest

import synth
from helpers import rel_fro

pytestmark = pytest.mark.gpu


def _solve(s, x, prec):
    import torch
    import paper_2403_12340_gb300 as pkg

    phi = pkg.to_fortran(s.phi)
    X = pkg.to_fortran(x)
    torch.cuda.synchronize()
    times = {}
    with pkg.IsdfSmw(s.n, s.cell) as sol:
        t0 = time.perf_counter()
        _, rank = sol.fit(phi, s.n_v, s.n_c, s.mu_idx, prec=prec)
        torch.cuda.synchronize()
        times["fit"] = time.perf_counter() - t0
        t0 = time.perf_counter()
        sol.polarizability(s.energies, [0.0])
        torch.cuda.synchronize()
        times["polar"] = time.perf_counter() - t0
        t0 = time.perf_counter()
        sol.smw(0)
        times["smw"] = time.perf_counter() - t0
        t0 = time.perf_counter()
        Y = sol.apply(X, 0)
        torch.cuda.synchronize()
        times["apply"] = time.perf_counter() - t0
        y = Y.cpu().numpy()
    del phi, X, Y
    torch.cuda.empty_cache()
    return y, rank, times


def test_config3_mixed_against_fp64_gpu():
    s = synth.workload("isdf72")
    x = synth.probe_block(s.n_r, 16)
    y_mixed, r1, t1 = _solve(s, x, 1)
    y_fp64, r0, t0 = _solve(s, x, 0)
    err = rel_fro(y_mixed, y_fp64)
    print(f"\n72^3 N_mu=6144: rank {r0} / {r1}; mixed {t1} s; fp64 {t0} s; rel err mixed vs fp64 {err:.3e}")
    assert r0 == r1 == len(s.mu_idx)
    assert err < 1e-6
