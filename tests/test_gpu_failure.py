"""Failure detection on the GPU without a GPU fault: a device-side wait that
runs out.  isdf_check_device_wait runs the library's bounded grid barrier
(the wait of the pivoted factorisation's cooperative kernel) on a barrier
that nothing completes; the kernel must give up after its limit and return,
the call must report ISDF_ERR_TIMEOUT, and the context must stay usable for
a full solve afterwards (checked against the oracle)."""
import time

import pytest

import oracle as O
import synth
from helpers import rel_fro, small_system

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2403_12340_gb300 as p

    p.load_library()
    return p


@pytest.mark.parametrize("limit_ns", [10_000, 1_000_000, 50_000_000])
def test_device_wait_runs_out_and_context_survives(pkg, limit_ns):
    s = small_system((12, 10, 14), 4, 9, 30, seed_index=8)
    x = synth.probe_block(s.n_r, 3)
    with pkg.IsdfSmw(s.n, s.cell) as ctx:
        t0 = time.perf_counter()
        rc = pkg.isdf_check_device_wait(ctx.ctx, limit_ns)
        dt = time.perf_counter() - t0
        assert rc == -7, pkg.isdf_last_error(ctx.ctx)
        assert "timed out" in pkg.isdf_last_error(ctx.ctx)
        assert dt >= limit_ns * 1e-9 and dt < limit_ns * 1e-9 + 2.0
        # the same context solves normally afterwards; a second timeout too
        ctx.fit(pkg.to_fortran(s.phi), s.n_v, s.n_c, s.mu_idx)
        ctx.polarizability(s.energies, [0.0])
        ctx.smw(0)
        y = ctx.apply(pkg.to_fortran(x), 0).cpu().numpy()
        assert pkg.isdf_check_device_wait(ctx.ctx, limit_ns) == -7
        y2 = ctx.apply(pkg.to_fortran(x), 0).cpu().numpy()
    ref = O.isdf_smw_solve(s.phi, s.energies, s.n_v, s.mu_idx, s.n, s.cell, x)
    assert rel_fro(y, ref.y) < 1e-10
    assert rel_fro(y2, ref.y) < 1e-10


def test_device_wait_argument_checks(pkg):
    with pkg.IsdfSmw((8, 8, 8), (4.0, 4.0, 4.0)) as ctx:
        assert pkg.isdf_check_device_wait(ctx.ctx, 10) == -1
        assert pkg.isdf_check_device_wait(ctx.ctx, 10**11) == -1
