"""apply_eps_inv_noalloc: the apply step for callers that must not allocate
device memory when they call (fixed memory budgets, latency-critical loops
where an allocation could synchronise the device).  Its scratch is a static
device array inside the library.  Checked against apply_eps_inv on the same
context, on two calls in a row, through the C ABI; that the calls allocate
nothing is read from the library's own allocation count.

The file name sorts last so that a run stopping at the first failure has
already run every other test."""
import ctypes

import numpy as np
import pytest

import synth
from helpers import rel_fro, small_system

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2403_12340_gb300 as p

    p.load_library()
    return p


def _noalloc(pkg, ctx, k, X, Y):
    lib = pkg.load_library()
    n_rhs = X.shape[1]
    rc = lib.apply_eps_inv_noalloc(ctx.ctx, k, ctypes.c_void_p(X.data_ptr()), n_rhs,
                                   ctypes.c_void_p(Y.data_ptr()))
    return rc, pkg.isdf_last_error(ctx.ctx)


CASES = [  # grid, n_v, n_c, n_mu, n_rhs, precision of the context
    ((16, 12, 10), 6, 20, 70, 5, 0),
    ((24, 24, 24), 8, 40, 160, 16, 0),
    # 40^3: seven probe columns fit the pool at a time, so 17 columns run
    # as chunks of 7, 7 and 3 (offsets into X and Y, the pool reused, a
    # short last chunk)
    ((40, 40, 40), 4, 10, 40, 17, 0),
    # a mixed-precision context: the allocation-free apply runs its FP64
    # kernels on that context's theta and K, apply_eps_inv its tensor-core
    # products, so they agree to the mixed path's bound
    ((24, 24, 24), 8, 40, 160, 16, 1),
]


@pytest.mark.parametrize("grid,nv,nc,nmu,nrhs,prec", CASES)
def test_noalloc_apply_matches_apply_twice(pkg, grid, nv, nc, nmu, nrhs, prec):
    import torch

    tol = TOL if prec == 0 else 1e-6
    s = small_system(grid, nv, nc, nmu, seed_index=31)
    x = synth.probe_block(s.n_r, nrhs)
    with pkg.IsdfSmw(s.n, s.cell) as ctx:
        ctx.fit(pkg.to_fortran(s.phi), s.n_v, s.n_c, s.mu_idx, prec=prec)
        ctx.polarizability(s.energies, [0.0, 0.5])
        ctx.smw(0)
        ctx.smw(1)
        X = pkg.to_fortran(x)
        for k in (0, 1):
            y_ref = ctx.apply(X, k).cpu().numpy()
            outs = [pkg.fortran_empty(s.n_r, nrhs) for _ in range(2)]
            for Y in outs:
                Y.fill_(float("nan"))
            torch.cuda.synchronize()
            for call, Y in enumerate(outs):
                allocs0 = pkg.isdf_device_allocations()
                free0 = torch.cuda.mem_get_info()[0]
                rc, msg = _noalloc(pkg, ctx, k, X, Y)
                assert rc == 0, msg
                torch.cuda.synchronize()
                # the library's own count of its device allocations
                assert pkg.isdf_device_allocations() == allocs0
                if call == 1:   # the first call may load the library's module; later ones allocate nothing
                    assert torch.cuda.mem_get_info()[0] == free0  # secondary: device-wide free memory
            for Y in outs:
                assert rel_fro(Y.cpu().numpy(), y_ref) < tol


def test_noalloc_rejects_grids_beyond_its_pool(pkg):
    """One probe column of a 96^3 grid needs more than the 8 MiB pool: a
    clear ISDF_ERR_SHAPE, and the output is left untouched."""
    import torch

    n = (96, 96, 96)
    n_v, n_c = 2, 2
    phi = synth.make_orbitals(n, n_v + n_c, 1099, n_pw=24)
    e = synth.make_energies(n_v, n_c, 2099)
    mu = synth.qrcp_points(phi, n_v, 4)
    cell = tuple(v * synth.GRID_SPACING_BOHR for v in n)
    with pkg.IsdfSmw(n, cell) as ctx:
        ctx.fit(pkg.to_fortran(phi), n_v, n_c, mu)
        ctx.polarizability(e, [0.0])
        ctx.smw(0)
        X = pkg.to_fortran(synth.probe_block(phi.shape[0], 1))
        Y = pkg.fortran_empty(phi.shape[0], 1)
        Y.fill_(7.0)
        rc, msg = _noalloc(pkg, ctx, 0, X, Y)
        assert rc == -2 and "static pool" in msg
        torch.cuda.synchronize()
        assert bool((Y == 7.0).all())
        rc, msg = _noalloc(pkg, ctx, 3, X, Y)
        assert rc == -9
