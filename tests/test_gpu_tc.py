"""The split-precision tensor-core GEMM (isdf_dgemm_split, tcgen05) against a
plain float64 product, on ragged shapes, several slice counts and long K
(split-K with FP64 reduction).  The bound is relative to |A| |B|^T, the
scale of the rounding of each product."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

BOUND = {1: 2e-2, 2: 1e-4, 3: 2e-6}


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2403_12340_gb300 as p

    p.load_library()
    return p


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (200, 130, 100), (1, 1, 1), (300, 7, 513), (1000, 600, 4096),
                                   (257, 129, 20000)])
@pytest.mark.parametrize("s", [1, 2, 3])
def test_dgemm_split_matches_fp64(pkg, M, N, K, s):
    import torch

    rng = np.random.default_rng(M * 7 + N * 3 + K + s)
    a = rng.standard_normal((M, K)) * np.exp(rng.uniform(-3, 3, (M, 1)))
    b = rng.standard_normal((N, K))
    c0 = rng.standard_normal((M, N))
    A, B, C = pkg.to_fortran(a), pkg.to_fortran(b), pkg.to_fortran(c0)
    pkg.isdf_dgemm_split(A, B, C, alpha=0.75, beta=-0.5, nslices=s)
    torch.cuda.synchronize()
    ref = 0.75 * a @ b.T - 0.5 * c0
    scale = 0.75 * np.abs(a) @ np.abs(b).T + 0.5 * np.abs(c0)
    err = np.abs(C.cpu().numpy() - ref) / scale
    assert err.max() < BOUND[s], err.max()


def test_dgemm_split_zero_k_and_errors(pkg):
    import torch

    A = pkg.to_fortran(np.ones((4, 1)))
    B = pkg.to_fortran(np.ones((3, 1)))
    C = pkg.to_fortran(np.full((4, 3), 2.0))
    pkg.isdf_dgemm_split(A, B, C, alpha=1.0, beta=0.5, nslices=3)
    torch.cuda.synchronize()
    assert np.allclose(C.cpu().numpy(), 1.0 + 1.0)
    with pytest.raises(pkg.IsdfError, match="ISDF_ERR_ARG"):
        pkg.isdf_dgemm_split(A, B, C, nslices=4)
