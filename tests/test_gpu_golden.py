"""The CUDA path (through the C ABI) against the closed form of the worked
example in tests/golden/plane_wave_two_pairs.txt, with no oracle in between:
eps^-1 X at three imaginary frequencies, FP64 path within 1e-10 and mixed
path within 1e-6, with 2 points (full-rank C C^T) and 6 (rank-deficient).
eps^-1 is close to I in this example, so the correction eps^-1 X - X is
checked on its own as well (1e-9 FP64, 1e-5 mixed)."""
import numpy as np
import pytest

import synth
from gpu_helpers import run_gpu
from helpers import plane_wave_golden, plane_wave_golden_eps_inv, rel_fro

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2403_12340_gb300 as pkg

    pkg.load_library()


@pytest.mark.parametrize("prec,tol,tol_corr", [(0, 1e-10, 1e-9), (1, 1e-6, 1e-5)])
@pytest.mark.parametrize("n_mu", [2, 6])
def test_plane_wave_closed_form(prec, tol, tol_corr, n_mu):
    s, u, g = plane_wave_golden(n_mu)
    x = synth.probe_block(s.n_r, 4)
    omegas = tuple(float(t) for t in g["frequencies"].split())
    out = run_gpu(s, x, omegas, prec=prec)
    assert out["rank"] == 2
    for k, w in enumerate(omegas):
        closed = plane_wave_golden_eps_inv(u, g, x, w)
        err = rel_fro(out["y"][k], closed)
        assert err < tol, (w, err)
        err = rel_fro(out["y"][k] - x, closed - x)
        assert err < tol_corr, (w, err)
