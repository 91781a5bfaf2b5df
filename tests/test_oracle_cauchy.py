"""Pins of the contour-integral polarizability oracle (oracle/cauchy.py,
Algorithm 2): the elliptic functions against SciPy's library routines and
closed forms, the quadrature of the scalar identity 1/(e_v - e_c) against
its exact value (geometric convergence, inside the bound of Eq.
rel_err_Cauchy), and the matrix B against the direct pair sum of Eq.
COmegaCstar."""
import math

import numpy as np
import pytest
import scipy.special as sp

from oracle import cauchy as C
from helpers import rel_fro, small_system


@pytest.mark.parametrize("k", [0.05, 0.5, 0.9, 0.995])
def test_elliptic_functions_match_library_and_closed_forms(k):
    kk = C.ellipk(k)
    assert abs(kk - sp.ellipk(k * k)) < 1e-14 * kk
    for u in (0.0, 0.3, 0.5 * kk, 0.9 * kk, 1.7 * kk, -0.4 * kk):
        s, c, d = C.jacobi_real(u, k)
        S, Cc, D, _ = sp.ellipj(u, k * k)
        assert max(abs(s - S), abs(c - Cc), abs(d - D)) < 1e-14
    # sn(K/2) = 1 / sqrt(1 + k'), and sn(i v, k) = i sc(v, k') (Jacobi imaginary transformation)
    kp = math.sqrt(1 - k * k)
    assert abs(C.jacobi_real(0.5 * kk, k)[0] - 1 / math.sqrt(1 + kp)) < 1e-14
    v = 0.37
    sn, cn, dn = C.jacobi_complex(0.0, v, k)
    s1, c1, d1 = C.jacobi_real(v, kp)
    assert abs(sn - 1j * s1 / c1) < 1e-14 and abs(cn - 1 / c1) < 1e-14 and abs(dn - d1 / c1) < 1e-14


def _energies(seed, n_v=6, n_c=9):
    rng = np.random.default_rng(seed)
    ev = np.sort(rng.uniform(-10, -2, n_v)) / 27.211386245988
    ec = np.sort(rng.uniform(0, 20, n_c)) / 27.211386245988
    return np.concatenate([ev, ec]), n_v


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_scalar_quadrature_converges_to_the_exact_reciprocal(seed):
    e, n_v = _energies(seed)
    errs = []
    for n in (6, 10, 14, 18, 24):
        z, w = C.contour_nodes(e, n_v, n)
        assert np.all(z.imag > 0)
        assert np.all((z - e[:n_v].max()).real > 0)  # the contour stays right of every occupied energy
        err = 0.0
        for a in e[:n_v]:
            for b in e[n_v:]:
                val = (np.sum(w / ((z - a) * (z - b)))).imag / math.pi
                err = max(err, abs(val - 1.0 / (a - b)) * abs(a - b))
        errs.append(err)
        assert err < 50.0 * C.contour_error_bound(e, n_v, n) + 1e-14
    assert errs[-1] < 1e-13
    assert all(e2 < e1 or e2 < 1e-14 for e1, e2 in zip(errs, errs[1:]))


def test_contour_polarizability_equals_direct_pair_sum():
    s = small_system(10, 3, 11, n_mu=24, seed_index=91)
    pm = s.phi[np.asarray(s.mu_idx)]
    ref = C.polarizability_direct(pm, s.energies, s.n_v)
    prev = None
    for n in (8, 12, 16, 24):
        b = C.polarizability_contour(pm, s.energies, s.n_v, n)
        err = rel_fro(b, ref)
        assert err < 50.0 * C.contour_error_bound(s.energies, s.n_v, n) + 1e-14
        if prev is not None:
            assert err < prev or err < 1e-14
        prev = err
    assert prev < 1e-13
    assert np.allclose(b, b.T, atol=1e-15 * np.abs(b).max())
