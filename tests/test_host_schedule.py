"""Host logic of the mixed capacitance route, checked on the CPU through the
C ABI: the bounds of the pair weights, which bound the spectrum of D(w)
(Eq. COmegaCstar), and the Newton-Schulz schedule for (I + G D)^-1 of the
capacitance K = -D (I + G D)^-1 (Algorithm 3 step 3).

The schedule is checked against the iteration itself.  On an eigenvector of
M = I + G D with eigenvalue lam, X_k acts as the scalar x_k, so X <- beta
(2 X - X (M X)) is y <- beta y (2 - y) for y = lam x.  It must take every
y_0 = lam alpha, lam in [1, kappa], to within 2^-26 of 1, and it must do so
in no more steps than it needs."""
import ctypes

import numpy as np
import pytest

import paper_2403_12340_gb300 as pkg

ERR_ARG, ERR_ORDER = -1, -5


@pytest.fixture(scope="module", autouse=True)
def lib():
    import os

    if not os.path.exists(pkg.LIB_PATH):
        from paper_2403_12340_gb300 import build

        build.build()
    return pkg.load_library()


def pair_weights(energies, n_v, w):
    """Every pair weight 2 d / (d^2 + w^2), d = e_c - e_v, by brute force."""
    e = np.asarray(energies, dtype=np.float64)
    d = (e[n_v:][None, :] - e[:n_v][:, None]).ravel()
    return 2.0 * d / (d * d + w * w)


@pytest.mark.parametrize("seed", range(6))
def test_pair_weight_bounds_bracket_every_pair(seed):
    rng = np.random.default_rng(seed)
    n_v, n_c = int(rng.integers(1, 9)), int(rng.integers(1, 30))
    occ = -rng.uniform(0.2, 2.0, n_v)
    unocc = rng.uniform(0.05, 3.0, n_c)
    energies = np.concatenate([occ, unocc])
    gap, width = unocc.min() - occ.max(), unocc.max() - occ.min()
    # below the gap, inside [gap, width] (the weight's peak at d = w), above
    for w in (0.0, 0.5 * gap, 0.5 * (gap + width), 3.0 * width):
        wmin, wmax = pkg.pair_weight_bounds(energies, n_v, n_c, w)
        f = pair_weights(energies, n_v, w)
        # the extreme pairs exist, so the lower bound is attained
        assert wmin == pytest.approx(f.min(), rel=1e-14)
        assert f.max() <= wmax * (1 + 1e-14)
        if not gap <= w <= width:
            assert wmax == pytest.approx(f.max(), rel=1e-14)
        else:
            assert wmax == pytest.approx(1.0 / w, rel=1e-14)  # the peak value 2 w / (2 w^2)


def test_pair_weight_bounds_argument_errors():
    lib = pkg.load_library()
    e = np.array([-1.0, 0.5, 2.0])
    lo, hi = ctypes.c_double(), ctypes.c_double()
    assert lib.isdf_pair_weight_bounds(e.ctypes.data, 1, 2, -0.1, ctypes.byref(lo), ctypes.byref(hi)) == ERR_ARG
    bad = np.array([1.0, 0.5, 2.0])  # occupied above an unoccupied energy
    assert lib.isdf_pair_weight_bounds(bad.ctypes.data, 1, 2, 0.0, ctypes.byref(lo), ctypes.byref(hi)) == ERR_ORDER
    assert lib.isdf_pair_weight_bounds(None, 1, 2, 0.0, ctypes.byref(lo), ctypes.byref(hi)) == ERR_ARG


def run_schedule(kappa, beta, lam):
    """y_k for every eigenvalue in lam, after each step."""
    y = lam * (2.0 / (1.0 + kappa))
    out = []
    for b in beta:
        y = b * y * (2.0 - y)
        out.append(y.copy())
    return out


KAPPAS = [1.0, 1.0 + 1e-9, 1.5, 3.0, 10.0, 137.0, 1e3, 2e4, 1e5]


@pytest.mark.parametrize("kappa", KAPPAS)
def test_ns_schedule_reaches_the_bound_on_the_whole_spectrum(kappa):
    plan = pkg.ns_schedule(kappa)
    assert plan is not None
    beta, slices = plan
    assert 1 <= len(beta) <= 12
    lam = np.concatenate([np.geomspace(1.0, kappa, 2001), [1.0, kappa, np.sqrt(kappa)]]) if kappa > 1 else np.ones(1)
    ys = run_schedule(kappa, beta, lam)
    assert np.max(np.abs(1.0 - ys[-1])) < 2.0**-26
    if len(beta) > 1:
        # no step too many: before the last one some eigenvalue was still off
        assert np.max(np.abs(1.0 - ys[-2])) >= 2.0**-26
    # slices: one to three, never fewer as the error shrinks, three at the end
    assert set(slices.tolist()) <= {1, 2, 3}
    assert np.all(np.diff(slices) >= 0)
    assert slices[-1] == 3 and (len(slices) < 2 or slices[-2] == 3)


@pytest.mark.parametrize("kappa", KAPPAS[1:])
def test_ns_schedule_error_is_symmetric_and_squares(kappa):
    """After each step the error 1 - y spans [-e, e] with the next e =
    e^2 / (2 - e^2): the ends of the spectrum land on +e, its midpoint
    (1 + kappa) / 2, where y_0 = 1, on -e."""
    beta, _ = pkg.ns_schedule(kappa)
    lam = np.concatenate([np.geomspace(1.0, kappa, 4001), [0.5 * (1.0 + kappa)]])
    e = (kappa - 1.0) / (kappa + 1.0)
    for y in run_schedule(kappa, beta, lam):
        e = e * e / (2.0 - e * e)
        err = 1.0 - y
        assert err.max() <= e * (1 + 1e-9) + 1e-15
        assert err.min() >= -e * (1 + 1e-9) - 1e-15
        assert max(err.max(), -err.min()) == pytest.approx(e, rel=1e-6, abs=1e-15)


@pytest.mark.parametrize("kappa", [1e6, 1e8, 1e12])
def test_ns_schedule_declines_when_twelve_steps_are_not_enough(kappa):
    assert pkg.ns_schedule(kappa) is None
    # twelve steps of the best-scaled iteration leave the spectrum's ends off
    e = (kappa - 1.0) / (kappa + 1.0)
    for _ in range(12):
        e = e * e / (2.0 - e * e)
    assert e > 2.0**-26


def test_ns_schedule_argument_errors():
    lib = pkg.load_library()
    b = np.zeros(12)
    s = np.zeros(12, dtype=np.int32)
    assert lib.isdf_ns_schedule(0.5, 12, b.ctypes.data, s.ctypes.data) == ERR_ARG
    assert lib.isdf_ns_schedule(float("nan"), 12, b.ctypes.data, s.ctypes.data) == ERR_ARG
    assert lib.isdf_ns_schedule(1e3, 2, b.ctypes.data, s.ctypes.data) == ERR_ARG  # no room for its 9 steps
    assert lib.isdf_ns_schedule(1e3, 12, None, s.ctypes.data) == ERR_ARG
