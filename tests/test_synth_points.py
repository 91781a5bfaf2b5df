"""The candidate-set QRCP point generator (synth.qrcp_points_on_candidates):
distinct in-range points, and a C C^T far better conditioned than that of
uniformly random points, close to QRCP over the whole grid.  CPU only."""
import numpy as np

import synth


def _cond(phi, n_v, mu):
    pm = phi[np.asarray(mu)]
    a = (pm[:, :n_v] @ pm[:, :n_v].T) * (pm[:, n_v:] @ pm[:, n_v:].T)
    w = np.linalg.eigvalsh(a)
    return w[-1] / w[0]


def test_candidate_qrcp_points_condition_c_ct():
    n, n_v, n_c, n_mu = (24, 24, 24), 8, 56, 256
    phi = synth.make_orbitals(n, n_v + n_c, 1234)
    n_r = phi.shape[0]
    mu = synth.qrcp_points_on_candidates(phi, n_v, n_mu, 4321)
    assert mu.dtype == np.int64 and mu.shape == (n_mu,)
    assert len(np.unique(mu)) == n_mu and mu.min() >= 0 and mu.max() < n_r
    c_cand = _cond(phi, n_v, mu)
    c_rand = _cond(phi, n_v, synth.random_points(n_r, n_mu, 4321))
    c_full = _cond(phi, n_v, synth.qrcp_points(phi, n_v, n_mu))
    assert c_cand < c_rand / 4
    assert c_cand < 2 * c_full
    # deterministic for the same seeds
    assert np.array_equal(mu, synth.qrcp_points_on_candidates(phi, n_v, n_mu, 4321))
