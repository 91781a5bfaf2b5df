"""Pins of the oracle adjoint (oracle/adjoint.py): the screened Coulomb
operator in the ISDF basis against a dense inverse, the gradients against
central finite differences of the forward, and two exact identities.  No
GPU; these pin the oracle before the CUDA adjoint is compared with it."""
import numpy as np
import pytest

import oracle as O
from oracle import adjoint as A
from helpers import rel_fro, small_system


def _setup(omega=0.0, n=8, n_v=2, n_c=6, n_mu=12, seed_index=61):
    s = small_system(n, n_v, n_c, n_mu=n_mu, seed_index=seed_index)
    theta, rank = O.isdf_fit(s.phi, n_v, s.mu_idx)
    assert rank == n_mu
    g = O.coulomb_in_basis(theta, s.n, s.cell)
    phi_mu = s.phi[np.asarray(s.mu_idx)].copy()
    pj = A.random_projector(n_mu, seed=13)
    return s, theta, g, phi_mu, pj


def test_screened_basis_equals_dense_inverse():
    """G + G K G = Theta^T eps_hat^-1 V Theta with eps_hat formed densely from
    M_hat = Theta C (first display of the SMW section) and inverted by LU."""
    for omega in (0.0, 0.4):
        s, theta, g, phi_mu, _ = _setup(omega)
        b = O.polarizability(phi_mu, s.energies, s.n_v, omega)
        w_p = A.screened_coulomb_basis(g, b)
        m_hat = theta @ O.pair_matrix(phi_mu, s.n_v)
        eps_hat = O.eps_dense(s.phi, s.energies, s.n_v, s.n, s.cell, omega=omega, m=m_hat)
        w_dense = np.linalg.solve(eps_hat, O.coulomb_dense(s.n, s.cell))
        assert rel_fro(w_p, theta.T @ w_dense @ theta) < 1e-11


@pytest.mark.parametrize("omega", [0.0, 0.3])
def test_gradients_match_central_differences(omega):
    s, _, g, phi_mu, pj = _setup(omega)
    ge, gphi = A.screened_loss_grad(g, phi_mu, s.energies, s.n_v, pj.T, omega)
    h = 1e-6

    def loss(e, p):
        return A.screened_loss(g, p, e, s.n_v, pj, omega)

    fe = np.empty_like(ge)
    for i in range(len(s.energies)):
        ep, em = s.energies.copy(), s.energies.copy()
        ep[i] += h
        em[i] -= h
        fe[i] = (loss(ep, phi_mu) - loss(em, phi_mu)) / (2 * h)
    fphi = np.empty_like(gphi)
    for a in range(phi_mu.shape[0]):
        for i in range(phi_mu.shape[1]):
            pp, pm = phi_mu.copy(), phi_mu.copy()
            pp[a, i] += h
            pm[a, i] -= h
            fphi[a, i] = (loss(s.energies, pp) - loss(s.energies, pm)) / (2 * h)
    assert rel_fro(ge, fe) < 1e-6
    assert rel_fro(gphi, fphi) < 1e-6


def test_translation_and_euler_identities():
    """Omega depends on e_v - e_c only, so sum_i dL/de_i = 0 (any w).  At
    w = 0, D is homogeneous of degree 4 in phi_mu and of degree -1 in the
    energies, so sum phi_mu * dL/dphi_mu = 4 <dL/dD, D> = -4 sum e * dL/de."""
    for omega in (0.0, 0.25):
        s, _, g, phi_mu, pj = _setup(omega, seed_index=62)
        ge, gphi = A.screened_loss_grad(g, phi_mu, s.energies, s.n_v, pj, omega)
        assert abs(ge.sum()) < 1e-12 * np.abs(ge).sum()
        if omega == 0.0:
            lhs = float(np.sum(phi_mu * gphi))
            rhs = -4.0 * float(np.dot(s.energies, ge))
            assert abs(lhs - rhs) < 1e-11 * abs(rhs)


def test_projector_is_a_symmetric_projector():
    pj = A.random_projector(10, seed=13)
    assert np.allclose(pj, pj.T, atol=1e-15)
    assert np.allclose(pj @ pj, pj, atol=1e-14)
    assert abs(np.trace(pj) - 5) < 1e-12


# ---- through the fit: dL/dPhi over the whole grid -----------------------

def _fit_case(omega, seed_index=63):
    s = small_system((5, 6, 7), 2, 4, n_mu=7, seed_index=seed_index)
    pj = A.random_projector(7, seed=13)
    return s, pj


@pytest.mark.parametrize("omega", [0.0, 0.3])
def test_fit_gradients_match_central_differences(omega):
    """Every entry of dL/dPhi (grid rows and point rows) and dL/de of
    L(Phi, e) = tr(W_P Pj), with P refitted for every perturbed Phi."""
    s, pj = _fit_case(omega)
    ge, gphi = A.fit_loss_grad(s.phi, s.energies, s.n_v, s.mu_idx, s.n, s.cell, pj, omega)
    h = 1e-6

    def loss(p, e):
        return A.fit_loss(p, e, s.n_v, s.mu_idx, s.n, s.cell, pj, omega)

    fphi = np.empty_like(gphi)
    for a in range(s.phi.shape[0]):
        for i in range(s.phi.shape[1]):
            pp, pm = s.phi.copy(), s.phi.copy()
            pp[a, i] += h
            pm[a, i] -= h
            fphi[a, i] = (loss(pp, s.energies) - loss(pm, s.energies)) / (2 * h)
    fe = np.empty_like(ge)
    for i in range(len(ge)):
        ep, em = s.energies.copy(), s.energies.copy()
        ep[i] += h
        em[i] -= h
        fe[i] = (loss(s.phi, ep) - loss(s.phi, em)) / (2 * h)
    assert rel_fro(gphi, fphi) < 1e-6
    assert rel_fro(ge, fe) < 1e-6
    # the grid rows away from the points carry gradient only through P
    off = np.setdiff1d(np.arange(s.phi.shape[0]), np.asarray(s.mu_idx))
    assert np.abs(gphi[off]).max() > 1e-3 * np.abs(gphi).max()


def test_fit_gradient_scale_identity():
    """P = Z A^-1 is unchanged when Phi is scaled (Z and A both scale with
    the fourth power), so only D carries the scaling: at w = 0,
    sum Phi * dL/dPhi = -4 sum e * dL/de, and the part through P alone sums
    to zero."""
    s, pj = _fit_case(0.0, seed_index=64)
    ge, gphi = A.fit_loss_grad(s.phi, s.energies, s.n_v, s.mu_idx, s.n, s.cell, pj, 0.0)
    lhs = float(np.sum(s.phi * gphi))
    rhs = -4.0 * float(np.dot(s.energies, ge))
    assert abs(lhs - rhs) < 1e-10 * abs(rhs)
    theta, _ = O.isdf_fit(s.phi, s.n_v, s.mu_idx)
    g = O.coulomb_in_basis(theta, s.n, s.cell)
    pm = s.phi[np.asarray(s.mu_idx)]
    _, gpm = A.screened_loss_grad(g, pm, s.energies, s.n_v, pj, 0.0)
    through_p = float(np.sum(s.phi * gphi) - np.sum(pm * gpm))
    assert abs(through_p) < 1e-10 * float(np.abs(s.phi * gphi).sum())
