"""Plain FP64 oracle of the adjoint of ISDF-SMW (TEST INFRASTRUCTURE: only the
tests, the smoke check and the benchmark's CPU legs import it).

The differentiated quantity is the screened Coulomb operator in the ISDF
basis, W_P = P^T eps_hat^-1 V P with P = Theta the interpolation vectors of
the fit (Eq. ISDF), which Eq. epsilon_with_SMW turns into
    W_P = G + G K G,   G = Theta^T V Theta,   K = -D (I + G D)^-1,
    D = -2 B = -2 C Omega^-1 C^T = sum_p d_p c_p c_p^T,  d_p = -2 Omega_p^-1,
with c_p the column of C = M[mu, :] of the pair p = (v, c) (Eq.
MatrixExpressionISDF, Eq. COmegaCstar).  Theta is held fixed (checkpointed):
the gradients are those of W_P with respect to the orbital energies and the
orbital samples at the interpolation points, phi_mu = Phi[mu, :], through
D alone.

Chain rule, each step from the derivative of an inverse,
d(A^-1) = -A^-1 dA A^-1:
    E  = (I + G D)^-1                       (so E = I + G K)
    dK = -E^T dD E                          (K = -D E, dE = -E G dD E)
    dL/dK = G Wbar G                        (dL/dW_P = Wbar, G symmetric)
    dL/dD = -E (dL/dK) E^T
    dL/dd_p = c_p^T (dL/dD) c_p
    dL/dC   = (dL/dD + dL/dD^T) C diag(d)
    dd_p/de_v = -2 (w^2 - Delta^2) / (Delta^2 + w^2)^2 = -dd_p/de_c,
        Delta = e_v - e_c, Omega(i w)^-1 = Delta / (Delta^2 + w^2)
    dL/dphi_v(a) = sum_c dL/dC(a, vc) phi_c(a),
    dL/dphi_c(a) = sum_v dL/dC(a, vc) phi_v(a).
For the loss L = tr(W_P Pj) of a symmetric projector Pj, Wbar = Pj^T = Pj.

Pinned by tests/test_oracle_adjoint.py against central finite differences of
the forward, translation invariance in the energies and Euler's identity
for the homogeneity of D in phi_mu.
"""
from __future__ import annotations

from typing import Tuple

import numpy as np

from .isdf_oracle import (apply_coulomb, capacitance, coulomb_in_basis, isdf_fit, omega_inverse, pair_matrix,
                          polarizability)

__all__ = ["screened_coulomb_basis", "screened_loss", "screened_loss_grad", "random_projector", "fit_loss",
           "fit_loss_grad"]


def screened_coulomb_basis(g: np.ndarray, b: np.ndarray) -> np.ndarray:
    """W_P = Theta^T eps_hat^-1 V Theta = G + G K G (Eq. epsilon_with_SMW
    times V, projected on the ISDF basis)."""
    k = capacitance(g, b)
    return g + g @ k @ g


def screened_loss(g: np.ndarray, phi_mu: np.ndarray, energies: np.ndarray, n_v: int, pj: np.ndarray,
                  omega: float = 0.0) -> float:
    """L = tr(W_P Pj) with W_P from the orbital samples at the points."""
    b = polarizability(phi_mu, energies, n_v, omega)
    return float(np.trace(screened_coulomb_basis(g, b) @ pj))


def screened_loss_grad(g: np.ndarray, phi_mu: np.ndarray, energies: np.ndarray, n_v: int, wbar: np.ndarray,
                       omega: float = 0.0) -> Tuple[np.ndarray, np.ndarray]:
    """(dL/de, dL/dphi_mu) for the upstream gradient wbar = dL/dW_P."""
    n = g.shape[0]
    n_e = phi_mu.shape[1]
    n_c = n_e - n_v
    c = pair_matrix(phi_mu, n_v)                       # N_mu x pairs, p = v n_c + c
    w_inv = omega_inverse(energies, n_v, omega)        # Omega^-1 per pair (< 0)
    d_p = -2.0 * w_inv
    dmat = (c * d_p[None, :]) @ c.T                    # D = -2 B
    kmat = capacitance(g, -0.5 * dmat)
    e = np.linalg.inv(np.eye(n) + g @ dmat)            # E = (I + G D)^-1
    kbar = g @ wbar @ g                                # dL/dK
    dbar = -e @ kbar @ e.T                             # dL/dD
    dsym = dbar + dbar.T
    grad_d = np.sum(c * (dbar @ c), axis=0)            # c_p^T dbar c_p
    cbar = (dsym @ c) * d_p[None, :]                   # dL/dC
    ev = energies[:n_v]
    ec = energies[n_v:]
    delta = (ev[:, None] - ec[None, :]).reshape(-1)
    w2 = omega * omega
    dd_ddelta = -2.0 * (w2 - delta * delta) / (delta * delta + w2) ** 2
    gp = (grad_d * dd_ddelta).reshape(n_v, n_c)
    grad_e = np.concatenate([gp.sum(axis=1), -gp.sum(axis=0)])
    cb = cbar.reshape(-1, n_v, n_c)
    grad_phi = np.empty_like(phi_mu)
    grad_phi[:, :n_v] = np.einsum("avc,ac->av", cb, phi_mu[:, n_v:])
    grad_phi[:, n_v:] = np.einsum("avc,av->ac", cb, phi_mu[:, :n_v])
    del kmat
    return grad_e, grad_phi


def random_projector(n: int, seed: int = 13) -> np.ndarray:
    """Pj = Q Q^T with Q an orthonormal basis of an n x (n/2) Gaussian."""
    rng = np.random.default_rng(seed)
    q, _ = np.linalg.qr(rng.standard_normal((n, n // 2)))
    return q @ q.T


# ---------------------------------------------------------------------------
# Through the fit: L as a function of the orbitals on the whole grid.
#
# P is now the least-squares ISDF vectors of Phi itself (full rank),
#     P = Z A^-1,  Z = M C^T = Zv .* Zc,  A = C C^T = Av .* Ac,
#     Zv = Phi_v Phi_v,mu^T, Zc = Phi_c Phi_c,mu^T, Av = Phi_v,mu Phi_v,mu^T,
#     Ac = Phi_c,mu Phi_c,mu^T (Eq. MatrixExpressionISDF with the Hadamard
#     identity), and G = P^T V P depends on Phi through P.  With
#     W_P = G + G K G = (G^-1 + D)^-1:
#     dL/dG = E^T Wbar E,  E = I + G K           (dW = W G^-1 dG G^-1 W, W G^-1 = E^T)
#     dL/dP = 2 V P dL/dG
#     dL/dZ = dL/dP A^-1,  dL/dA = -sym(A^-1 (dL/dP)^T P)
#     dL/dPhi_v = (dL/dZ .* Zc) Phi_v,mu,  dL/dPhi_v,mu += (dL/dZ .* Zc)^T Phi_v
#         + 2 (dL/dA .* Ac) Phi_v,mu  (and v <-> c),
# and the rows mu of dL/dPhi also collect dL/dphi_mu through D (above).


def fit_loss(phi: np.ndarray, energies: np.ndarray, n_v: int, mu_idx, n, cell, pj: np.ndarray,
             omega: float = 0.0) -> float:
    """L(Phi) = tr(W_P Pj), every step of W_P recomputed from the orbitals."""
    mu = np.asarray(mu_idx)
    p, _ = isdf_fit(phi, n_v, mu)
    g = coulomb_in_basis(p, n, cell)
    b = polarizability(phi[mu], energies, n_v, omega)
    return float(np.trace(screened_coulomb_basis(g, b) @ pj))


def fit_loss_grad(phi: np.ndarray, energies: np.ndarray, n_v: int, mu_idx, n, cell, wbar: np.ndarray,
                  omega: float = 0.0) -> Tuple[np.ndarray, np.ndarray]:
    """(dL/de, dL/dPhi) of L(W_P(Phi, e)) for dL/dW_P = wbar (symmetric),
    dL/dPhi over the whole grid (N_r x N_e).  Needs C C^T of full rank."""
    mu = np.asarray(mu_idx)
    pm = phi[mu]
    p, rank = isdf_fit(phi, n_v, mu)
    if rank != len(mu):
        raise ValueError("fit_loss_grad needs a full-rank C C^T")
    g = coulomb_in_basis(p, n, cell)
    b = polarizability(pm, energies, n_v, omega)
    k = capacitance(g, b)
    e = np.eye(g.shape[0]) + g @ k
    # through D, P held fixed
    grad_e, gpm = screened_loss_grad(g, pm, energies, n_v, wbar, omega)
    # through G and P
    gbar = e.T @ wbar @ e
    pbar = 2.0 * apply_coulomb(p @ gbar, n, cell)
    pv, pc = phi[:, :n_v], phi[:, n_v:]
    pmv, pmc = pm[:, :n_v], pm[:, n_v:]
    av, ac = pmv @ pmv.T, pmc @ pmc.T
    ainv = np.linalg.inv(av * ac)
    zbar = pbar @ ainv
    abar = -ainv @ pbar.T @ p
    abar = 0.5 * (abar + abar.T)
    zv, zc = pv @ pmv.T, pc @ pmc.T
    zbv, zbc = zbar * zc, zbar * zv
    grad_phi = np.zeros_like(phi)
    grad_phi[:, :n_v] = zbv @ pmv
    grad_phi[:, n_v:] = zbc @ pmc
    gpm = gpm.copy()
    gpm[:, :n_v] += zbv.T @ pv + 2.0 * (abar * ac) @ pmv
    gpm[:, n_v:] += zbc.T @ pc + 2.0 * (abar * av) @ pmc
    grad_phi[mu] += gpm
    return grad_e, grad_phi
