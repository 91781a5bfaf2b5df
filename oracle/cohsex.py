"""Plain FP64 oracle of the static COHSEX self-energies (TEST INFRASTRUCTURE:
only the tests, the smoke check and the benchmark's CPU legs import it).

Exact form (Section "GW approximation", the matrix form of the band
self-energies of Eq. AllPartSelfEnergies, with W = eps^-1 V and w = 0):
    Sigma_SEX_X(n) = - sum_{i occ} (psi_n .* psi_i)^T (W - V) (psi_n .* psi_i)
    Sigma_X(n)     = - sum_{i occ} (psi_n .* psi_i)^T  V      (psi_n .* psi_i)
    Sigma_COH(n)   = 1/2 sum_{m all} (psi_n .* psi_m)^T (W - V) (psi_n .* psi_m)
ISDF form (Algorithm 3 steps 1-7): three fits, of the pair sets vc (the
dielectric matrix), vn (occupied x all) and nn (all x all), with bases
P_vc, P_vn, P_nn; eps^-1 - I = V P_vc K P_vc^T (Eq. epsilon_with_SMW), so
(W - V) ~ V P_vc K P_vc^T V and, with psi_n .* psi_i ~ P_vn c_ni and
c_ni(mu) = psi_n(r_mu) psi_i(r_mu),
    W_vn = (P_vn^T V P_vc) K (P_vc^T V P_vn),  V_vn = P_vn^T V P_vn,
    W_nn = (P_nn^T V P_vc) K (P_vc^T V P_nn),
and the sums over i collapse by the Hadamard identity (Eq. Hadamard):
    Sigma_SEX_X(n) = - psi_n^T (W_vn .* (Psi_v Psi_v^T)) psi_n   (at the vn points)
    Sigma_X(n)     = - psi_n^T (V_vn .* (Psi_v Psi_v^T)) psi_n   (at the vn points)
    Sigma_COH(n)   = 1/2 psi_n^T (W_nn .* (Psi Psi^T)) psi_n     (at the nn points)
Pinned by tests/test_oracle_cohsex.py: the ISDF form equals the exact form
when every pair set is fitted at full rank, and with a complete orbital set
the COH sum over states equals the local form 1/2 sum_r psi_n(r)^2 (W - V)(r, r)
of Eq. Sigma_G0W0.
"""
from __future__ import annotations

from typing import Tuple

import numpy as np

from .isdf_oracle import (apply_coulomb, capacitance, coulomb_dense, coulomb_in_basis, eps_inv_dense, isdf_fit,
                          polarizability)

__all__ = ["sigma_exact", "sigma_isdf", "pair_phi_vn", "pair_phi_nn"]


def sigma_exact(phi: np.ndarray, energies: np.ndarray, n_v: int, n, cell) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """(SEX_X, X, COH) for every band n from the dense eps^-1 (small grids)."""
    n_r, n_e = phi.shape
    vd = coulomb_dense(n, cell)
    wmv = (eps_inv_dense(phi, energies, n_v, n, cell) - np.eye(n_r)) @ vd
    sex_x = np.zeros(n_e)
    x = np.zeros(n_e)
    coh = np.zeros(n_e)
    for b in range(n_e):
        pv = phi[:, b:b + 1] * phi[:, :n_v]           # psi_n .* psi_i, i occupied
        pa = phi[:, b:b + 1] * phi                    # psi_n .* psi_m, m all
        sex_x[b] = -np.einsum("ri,rs,si->", pv, wmv, pv)
        x[b] = -np.einsum("ri,rs,si->", pv, vd, pv)
        coh[b] = 0.5 * np.einsum("ri,rs,si->", pa, wmv, pa)
    return sex_x, x, coh


def pair_phi_vn(phi: np.ndarray, n_v: int) -> np.ndarray:
    """Orbitals arranged so that the vc fit of this module fits the vn pairs:
    [Phi_v | Phi_all] with n_v 'occupied' columns."""
    return np.asfortranarray(np.concatenate([phi[:, :n_v], phi], axis=1))


def pair_phi_nn(phi: np.ndarray) -> np.ndarray:
    """[Phi_all | Phi_all]: the nn pairs, with n_e 'occupied' columns."""
    return np.asfortranarray(np.concatenate([phi, phi], axis=1))


def sigma_isdf(phi: np.ndarray, energies: np.ndarray, n_v: int, mu_vc, mu_vn, mu_nn, n, cell,
               rcond: float = 1e-13) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """(SEX_X, X, COH) for every band by Algorithm 3 steps 1-7."""
    n_e = phi.shape[1]
    mu_vc, mu_vn, mu_nn = (np.asarray(m) for m in (mu_vc, mu_vn, mu_nn))
    th_vc, _ = isdf_fit(phi, n_v, mu_vc, rcond=rcond)
    th_vn, _ = isdf_fit(pair_phi_vn(phi, n_v), n_v, mu_vn, rcond=rcond)
    th_nn, _ = isdf_fit(pair_phi_nn(phi), n_e, mu_nn, rcond=rcond)
    k = capacitance(coulomb_in_basis(th_vc, n, cell), polarizability(phi[mu_vc], energies, n_v))
    v_vc = apply_coulomb(th_vc, n, cell)
    a_vn = th_vn.T @ v_vc
    a_nn = th_nn.T @ v_vc
    w_vn = a_vn @ k @ a_vn.T
    w_nn = a_nn @ k @ a_nn.T
    v_vn = th_vn.T @ apply_coulomb(th_vn, n, cell)
    psi_vn = phi[mu_vn]
    psi_nn = phi[mu_nn]
    occ_vn = psi_vn[:, :n_v] @ psi_vn[:, :n_v].T
    all_nn = psi_nn @ psi_nn.T
    sex_x = -np.einsum("an,ab,bn->n", psi_vn, w_vn * occ_vn, psi_vn)
    x = -np.einsum("an,ab,bn->n", psi_vn, v_vn * occ_vn, psi_vn)
    coh = 0.5 * np.einsum("an,ab,bn->n", psi_nn, w_nn * all_nn, psi_nn)
    assert sex_x.shape == (n_e,)
    return sex_x, x, coh
