"""Plain FP64 oracle for ISDF-SMW (arXiv 2403.12340), written from the paper.

TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's CPU
baseline import this module.  It is deliberately slow and direct: numpy /
scipy in float64, library primitives (matmul, FFT, SVD, LU) as single steps,
no blocking or fusion.  It shares nothing with the CUDA path.

Discretisation (the paper drops the quadrature weights, Section "GW
approximation", text after Eq. 8; these are the readings used here):
  * orbitals are discretely orthonormal, sum_r phi_i(r) phi_j(r) = delta_ij;
  * the Coulomb operator on grid vectors is V = F^-1 diag(v_G / dV) F with
    v_G = 4 pi / |G|^2, v_0 = 0, dV = cell volume / N_r, G = 2 pi m / L;
  * everything is real (Gamma point, Eq. 8), so ^H becomes ^T;
  * on the imaginary frequency axis Omega(i w)^-1 = diag(D / (D^2 + w^2))
    with D_ij = e_i - e_j < 0 (Eq. Hedin_fourier with w -> i w, eta -> 0);
    w = 0 is the static case of Eq. matrices.
With these, chi0 = 2 M Omega^-1 M^T, eps = I - V chi0, W = eps^-1 V (Eq.
matrices) are plain matrices.

Functions and the passages they follow:
  coulomb_kernel / apply_coulomb ....... V by FFT (Eq. Hedin_fourier, V)
  coulomb_dense ........................ V as an explicit sum over G (tiny grids)
  pair_matrix .......................... M_(n; i,j) = psi_i(r_n) psi_j(r_n) (Eq. Omega text)
  omega_inverse ........................ Omega^-1 (Eq. Omega), imaginary axis
  chi0_dense / eps_dense / eps_inv_dense Eq. matrices
  eps_tilde_dense ...................... I + X, X = V^1/2 M (-2 Omega^-1) M^T V^1/2
                                         (supplementary error analysis)
  pair_space_eps_inv ................... eps^-1 = I + V M (Omega/2 - M^T V M)^-1 M^T
                                         (supplementary, SMW on the exact M)
  isdf_coefficients .................... C = M[mu, :] (Eq. MatrixExpressionISDF)
  isdf_fit ............................. least-squares P (Theta) with M ~ P C
  facesplit_gram ....................... M C^T via the Hadamard identity (Eq. Hadamard)
  polarizability ....................... B = C Omega^-1 C^T (Eq. COmegaCstar), explicit over pairs
  coulomb_in_basis ..................... G = Theta^T V Theta (Algorithm 3 step 2)
  capacitance .......................... K = (B^-1/2 - G)^-1 (Section "Cubic scaling
                                         algorithm"), in the B^-1-free form -D (I + G D)^-1
  apply_eps_inv ........................ eps^-1 X = X + V Theta K Theta^T X (Eq. epsilon_with_SMW)
  apply_eps_hat ........................ eps_hat X = X - 2 V Theta B Theta^T X (the ISDF eps)

Parity: every function here is pinned by tests/test_oracle_pins.py against
closed forms, brute force, identities or physical laws (see that file).
"""
from __future__ import annotations

import math
from typing import Optional, Sequence, Tuple

import numpy as np
import scipy.linalg

__all__ = [
    "grid_frequencies", "coulomb_kernel", "apply_coulomb", "coulomb_dense",
    "pair_matrix", "pair_energies", "omega_inverse", "chi0_dense", "eps_dense",
    "eps_inv_dense", "eps_tilde_dense", "screened_coulomb_dense", "pair_space_eps_inv",
    "isdf_coefficients", "isdf_fit", "facesplit_gram", "polarizability",
    "coulomb_in_basis", "capacitance", "capacitance_paper_form", "apply_eps_inv",
    "apply_eps_hat", "IsdfSmwResult", "isdf_smw_solve",
]


# --------------------------------------------------------------------------
# Coulomb operator on the periodic grid
# --------------------------------------------------------------------------

def grid_frequencies(n: Sequence[int], cell: Sequence[float]) -> np.ndarray:
    """|G|^2 on the full FFT grid, array shape (n3, n2, n1).

    G_k = 2 pi m_k / L_k with m_k the FFT integer frequencies.  The array
    axes follow a grid vector reshaped in C order from r = x + n1 (y + n2 z).
    """
    n1, n2, n3 = (int(v) for v in n)
    L1, L2, L3 = (float(v) for v in cell)
    g1 = 2.0 * np.pi * np.fft.fftfreq(n1, d=1.0 / n1) / L1
    g2 = 2.0 * np.pi * np.fft.fftfreq(n2, d=1.0 / n2) / L2
    g3 = 2.0 * np.pi * np.fft.fftfreq(n3, d=1.0 / n3) / L3
    return g3[:, None, None] ** 2 + g2[None, :, None] ** 2 + g1[None, None, :] ** 2


def coulomb_kernel(n: Sequence[int], cell: Sequence[float]) -> np.ndarray:
    """v_G / dV with v_G = 4 pi / |G|^2 and the G = 0 term set to zero."""
    n_r = int(np.prod(n))
    dv = float(np.prod(cell)) / n_r
    g2 = grid_frequencies(n, cell)
    v = np.zeros_like(g2)
    nz = g2 > 0
    v[nz] = 4.0 * np.pi / g2[nz]
    return v / dv


def apply_coulomb(x: np.ndarray, n: Sequence[int], cell: Sequence[float],
                  power: float = 1.0) -> np.ndarray:
    """V^power x for grid vectors x of shape (N_r,) or (N_r, k), via full FFTs."""
    n1, n2, n3 = (int(v) for v in n)
    vec = x.ndim == 1
    xs = x.reshape(-1, 1) if vec else x
    k = xs.shape[1]
    kern = coulomb_kernel(n, cell) ** power
    cube = np.asarray(xs.T, dtype=np.float64).reshape(k, n3, n2, n1)
    spec = np.fft.fftn(cube, axes=(1, 2, 3))
    out = np.fft.ifftn(spec * kern[None], axes=(1, 2, 3)).real
    out = out.reshape(k, -1).T
    return out[:, 0].copy() if vec else np.asfortranarray(out)


def coulomb_dense(n: Sequence[int], cell: Sequence[float]) -> np.ndarray:
    """V as an explicit N_r x N_r matrix, V[r, r'] = sum_G v_G cos(G.(r - r')) / (N_r dV).

    A direct double sum over grid points and G vectors; only for tiny grids.
    """
    n1, n2, n3 = (int(v) for v in n)
    L = [float(v) for v in cell]
    n_r = n1 * n2 * n3
    dv = float(np.prod(cell)) / n_r
    pos = np.array([(x * L[0] / n1, y * L[1] / n2, z * L[2] / n3)
                    for z in range(n3) for y in range(n2) for x in range(n1)])
    gs = []
    for m3 in np.fft.fftfreq(n3, d=1.0 / n3):
        for m2 in np.fft.fftfreq(n2, d=1.0 / n2):
            for m1 in np.fft.fftfreq(n1, d=1.0 / n1):
                if m1 == 0 and m2 == 0 and m3 == 0:
                    continue
                gs.append((2 * np.pi * m1 / L[0], 2 * np.pi * m2 / L[1], 2 * np.pi * m3 / L[2]))
    out = np.zeros((n_r, n_r))
    for g in gs:
        g = np.array(g)
        vg = 4.0 * np.pi / float(g @ g)
        phase = pos @ g
        out += vg * np.cos(phase[:, None] - phase[None, :])
    return out / (n_r * dv)


# --------------------------------------------------------------------------
# Pair functions, Omega and the dense operators (Eq. matrices)
# --------------------------------------------------------------------------

def pair_matrix(phi: np.ndarray, n_v: int) -> np.ndarray:
    """M_(n; i,j) = psi_i(r_n) psi_j(r_n), i occupied, j unoccupied; column i*N_c + j."""
    n_r = phi.shape[0]
    pv, pc = phi[:, :n_v], phi[:, n_v:]
    return (pv[:, :, None] * pc[:, None, :]).reshape(n_r, -1)


def pair_energies(energies: np.ndarray, n_v: int) -> np.ndarray:
    """Diagonal of Omega (Eq. Omega): e_i - e_j, ordered like the pair columns."""
    ev, ec = energies[:n_v], energies[n_v:]
    return (ev[:, None] - ec[None, :]).reshape(-1)


def omega_inverse(energies: np.ndarray, n_v: int, omega: float = 0.0) -> np.ndarray:
    """Diagonal of Omega(i w)^-1 = D / (D^2 + w^2), D = e_i - e_j (w = 0: 1 / D)."""
    d = pair_energies(energies, n_v)
    return d / (d * d + omega * omega)


def chi0_dense(phi, energies, n_v, omega=0.0, m=None):
    """chi0 = 2 M Omega^-1 M^T (Eq. matrices); M may be passed in (e.g. the ISDF M_hat)."""
    if m is None:
        m = pair_matrix(phi, n_v)
    return 2.0 * (m * omega_inverse(energies, n_v, omega)[None, :]) @ m.T


def eps_dense(phi, energies, n_v, n, cell, omega=0.0, m=None):
    """eps = I - V chi0 (Eq. matrices), dense N_r x N_r."""
    chi0 = chi0_dense(phi, energies, n_v, omega, m)
    return np.eye(chi0.shape[0]) - apply_coulomb(chi0, n, cell)


def eps_inv_dense(phi, energies, n_v, n, cell, omega=0.0, m=None):
    """eps^-1 by a dense LU solve (Algorithm 1 step 2)."""
    e = eps_dense(phi, energies, n_v, n, cell, omega, m)
    return np.linalg.solve(e, np.eye(e.shape[0]))


def eps_tilde_dense(phi, energies, n_v, n, cell, omega=0.0, m=None):
    """Symmetrised eps~ = I - V^1/2 chi0 V^1/2 = I + X (supplementary error
    analysis: X = V^1/2 M (-2 Omega^-1) M^T V^1/2 is positive semidefinite)."""
    chi0 = chi0_dense(phi, energies, n_v, omega, m)
    half = apply_coulomb(apply_coulomb(chi0, n, cell, 0.5).T, n, cell, 0.5).T
    return np.eye(chi0.shape[0]) - half


def screened_coulomb_dense(phi, energies, n_v, n, cell, omega=0.0, m=None):
    """W = eps^-1 V (Eq. matrices), dense."""
    einv = eps_inv_dense(phi, energies, n_v, n, cell, omega, m)
    return apply_coulomb(einv.T, n, cell).T   # eps^-1 V = (V eps^-T)^T, V symmetric


def pair_space_eps_inv(phi, energies, n_v, n, cell, omega=0.0):
    """eps^-1 = I + V M (Omega/2 - M^T V M)^-1 M^T (supplementary: SMW on the
    exact pair matrix), with Omega(i w) the inverse of `omega_inverse`."""
    m = pair_matrix(phi, n_v)
    vm = apply_coulomb(m, n, cell)
    om = 1.0 / omega_inverse(energies, n_v, omega)
    cap = np.diag(0.5 * om) - m.T @ vm
    return np.eye(m.shape[0]) + vm @ np.linalg.solve(cap, m.T)


# --------------------------------------------------------------------------
# ISDF (Eq. ISDF, Eq. MatrixExpressionISDF) and the SMW inverse
# --------------------------------------------------------------------------

def isdf_coefficients(phi: np.ndarray, n_v: int, mu_idx: np.ndarray) -> np.ndarray:
    """C_(mu; i,j) = psi_i(r_mu) psi_j(r_mu): the pair matrix at the points."""
    return pair_matrix(phi[np.asarray(mu_idx)], n_v)


def facesplit_gram(phi: np.ndarray, n_v: int, mu_idx: np.ndarray) -> np.ndarray:
    """M C^T = (Phi_v Phi_v,mu^T) .* (Phi_c Phi_c,mu^T), by the Hadamard identity
    (Eq. Hadamard with C = I): sum_ij psi_i(r) psi_j(r) psi_i(r_mu) psi_j(r_mu)
    factorises into a product of two sums."""
    pm = phi[np.asarray(mu_idx)]
    return (phi[:, :n_v] @ pm[:, :n_v].T) * (phi[:, n_v:] @ pm[:, n_v:].T)


def isdf_fit(phi: np.ndarray, n_v: int, mu_idx: np.ndarray, rcond: float = 1e-13,
             explicit: Optional[bool] = None) -> Tuple[np.ndarray, int]:
    """Least-squares auxiliary functions Theta (the paper's P) with M ~ Theta C.

    The paper states M = P C (Eq. MatrixExpressionISDF) without the fitting
    rule; the reading here is least squares, Theta = M C^+ (minimum-norm
    solution when C is rank deficient), with C^+ from an SVD that discards
    singular values below rcond * sigma_max.  For small systems M C^+ is
    formed from the explicit M; otherwise M C^T (C C^T)^+ with M C^T from the
    Hadamard identity and (C C^T)^+ from a symmetric eigendecomposition with
    the same cut (eigenvalues below rcond^2 * lambda_max).
    Returns (Theta, numerical rank of C).
    """
    mu_idx = np.asarray(mu_idx)
    n_r = phi.shape[0]
    n_pairs = n_v * (phi.shape[1] - n_v)
    if explicit is None:
        explicit = n_r * n_pairs <= 4e7
    c = isdf_coefficients(phi, n_v, mu_idx)
    if explicit:
        u, s, vt = np.linalg.svd(c, full_matrices=False)
        keep = s > rcond * s[0]
        cplus = (vt[keep].T / s[keep]) @ u[:, keep].T
        return pair_matrix(phi, n_v) @ cplus, int(keep.sum())
    z = facesplit_gram(phi, n_v, mu_idx)
    w, q = np.linalg.eigh(c @ c.T)
    keep = w > (rcond ** 2) * w[-1]
    pinv = (q[:, keep] / w[keep]) @ q[:, keep].T
    return z @ pinv, int(keep.sum())


def polarizability(phi_mu: np.ndarray, energies: np.ndarray, n_v: int,
                   omega: float = 0.0) -> np.ndarray:
    """B = C Omega^-1 C^T (Eq. COmegaCstar), summed explicitly over all pairs."""
    c = pair_matrix(phi_mu, n_v)
    return (c * omega_inverse(energies, n_v, omega)[None, :]) @ c.T


def coulomb_in_basis(theta: np.ndarray, n, cell) -> np.ndarray:
    """G = Theta^T V Theta (Algorithm 3 step 2, P_vc^H V P_vc)."""
    return theta.T @ apply_coulomb(theta, n, cell)


def capacitance(g: np.ndarray, b: np.ndarray) -> np.ndarray:
    """K = (B^-1 / 2 - G)^-1 written without B^-1.

    With D = -2 B (positive semidefinite because Omega < 0):
    B^-1/2 - G = -(D^-1 + G), so K = -(D^-1 + G)^-1 = -D (I + G D)^-1.
    The last form exists whenever I + G D is invertible, which holds for
    positive semidefinite G and D, so it also covers a singular B (more
    points than independent pairs).  Solved by LU.
    """
    d = -2.0 * b
    n = g.shape[0]
    # K = -D (I + G D)^-1  <=>  K^T = -(I + D G)^-1 D ; K is symmetric
    kt = -np.linalg.solve(np.eye(n) + d @ g, d)
    return kt.T


def capacitance_paper_form(g: np.ndarray, b: np.ndarray) -> np.ndarray:
    """K = (B^-1 / 2 - G)^-1 literally (Section "Cubic scaling algorithm");
    needs an invertible B."""
    return np.linalg.inv(0.5 * np.linalg.inv(b) - g)


def apply_eps_inv(theta, k, x, n, cell):
    """eps^-1 X = X + V Theta K Theta^T X (Eq. epsilon_with_SMW with K)."""
    return x + apply_coulomb(theta @ (k @ (theta.T @ x)), n, cell)


def apply_eps_hat(theta, b, x, n, cell):
    """eps_hat X = X - 2 V Theta B Theta^T X: the dielectric matrix built from
    the ISDF pair matrix M_hat = Theta C (first display of the SMW section)."""
    return x - 2.0 * apply_coulomb(theta @ (b @ (theta.T @ x)), n, cell)


class IsdfSmwResult:
    """Everything one ISDF-SMW solve produces (oracle side)."""

    def __init__(self, theta, rank, b, g, k, y):
        self.theta, self.rank, self.b, self.g, self.k, self.y = theta, rank, b, g, k, y


def isdf_smw_solve(phi, energies, n_v, mu_idx, n, cell, x, omega=0.0,
                   rcond=1e-13) -> IsdfSmwResult:
    """One full solve: fit, B, G, K and Y = eps_hat^-1 X (Algorithm 3 steps 1-3
    with the direct sum for B, then Eq. epsilon_with_SMW applied to X)."""
    theta, rank = isdf_fit(phi, n_v, mu_idx, rcond=rcond)
    b = polarizability(phi[np.asarray(mu_idx)], energies, n_v, omega)
    g = coulomb_in_basis(theta, n, cell)
    k = capacitance(g, b)
    y = apply_eps_inv(theta, k, x, n, cell)
    return IsdfSmwResult(theta, rank, b, g, k, y)
