"""Plain FP64 oracle of the contour-integral polarizability (Algorithm 2 and
the supplementary derivation "Detailed derivation process of Algorithm 2").
TEST INFRASTRUCTURE: only the tests, the smoke check and the benchmark's CPU
legs import it.

The sum over pairs of Eq. COmegaCstar is replaced by a contour integral: for
a closed contour I that encloses every unoccupied energy and no occupied one,
    1 / (e_v - e_c) = -(1 / 2 pi i) oint_I d lambda / ((lambda - e_v)(lambda - e_c)),
so that
    B = C Omega^-1 C^T = -(1 / 2 pi i) oint_I J(lambda) d lambda,
    J(lambda) = (Psi_v diag(1/(lambda - e_v)) Psi_v^T) .* (Psi_c diag(1/(lambda - e_c)) Psi_c^T),
with Psi_v, Psi_c the orbitals at the interpolation points.  Everything is
real (Gamma point), so J(conj lambda) = conj J(lambda), and with I symmetric
about the real axis the closed integral is 2 i Im of the integral over the
upper half I+ traversed counterclockwise (right to left).  The segment below
maps onto I+ left to right (t = -K + i K'/2 lands between e_N and the gap,
t = K + i K'/2 beyond the top of the unoccupied band), which is the
clockwise sense, hence B = +(1/pi) Im int_{I+, left to right} J(z) dz
(reading of the garbled formula of Algorithm 2 step 3: the imaginary part is
taken of J(z(t)) z'(t), the whole integrand).

The contour is the image of the segment t in [-K + i K'/2, K + i K'/2]
under the conformal map of Algorithm 2,
    z(t) = e_N + sqrt(q Q) (k^-1 + sn(t, k)) / (k^-1 - sn(t, k)),
    k = (sqrt(Q/q) - 1) / (sqrt(Q/q) + 1),
q = e_{N_v+1} - e_{N_v} (the gap), Q = e_{N_v+N_c} - e_{N_v}, e_N = e_{N_v};
K = K(k), K' = K(sqrt(1 - k^2)) are complete elliptic integrals of the first
kind (reading of the garbled R and L of Algorithm 2: R = K, L = K'/2).  The
map sends C \\ ((-inf, e_N] U [e_N + q, e_N + Q]) to a rectangle, so the
midpoint rule in t converges geometrically; the paper quotes the bound
O(exp(-pi^2 N / (2 log(Q/q) + 6))) (Eq. rel_err_Cauchy).

Jacobi elliptic functions: real argument by the arithmetic-geometric mean
(descending Landen) recursion, complex argument by the addition formulas
for sn, cn, dn of u + i v with the complementary modulus.
"""
from __future__ import annotations

import math
from typing import Tuple

import numpy as np

from .isdf_oracle import pair_matrix

__all__ = ["ellipk", "jacobi_real", "jacobi_complex", "contour_nodes", "contour_error_bound",
           "polarizability_contour", "polarizability_direct"]


def ellipk(k: float) -> float:
    """K(k) = int_0^{pi/2} (1 - k^2 sin^2)^-1/2 = pi / (2 AGM(1, sqrt(1 - k^2)))."""
    a, b = 1.0, math.sqrt(1.0 - k * k)
    for _ in range(60):
        if abs(a - b) <= 1e-16 * a:
            break
        a, b = 0.5 * (a + b), math.sqrt(a * b)
    return math.pi / (a + b)


def jacobi_real(u: float, k: float) -> Tuple[float, float, float]:
    """sn, cn, dn of a real argument u, modulus 0 <= k < 1, by the descending
    Landen (AGM) recursion: a_0 = 1, b_0 = sqrt(1 - k^2), c_0 = k; then
    phi_N = 2^N a_N u and phi_{n-1} = (phi_n + asin(c_n sin(phi_n) / a_n)) / 2."""
    a = [1.0]
    c = [k]
    b = math.sqrt(1.0 - k * k)
    while abs(c[-1]) > 1e-17 and len(a) < 40:
        an = 0.5 * (a[-1] + b)
        cn_ = 0.5 * (a[-1] - b)
        b = math.sqrt(a[-1] * b)
        a.append(an)
        c.append(cn_)
    n = len(a) - 1
    phi = (2.0 ** n) * a[n] * u
    phis = [phi]
    for i in range(n, 0, -1):
        phi = 0.5 * (phi + math.asin(c[i] * math.sin(phi) / a[i]))
        phis.append(phi)
    phi0 = phis[-1]
    sn = math.sin(phi0)
    cn = math.cos(phi0)
    dn = cn / math.cos(phis[-2] - phi0) if n > 0 else 1.0
    return sn, cn, dn


def jacobi_complex(u: float, v: float, k: float) -> Tuple[complex, complex, complex]:
    """sn, cn, dn of u + i v (modulus k) from the real-argument functions of
    u (modulus k) and of v (complementary modulus k')."""
    kp = math.sqrt(1.0 - k * k)
    s, c, d = jacobi_real(u, k)
    s1, c1, d1 = jacobi_real(v, kp)
    den = c1 * c1 + k * k * s * s * s1 * s1
    sn = complex(s * d1, c * d * s1 * c1) / den
    cn = complex(c * c1, -s * d * s1 * d1) / den
    dn = complex(d * c1 * d1, -k * k * s * c * s1) / den
    return sn, cn, dn


def contour_nodes(energies: np.ndarray, n_v: int, n_nodes: int) -> Tuple[np.ndarray, np.ndarray]:
    """Midpoint nodes z_j on the upper half contour and the weights h z'(t_j)
    (h = 2K / n_nodes), so that int_{I+} f(z) dz ~ sum_j f(z_j) w_j."""
    e = np.asarray(energies, dtype=np.float64)
    e_n = float(np.max(e[:n_v]))
    q = float(np.min(e[n_v:])) - e_n
    big_q = float(np.max(e[n_v:])) - e_n
    if not q > 0.0:
        raise ValueError("no gap between occupied and unoccupied energies")
    ratio = math.sqrt(big_q / q)
    k = (ratio - 1.0) / (ratio + 1.0)
    kk = ellipk(k)
    kkp = ellipk(math.sqrt(1.0 - k * k))
    scale = math.sqrt(q * big_q)
    h = 2.0 * kk / n_nodes
    z = np.empty(n_nodes, dtype=np.complex128)
    w = np.empty(n_nodes, dtype=np.complex128)
    for j in range(n_nodes):
        u = -kk + (j + 0.5) * h
        sn, cn, dn = jacobi_complex(u, 0.5 * kkp, k)
        z[j] = e_n + scale * (1.0 / k + sn) / (1.0 / k - sn)
        w[j] = h * scale * (2.0 / k) * cn * dn / (1.0 / k - sn) ** 2
    return z, w


def contour_error_bound(energies: np.ndarray, n_v: int, n_nodes: int) -> float:
    """exp(-pi^2 N / (2 log(Q/q) + 6)) of Eq. rel_err_Cauchy (without its constant)."""
    e = np.asarray(energies, dtype=np.float64)
    e_n = float(np.max(e[:n_v]))
    q = float(np.min(e[n_v:])) - e_n
    big_q = float(np.max(e[n_v:])) - e_n
    return math.exp(-math.pi ** 2 * n_nodes / (2.0 * math.log(big_q / q) + 6.0))


def polarizability_contour(phi_mu: np.ndarray, energies: np.ndarray, n_v: int, n_nodes: int) -> np.ndarray:
    """B = C Omega^-1 C^T (static) by the contour integral of Algorithm 2:
    B = (1/pi) Im sum_j J(z_j) w_j (nodes left to right on I+), each J(z_j)
    the Hadamard product of the occupied and unoccupied resolvent Grams at
    the points."""
    pv = phi_mu[:, :n_v]
    pc = phi_mu[:, n_v:]
    ev = np.asarray(energies[:n_v], dtype=np.float64)
    ec = np.asarray(energies[n_v:], dtype=np.float64)
    z, w = contour_nodes(energies, n_v, n_nodes)
    acc = np.zeros((phi_mu.shape[0], phi_mu.shape[0]), dtype=np.complex128)
    for zj, wj in zip(z, w):
        av = (pv * (1.0 / (zj - ev))[None, :]) @ pv.T
        ac = (pc * (1.0 / (zj - ec))[None, :]) @ pc.T
        acc += (av * ac) * wj
    return acc.imag / math.pi


def polarizability_direct(phi_mu: np.ndarray, energies: np.ndarray, n_v: int) -> np.ndarray:
    """The direct pair sum of Eq. COmegaCstar (static), for comparison."""
    c = pair_matrix(phi_mu, n_v)
    e = np.asarray(energies, dtype=np.float64)
    d = (e[:n_v, None] - e[None, n_v:]).reshape(-1)
    return (c / d[None, :]) @ c.T
