"""Seeded synthetic Gamma-point systems for the ISDF-SMW dielectric inverse.

This module only *makes inputs*: orbitals on a periodic real-space grid,
orbital energies, interpolation-point indices, imaginary frequencies and
probe blocks.  It holds none of the method's arithmetic (no pair matrix, no
polarizability, no Coulomb operator, no fit, no inverse), so both the FP64
oracle and the CUDA path can be fed from it without sharing any step of the
computation.

The paper's test systems (KSSOLV ground states of Si_8..Si_64, (SrTiO3)_8 and
C60, Table S1) are not available, so these systems stand in for them with the
structure the paper describes: real orbitals at the Gamma point (Eq. 8), a
gapped spectrum with the lowest N_v states occupied, band-limited orbitals on
a uniform grid with N_r / N_e in the 100..1000 range (abstract), and
N_mu = k_mu * sqrt(N_v N_c) interpolation points with k_mu of order ten
(Section "Interpolative separable density fitting").

Conventions (readings of points the paper leaves open):
  * cubic cell, grid spacing h = 0.5 Bohr, so L = n h and dV = h^3;
  * orbitals are discretely orthonormal: sum_r phi_i(r) phi_j(r) = delta_ij;
  * Phi is stored column-major N_r x N_e (grid index fastest), the grid index
    of point (x, y, z) being r = x + n1 * (y + n2 * z);
  * energies in Hartree (1 Ha = 27.211386245988 eV), ascending, the first
    N_v occupied;
  * interpolation points by QR with column pivoting (QRCP) on the pair
    functions, or on a Gaussian face-split sketch of them when the number of
    pairs exceeds the sketch width.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

HARTREE_EV = 27.211386245988
GRID_SPACING_BOHR = 0.5

# Seeds: orbitals 1000 + c, energies 2000 + c (c = index of the named
# workload), probes 7, sketch 11, projector 13.
SEED_PROBE = 7
SEED_SKETCH = 11
SEED_PROJECTOR = 13


@dataclasses.dataclass
class System:
    """One synthetic Gamma-point system (all arrays float64 / int64, host)."""

    n: Tuple[int, int, int]          # grid points per axis (n1, n2, n3)
    cell: Tuple[float, float, float]  # cell lengths in Bohr
    n_v: int
    n_c: int
    phi: np.ndarray                   # (N_r, N_v + N_c), Fortran order
    energies: np.ndarray              # (N_v + N_c,), Hartree, ascending
    mu_idx: np.ndarray                # (N_mu,), int64 grid indices
    name: str = ""

    @property
    def n_r(self) -> int:
        return int(np.prod(self.n))

    @property
    def n_e(self) -> int:
        return self.n_v + self.n_c

    @property
    def n_mu(self) -> int:
        return int(self.mu_idx.shape[0])

    @property
    def dv(self) -> float:
        return float(np.prod(self.cell)) / self.n_r


def real_plane_wave_modes(n: Sequence[int], count: int) -> List[Tuple[int, int, int, int]]:
    """The `count` lowest real plane waves on an n1 x n2 x n3 grid.

    Returns (m1, m2, m3, kind) with kind 0 = constant, 1 = cos, 2 = sin.  The
    modes are sorted by |G|^2 (G_i = 2 pi m_i / L_i with L_i = n_i h), ties
    broken lexicographically on (m1, m2, m3) and cos before sin.  Only m in
    the half space "first non-zero component positive" is used (cos and sin
    of -m repeat those of m), and |m_i| < n_i / 2 so that no mode sits on a
    Nyquist plane; these functions are then exactly orthogonal on the grid.
    """
    n = tuple(int(v) for v in n)
    lens = np.array([v * GRID_SPACING_BOHR for v in n])
    lim = [(v - 1) // 2 for v in n]
    m1, m2, m3 = np.meshgrid(*[np.arange(-l, l + 1) for l in lim], indexing="ij")
    m = np.stack([m1.ravel(), m2.ravel(), m3.ravel()], axis=1)
    first = np.where(m[:, 0] != 0, m[:, 0], np.where(m[:, 1] != 0, m[:, 1], m[:, 2]))
    m = m[first >= 0]
    g2 = (((2.0 * np.pi * m) / lens) ** 2).sum(axis=1)
    order = np.lexsort((m[:, 2], m[:, 1], m[:, 0], np.round(g2, 12)))
    modes: List[Tuple[int, int, int, int]] = []
    for k in order:
        a, b, c = (int(v) for v in m[k])
        if a == 0 and b == 0 and c == 0:
            modes.append((0, 0, 0, 0))
        else:
            modes.append((a, b, c, 1))
            modes.append((a, b, c, 2))
        if len(modes) >= count:
            return modes[:count]
    raise ValueError(f"grid {n} holds only {len(modes)} real plane waves, need {count}")


def plane_wave_matrix(n: Sequence[int], modes) -> np.ndarray:
    """Orthonormal real plane waves sampled on the grid, (N_r, len(modes))."""
    n1, n2, n3 = (int(v) for v in n)
    n_r = n1 * n2 * n3
    z, y, x = np.meshgrid(np.arange(n3), np.arange(n2), np.arange(n1), indexing="ij")
    x = x.reshape(-1).astype(np.float64)
    y = y.reshape(-1).astype(np.float64)
    z = z.reshape(-1).astype(np.float64)
    out = np.empty((n_r, len(modes)), dtype=np.float64, order="F")
    for k, (m1, m2, m3, kind) in enumerate(modes):
        if kind == 0:
            out[:, k] = 1.0 / math.sqrt(n_r)
            continue
        arg = 2.0 * math.pi * (m1 * x / n1 + m2 * y / n2 + m3 * z / n3)
        f = np.cos(arg) if kind == 1 else np.sin(arg)
        out[:, k] = math.sqrt(2.0 / n_r) * f
    return out


def lowdin(a: np.ndarray) -> np.ndarray:
    """A (A^T A)^{-1/2}: the orthonormal matrix closest to A."""
    w, u = np.linalg.eigh(a.T @ a)
    return a @ ((u / np.sqrt(w)) @ u.T)


def make_orbitals(n: Sequence[int], n_e: int, seed: int, n_pw: Optional[int] = None) -> np.ndarray:
    """Seeded, Lowdin-orthonormalised random combinations of the lowest
    max(200, 2 N_e) real plane waves (band-limited real Gamma-point orbitals)."""
    if n_pw is None:
        n_pw = max(200, 2 * n_e)
    modes = real_plane_wave_modes(n, n_pw)
    basis = plane_wave_matrix(n, modes)
    rng = np.random.Generator(np.random.PCG64(seed))
    coef = rng.standard_normal((n_pw, n_e))
    coef = lowdin(coef)   # basis is orthonormal, so basis @ coef is too
    return np.asfortranarray(basis @ coef)


def make_energies(n_v: int, n_c: int, seed: int,
                  occ_ev=(-10.0, -2.0), unocc_ev=(0.0, 20.0)) -> np.ndarray:
    """Occupied uniform in [-10,-2] eV, unoccupied uniform in [0,20] eV,
    each set sorted ascending, returned in Hartree."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ev = np.sort(rng.uniform(occ_ev[0], occ_ev[1], n_v))
    ec = np.sort(rng.uniform(unocc_ev[0], unocc_ev[1], n_c))
    return np.concatenate([ev, ec]) / HARTREE_EV


def qrcp_points(phi: np.ndarray, n_v: int, n_mu: int, sketch_extra: int = 64,
                seed: int = SEED_SKETCH) -> np.ndarray:
    """Interpolation points by QR with column pivoting.

    The columns pivoted are grid points of the (pairs x N_r) matrix whose rows
    are the pair functions, or of a Gaussian sketch of it with
    p = N_mu + sketch_extra rows, (Phi_v R_v) .* (Phi_c R_c), when the number
    of pairs exceeds p.  The first N_mu pivots are returned in pivot order.
    """
    import scipy.linalg

    n_r, n_e = phi.shape
    n_c = n_e - n_v
    p = n_mu + sketch_extra
    pv, pc = phi[:, :n_v], phi[:, n_v:]
    if n_v * n_c <= p:
        rows = (pv[:, :, None] * pc[:, None, :]).reshape(n_r, n_v * n_c)
    else:
        rng = np.random.Generator(np.random.PCG64(seed))
        rv = rng.standard_normal((n_v, p))
        rc = rng.standard_normal((n_c, p))
        rows = (pv @ rv) * (pc @ rc)
    _, piv = scipy.linalg.qr(np.ascontiguousarray(rows.T), mode="r", pivoting=True)
    if piv.shape[0] < n_mu:
        raise ValueError("fewer grid points than requested interpolation points")
    return np.asarray(piv[:n_mu], dtype=np.int64)


def make_system(n, n_v: int, n_c: int, n_mu: int, seed_index: int, name: str = "",
                n_pw: Optional[int] = None) -> System:
    """A full synthetic system with orbitals seed 1000 + c and energies seed
    2000 + c, c = seed_index."""
    if isinstance(n, int):
        n = (n, n, n)
    n = tuple(int(v) for v in n)
    phi = make_orbitals(n, n_v + n_c, 1000 + seed_index, n_pw=n_pw)
    energies = make_energies(n_v, n_c, 2000 + seed_index)
    mu = qrcp_points(phi, n_v, n_mu)
    cell = tuple(v * GRID_SPACING_BOHR for v in n)
    return System(n=n, cell=cell, n_v=n_v, n_c=n_c, phi=phi, energies=energies,
                  mu_idx=mu, name=name)


def probe_block(n_r: int, n_rhs: int = 16, seed: int = SEED_PROBE) -> np.ndarray:
    """Seeded N(0,1) probe block X (N_r x n_rhs, Fortran order)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.asfortranarray(rng.standard_normal((n_r, n_rhs)))


def gauss_legendre_frequencies(count: int = 32, omega0: float = 1.0) -> Tuple[np.ndarray, np.ndarray]:
    """Imaginary frequencies on [0, inf): Gauss-Legendre nodes x_k on (-1, 1)
    mapped by omega = omega0 (1 + x) / (1 - x); returns (omega, weights), the
    weights including the Jacobian 2 omega0 / (1 - x)^2."""
    x, w = np.polynomial.legendre.leggauss(count)
    om = omega0 * (1.0 + x) / (1.0 - x)
    return om, w * 2.0 * omega0 / (1.0 - x) ** 2


# Named workloads: grid n, N_v, N_c, N_mu.
WORKLOADS = {
    "isdf16": dict(n=16, n_v=4, n_c=28, n_mu=128, seed_index=0),
    "isdf48": dict(n=48, n_v=64, n_c=448, n_mu=1536, seed_index=1),
    "isdf72": dict(n=72, n_v=256, n_c=1792, n_mu=6144, seed_index=2, points="candidates"),
}

# Batched full-frequency set: 16 systems (grid n, N_v), N_c = 7 N_v,
# N_mu = 6 N_e with N_e = 2 N_v.
BATCH_SYSTEMS = [(24, 8), (27, 18), (30, 28), (32, 38), (32, 49), (36, 59), (40, 69), (40, 79),
                 (45, 89), (45, 99), (48, 109), (50, 119), (54, 130), (54, 140), (60, 150), (60, 160)]


def random_points(n_r: int, n_mu: int, seed: int) -> np.ndarray:
    """n_mu distinct grid points drawn uniformly (seeded)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.asarray(rng.choice(n_r, size=n_mu, replace=False), dtype=np.int64)


def qrcp_points_on_candidates(phi: np.ndarray, n_v: int, n_mu: int, cand_seed: int, factor: int = 2,
                              sketch_extra: int = 64, seed: int = SEED_SKETCH) -> np.ndarray:
    """QRCP points for systems too large for QRCP over the whole grid.

    The grid points eligible as pivots are first cut to a seeded uniform
    candidate set of factor * N_mu points (seed cand_seed); the columns
    pivoted are those candidates in the Gaussian face-split sketch
    (Phi_v R_v) .* (Phi_c R_c) with p = N_mu + sketch_extra rows (seed
    `seed`), as in qrcp_points.  This costs O(p^2 factor N_mu) instead of
    O(p^2 N_r): half a minute for the 72^3 workload (N_mu = 6144) instead of
    hours, and keeps C C^T as well conditioned as QRCP over the whole grid
    does (cond(C C^T) = 9.4 there, against 531 for uniformly random points).
    Returns the first N_mu pivots in pivot order."""
    import scipy.linalg

    n_r, n_e = phi.shape
    m = min(n_r, factor * n_mu)
    crng = np.random.Generator(np.random.PCG64(cand_seed))
    cand = np.sort(crng.choice(n_r, size=m, replace=False))
    p = n_mu + sketch_extra
    rng = np.random.Generator(np.random.PCG64(seed))
    rv = rng.standard_normal((n_v, p))
    rc = rng.standard_normal((n_e - n_v, p))
    rows = (phi[cand, :n_v] @ rv) * (phi[cand, n_v:] @ rc)
    _, piv = scipy.linalg.qr(np.ascontiguousarray(rows.T), mode="r", pivoting=True)
    if piv.shape[0] < n_mu:
        raise ValueError("fewer candidate points than requested interpolation points")
    return np.asarray(cand[piv[:n_mu]], dtype=np.int64)


def batch_system(i: int) -> System:
    """System i of the batched full-frequency set (seed index c = 100 + i):
    orbitals seed 1000 + c, energies 2000 + c, and N_mu points by QRCP of the
    sketch over 2 N_mu seeded candidate points (seed 3000 + c; QRCP over the
    whole grid would take minutes of host time for the largest systems)."""
    n, n_v = BATCH_SYSTEMS[i]
    c = 100 + i
    nn = (n, n, n)
    n_c = 7 * n_v
    phi = make_orbitals(nn, n_v + n_c, 1000 + c)
    energies = make_energies(n_v, n_c, 2000 + c)
    mu = qrcp_points_on_candidates(phi, n_v, 12 * n_v, 3000 + c)
    cell = tuple(v * GRID_SPACING_BOHR for v in nn)
    return System(n=nn, cell=cell, n_v=n_v, n_c=n_c, phi=phi, energies=energies, mu_idx=mu, name=f"batch{i}")


def workload(name: str) -> System:
    """A named workload; points by QRCP, or (isdf72, whose QRCP over the
    whole grid would take hours of host time) by QRCP over 2 N_mu seeded
    candidate points, seed 3000 + c."""
    cfg = WORKLOADS[name]
    if cfg.get("points") != "candidates":
        return make_system(cfg["n"], cfg["n_v"], cfg["n_c"], cfg["n_mu"], cfg["seed_index"], name=name)
    c = cfg["seed_index"]
    nn = (cfg["n"],) * 3
    phi = make_orbitals(nn, cfg["n_v"] + cfg["n_c"], 1000 + c)
    energies = make_energies(cfg["n_v"], cfg["n_c"], 2000 + c)
    mu = qrcp_points_on_candidates(phi, cfg["n_v"], cfg["n_mu"], 3000 + c)
    cell = tuple(v * GRID_SPACING_BOHR for v in nn)
    return System(n=nn, cell=cell, n_v=cfg["n_v"], n_c=cfg["n_c"], phi=phi, energies=energies, mu_idx=mu, name=name)
