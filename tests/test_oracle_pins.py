"""Pins for the FP64 oracle: each check ties it to something other than itself
(brute force, closed forms, physical laws, identities, invariants), chosen so
that a dropped term, a wrong sign or factor, a transposed operand or a wrong
index fails at least one of them.  CPU only."""
import math

import numpy as np
import pytest
from scipy.special import erf

import oracle as O
import synth
from helpers import rel_fro, small_system


# ---------------------------------------------------------------- Coulomb V

def test_coulomb_fft_equals_explicit_double_sum():
    """V by FFT equals the explicit sum over G on a tiny non-cubic grid
    (odd and even axes): catches a transposed axis or reshape order."""
    n, cell = (4, 5, 3), (2.0, 3.0, 1.7)
    vd = O.coulomb_dense(n, cell)
    x = np.random.default_rng(1).standard_normal((vd.shape[0], 3))
    assert rel_fro(O.apply_coulomb(x, n, cell), vd @ x) < 1e-12
    assert np.allclose(vd, vd.T, atol=1e-12 * np.abs(vd).max())


def test_coulomb_gauss_law_potential_of_gaussian_charge():
    """Physical pin (Poisson / Gauss's law): the periodic potential of a unit
    Gaussian charge with neutralising background is, near the charge,
    erf(d / (sqrt(2) s)) / d + (2 pi / (3 Omega_cell)) d^2 + const + O(d^4 / L^5)
    in a cubic cell.  Pins v_G = 4 pi / |G|^2, G = 2 pi m / L and the 1/dV."""
    n = 32
    h = synth.GRID_SPACING_BOHR
    cell = (n * h,) * 3
    s = 1.0
    c = n // 2
    idx = np.arange(n)
    dx = (idx - c) * h
    X, Y, Z = np.meshgrid(dx, dx, dx, indexing="ij")           # axes (x, y, z)
    d2 = X ** 2 + Y ** 2 + Z ** 2
    rho = (2 * np.pi * s * s) ** -1.5 * np.exp(-d2 / (2 * s * s))
    # grid vector with r = x + n (y + n z): C-order array indexed [z, y, x]
    rho_vec = np.transpose(rho, (2, 1, 0)).reshape(-1)
    dv = h ** 3
    assert abs(rho_vec.sum() * dv - 1.0) < 1e-9
    pot = dv * O.apply_coulomb(rho_vec, (n, n, n), cell)        # potential, Hartree / e
    pot = pot.reshape(n, n, n).transpose(2, 1, 0)               # back to [x, y, z]
    omega_cell = cell[0] ** 3
    p0 = pot[c, c, c]
    iso0 = math.sqrt(2.0 / math.pi) / s
    for (i, j, k) in [(c + 2, c, c), (c, c + 3, c + 1), (c + 4, c + 2, c + 2), (c - 5, c + 1, c), (c + 3, c - 3, c + 3)]:
        d = math.sqrt(float(d2[i, j, k]))
        want = (erf(d / (math.sqrt(2) * s)) / d - iso0) + 2 * math.pi / (3 * omega_cell) * d * d
        got = pot[i, j, k] - p0
        assert abs(got - want) < 2e-3 * abs(want), (d, got, want)


def test_coulomb_plane_wave_eigenvalue_non_cubic():
    """cos(G.r) is an eigenvector of V with eigenvalue 4 pi / (|G|^2 dV), on a
    non-cubic cell so that mixing up axes changes the answer."""
    n, cell = (6, 5, 8), (3.0, 2.5, 4.4)
    z, y, x = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    m = (1, 2, 3)
    f = np.cos(2 * np.pi * (m[0] * x / n[0] + m[1] * y / n[1] + m[2] * z / n[2])).reshape(-1)
    g2 = sum((2 * np.pi * mi / Li) ** 2 for mi, Li in zip(m, cell))
    dv = np.prod(cell) / np.prod(n)
    lam = 4 * np.pi / g2 / dv
    assert rel_fro(O.apply_coulomb(f, n, cell), lam * f) < 1e-12
    # the constant vector is annihilated (G = 0 dropped)
    assert np.abs(O.apply_coulomb(np.ones(np.prod(n)), n, cell)).max() < 1e-10


def test_coulomb_square_root():
    n, cell = (6, 6, 6), (3.0, 3.0, 3.0)
    x = np.random.default_rng(2).standard_normal((216, 2))
    vv = O.apply_coulomb(O.apply_coulomb(x, n, cell, 0.5), n, cell, 0.5)
    assert rel_fro(vv, O.apply_coulomb(x, n, cell)) < 1e-12


# ---------------------------------------------------------- chi0 and Omega

def test_chi0_matches_brute_force_pair_sum():
    """chi0 = 2 M Omega^-1 M^T against a literal loop over r, r', i, j of the
    static two-term sum (Eq. Hedin_G0W0, first line)."""
    s = small_system(4, 2, 3, n_mu=8, n_pw=12)
    phi, e, nv = s.phi, s.energies, s.n_v
    n_r = phi.shape[0]
    ref = np.zeros((n_r, n_r))
    for r in range(n_r):
        for rp in range(n_r):
            acc = 0.0
            for i in range(nv):
                for j in range(nv, phi.shape[1]):
                    acc += phi[r, i] * phi[rp, i] * phi[rp, j] * phi[r, j] / (e[i] - e[j])
            ref[r, rp] = 2.0 * acc
    assert rel_fro(O.chi0_dense(phi, e, nv), ref) < 1e-13
    # and the pair ordering of M: column i*N_c + j
    m = O.pair_matrix(phi, nv)
    assert np.allclose(m[:, 1 * 3 + 2], phi[:, 1] * phi[:, nv + 2])


def test_imaginary_axis_continuation():
    """Omega(i w)^-1 against the two-term Hedin sum evaluated at complex
    frequency i w with a tiny eta: 1/(iw + D + i eta) - 1/(iw - D - i eta)
    = 2 Omega(iw)^-1 (the factor 2 goes to chi0 = 2 M Omega^-1 M^T)."""
    e = synth.make_energies(3, 4, 5)
    d = O.pair_energies(e, 3)
    for w in [0.0, 0.05, 0.7, 13.0]:
        eta = 1e-12
        two_term = 1.0 / (1j * w + d + 1j * eta) - 1.0 / (1j * w - d - 1j * eta)
        assert np.allclose(two_term.imag, 0.0, atol=1e-9)
        assert np.allclose(two_term.real, 2.0 * O.omega_inverse(e, 3, w), rtol=1e-9)
    assert np.all(d < 0)


# ----------------------------------------------------- dense and SMW inverse

def test_sherman_morrison_one_pair_closed_form():
    """N_v = N_c = 1: chi0 = (2/D) m m^T and eps^-1 = I + 2 (V m) m^T / (D - 2 m^T V m)."""
    s = small_system(5, 1, 1, n_mu=1, n_pw=6)
    m = s.phi[:, 0] * s.phi[:, 1]
    d = s.energies[0] - s.energies[1]
    vm = O.apply_coulomb(m, s.n, s.cell)
    closed = np.eye(m.size) + 2.0 * np.outer(vm, m) / (d - 2.0 * m @ vm)
    assert rel_fro(O.eps_inv_dense(s.phi, s.energies, 1, s.n, s.cell), closed) < 1e-12
    assert rel_fro(O.pair_space_eps_inv(s.phi, s.energies, 1, s.n, s.cell), closed) < 1e-12


def test_plane_wave_pair_dielectric_eigenvalue():
    """phi_v = 1/sqrt(N_r), phi_c = sqrt(2/N_r) cos(G.r): the pair m is an
    eigenvector of eps with eigenvalue 1 + 2 v_G / (Omega_cell |D|), so
    eps^-1 m = m / lambda."""
    n = (8, 8, 8)
    cell = tuple(v * 0.5 for v in n)
    n_r = 512
    z, y, x = np.meshgrid(np.arange(8), np.arange(8), np.arange(8), indexing="ij")
    phi = np.empty((n_r, 2))
    phi[:, 0] = 1 / math.sqrt(n_r)
    phi[:, 1] = math.sqrt(2 / n_r) * np.cos(2 * np.pi * (2 * x + 1 * z) / 8).reshape(-1)
    e = np.array([-0.3, 0.2])
    m = phi[:, 0] * phi[:, 1]
    g2 = (2 * np.pi * 2 / cell[0]) ** 2 + (2 * np.pi * 1 / cell[2]) ** 2
    lam = 1 + 2 * (4 * np.pi / g2) / (np.prod(cell) * abs(e[0] - e[1]))
    eps = O.eps_dense(phi, e, 1, n, cell)
    assert rel_fro(eps @ m, lam * m) < 1e-12
    assert rel_fro(O.eps_inv_dense(phi, e, 1, n, cell) @ m, m / lam) < 1e-12


def test_pair_space_smw_equals_dense_inverse():
    """Supplementary SMW on the exact pair matrix = dense LU inverse."""
    s = small_system(6, 2, 5, n_mu=10)
    a = O.pair_space_eps_inv(s.phi, s.energies, s.n_v, s.n, s.cell)
    b = O.eps_inv_dense(s.phi, s.energies, s.n_v, s.n, s.cell)
    assert rel_fro(a, b) < 1e-12
    for w in [0.3, 4.0]:
        a = O.pair_space_eps_inv(s.phi, s.energies, s.n_v, s.n, s.cell, omega=w)
        b = O.eps_inv_dense(s.phi, s.energies, s.n_v, s.n, s.cell, omega=w)
        assert rel_fro(a, b) < 1e-12


def test_capacitance_forms_and_smw_identity():
    """K = -D (I + G D)^-1 equals the paper's (B^-1/2 - G)^-1 for invertible B,
    and I + V Theta K Theta^T inverts I - 2 V Theta B Theta^T for random
    Theta, including a singular B."""
    rng = np.random.default_rng(3)
    k = 7
    a = rng.standard_normal((k, k))
    g = a @ a.T
    c = rng.standard_normal((k, 12))
    b = -(c * rng.uniform(0.5, 3.0, 12)) @ c.T          # negative definite, like C Omega^-1 C^T
    assert rel_fro(O.capacitance(g, b), O.capacitance_paper_form(g, b)) < 1e-11
    n, cell = (5, 4, 3), (2.5, 2.0, 1.5)
    theta = 0.3 * np.linalg.qr(rng.standard_normal((60, k)))[0]   # well-scaled basis
    g = O.coulomb_in_basis(theta, n, cell)
    for bb in (b, -(c[:, :4] * 2.0) @ c[:, :4].T):       # second B has rank 4 < 7
        kk = O.capacitance(g, bb)
        x = rng.standard_normal((60, 3))
        y = O.apply_eps_inv(theta, kk, x, n, cell)
        assert rel_fro(O.apply_eps_hat(theta, bb, y, n, cell), x) < 1e-12
        assert np.allclose(kk, kk.T, atol=1e-12 * np.abs(kk).max())


# ------------------------------------------------------------------- ISDF

def test_facesplit_gram_equals_m_c_transpose():
    s = small_system(6, 3, 4, n_mu=9)
    m = O.pair_matrix(s.phi, s.n_v)
    c = O.isdf_coefficients(s.phi, s.n_v, s.mu_idx)
    assert rel_fro(O.facesplit_gram(s.phi, s.n_v, s.mu_idx), m @ c.T) < 1e-13
    assert np.allclose(c, m[s.mu_idx])


def test_isdf_fit_is_least_squares_and_routes_agree():
    """Theta C is the orthogonal projection of M onto the row space of C:
    residual orthogonal to C (normal equations), same result as scipy lstsq,
    and the explicit-M and Hadamard routes agree."""
    s = small_system(6, 3, 5, n_mu=12)
    m = O.pair_matrix(s.phi, s.n_v)
    c = O.isdf_coefficients(s.phi, s.n_v, s.mu_idx)
    th, rank = O.isdf_fit(s.phi, s.n_v, s.mu_idx, explicit=True)
    th2, rank2 = O.isdf_fit(s.phi, s.n_v, s.mu_idx, explicit=False)
    assert rank == rank2 == 12
    res = m - th @ c
    assert np.abs(res @ c.T).max() < 1e-12 * np.abs(m).max() * np.abs(c).max() * c.shape[1]
    import scipy.linalg
    ls = scipy.linalg.lstsq(c.T, m.T)[0].T
    assert rel_fro(th, ls) < 1e-9
    assert rel_fro(th2, th) < 1e-8


def test_isdf_error_non_increasing_on_nested_points():
    """The ISDF error ||M - Theta C||_F cannot grow when points are added
    (projection onto a growing row space) and vanishes at full pair rank."""
    s = synth.workload("isdf16")
    m = O.pair_matrix(s.phi, s.n_v)
    errs = []
    for k in [16, 32, 64, 96, 112, 128]:
        th, _ = O.isdf_fit(s.phi, s.n_v, s.mu_idx[:k])
        errs.append(np.linalg.norm(m - th @ O.isdf_coefficients(s.phi, s.n_v, s.mu_idx[:k])))
    errs = np.array(errs) / np.linalg.norm(m)
    assert np.all(np.diff(errs) <= 1e-12), errs
    assert errs[0] > 0.1 and errs[-1] < 1e-10 and errs[-2] < 1e-10


def test_isdf_smw_exact_at_full_pair_rank():
    """North-star pin: with N_mu (128) above the pair rank (112) the
    ISDF-SMW inverse equals the dense 4096 x 4096 inverse of eps."""
    s = synth.workload("isdf16")
    x = synth.probe_block(s.n_r)
    res = O.isdf_smw_solve(s.phi, s.energies, s.n_v, s.mu_idx, s.n, s.cell, x)
    assert res.rank == s.n_v * s.n_c
    einv = O.eps_inv_dense(s.phi, s.energies, s.n_v, s.n, s.cell)
    assert rel_fro(res.y, einv @ x) < 1e-10


# ---------------------------------------------- symmetry and spectral bounds

def test_symmetries_and_spectral_bounds():
    """W = eps^-1 V and eps~^-1 are symmetric, eps^-1 is not; eps~ = I + X
    with X positive semidefinite, so eig(eps~^-1) lies in (0, 1] and
    ||X (I + X)^-1||_2 <= 1; K is negative semidefinite."""
    s = small_system(6, 3, 6, n_mu=18)
    phi, e, nv, n, cell = s.phi, s.energies, s.n_v, s.n, s.cell
    einv = O.eps_inv_dense(phi, e, nv, n, cell)
    w = O.screened_coulomb_dense(phi, e, nv, n, cell)
    et = O.eps_tilde_dense(phi, e, nv, n, cell)
    eti = np.linalg.inv(et)
    assert np.abs(w - w.T).max() < 1e-10 * np.abs(w).max()
    assert np.abs(eti - eti.T).max() < 1e-12
    assert np.abs(einv - einv.T).max() > 1e-3 * np.abs(einv).max()
    lam = np.linalg.eigvalsh(0.5 * (eti + eti.T))
    assert lam.min() > 0 and lam.max() <= 1 + 1e-12
    xm = et - np.eye(et.shape[0])
    assert np.linalg.eigvalsh(0.5 * (xm + xm.T)).min() > -1e-10
    assert np.linalg.norm(xm @ eti, 2) <= 1 + 1e-12
    # W = V^1/2 eps~^-1 V^1/2
    half = O.apply_coulomb(O.apply_coulomb(eti, n, cell, 0.5).T, n, cell, 0.5).T
    assert rel_fro(half, w) < 1e-10
    res = O.isdf_smw_solve(phi, e, nv, s.mu_idx, n, cell, np.eye(phi.shape[0])[:, :3])
    assert np.linalg.eigvalsh(0.5 * (res.k + res.k.T)).max() < 1e-12


def test_frequency_limits():
    """w = 0 is the static case; large w switches screening off (K -> 0)."""
    s = small_system(6, 2, 5, n_mu=10)
    x = synth.probe_block(s.n_r, 2)
    r0 = O.isdf_smw_solve(s.phi, s.energies, s.n_v, s.mu_idx, s.n, s.cell, x, omega=0.0)
    ref = O.eps_inv_dense(s.phi, s.energies, s.n_v, s.n, s.cell) @ x
    assert rel_fro(r0.y, ref) < 1e-10
    rbig = O.isdf_smw_solve(s.phi, s.energies, s.n_v, s.mu_idx, s.n, s.cell, x, omega=1e6)
    assert rel_fro(rbig.y, x) < 1e-9


def test_generator_orbitals_orthonormal_and_gapped():
    s = small_system(8, 3, 9, n_mu=20)
    assert np.abs(s.phi.T @ s.phi - np.eye(12)).max() < 1e-13
    assert s.energies[:3].max() < s.energies[3:].min()
    assert len(set(s.mu_idx.tolist())) == 20
