"""GPU parity of the adjoint: W_P = P^T eps^-1 V P and the gradients of
L = tr(W_P Pj) with respect to the orbital energies and the orbital samples
at the points, CUDA (through the C ABI) against the FP64 oracle adjoint
(oracle/adjoint.py), against central finite differences of the CUDA
forward (h = 1e-6), and through torch.autograd.

Tolerance: 1e-10 relative (Frobenius) on W_P and on both gradients, the
FP64 target.  These quantities depend on the ISDF vectors P, which are well
determined only when C C^T is well conditioned and of full rank; every case
here is (cond(C C^T) = 9.3 at 48^3 / N_mu = 1536, where two different FP64
least-squares routes agree to 5e-15).  Finite differences: 1e-6 relative
(truncation h^2 plus rounding eps / h)."""
import numpy as np
import pytest

import oracle as O
import synth
from oracle import adjoint as A
from helpers import rel_fro, small_system

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2403_12340_gb300 as pkg

    pkg.load_library()


def _oracle(s, omega, pj):
    mu = np.asarray(s.mu_idx)
    theta, rank = O.isdf_fit(s.phi, s.n_v, mu)
    assert rank == len(mu)
    g = O.coulomb_in_basis(theta, s.n, s.cell)
    pm = s.phi[mu]
    w = A.screened_coulomb_basis(g, O.polarizability(pm, s.energies, s.n_v, omega))
    ge, gp = A.screened_loss_grad(g, pm, s.energies, s.n_v, pj.T, omega)
    return w, ge, gp


def _gpu(s, omega, pj, prec=0):
    import torch
    import paper_2403_12340_gb300 as pkg

    with pkg.IsdfSmw(s.n, s.cell) as sol:
        sol.fit(pkg.to_fortran(s.phi), s.n_v, s.n_c, s.mu_idx, prec=prec)
        sol.polarizability(s.energies, [omega])
        sol.smw(0)
        W = sol.screened_basis(0)
        ge, gp = sol.adjoint(pkg.to_fortran(pj.T), s.n_v + s.n_c)
        torch.cuda.synchronize()
        return W.cpu().numpy(), ge.cpu().numpy(), gp.cpu().numpy()


CASES = [  # (grid, n_v, n_c, n_mu, seed index, omega)
    (12, 3, 9, 20, 71, 0.0),
    (12, 3, 9, 20, 71, 0.35),
    ((10, 12, 9), 2, 10, 16, 72, 0.0),
    (16, 4, 12, 40, 73, 1.5),
]


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}-{c[1]}-{c[2]}-{c[3]}-w{c[5]}" for c in CASES])
def test_adjoint_matches_oracle(case):
    n, n_v, n_c, n_mu, seed, omega = case
    s = small_system(n, n_v, n_c, n_mu=n_mu, seed_index=seed)
    pj = A.random_projector(n_mu, seed=13)
    w_o, ge_o, gp_o = _oracle(s, omega, pj)
    w_g, ge_g, gp_g = _gpu(s, omega, pj)
    assert rel_fro(w_g, w_o) < TOL
    assert rel_fro(ge_g, ge_o) < TOL
    assert rel_fro(gp_g, gp_o) < TOL


def test_adjoint_matches_cuda_finite_differences():
    """Central differences of the CUDA forward itself (no oracle)."""
    import torch
    import paper_2403_12340_gb300 as pkg

    s = small_system(12, 3, 9, n_mu=20, seed_index=74)
    pj = A.random_projector(20, seed=13)
    h, omega = 1e-6, 0.2
    mu = np.asarray(s.mu_idx)
    with pkg.IsdfSmw(s.n, s.cell) as sol:
        sol.fit(pkg.to_fortran(s.phi), s.n_v, s.n_c, mu)

        def loss(e, pm):
            sol.set_point_orbitals(pkg.to_fortran(pm))
            sol.polarizability(e, [omega])
            sol.smw(0)
            return float(np.sum(sol.screened_basis(0).cpu().numpy() * pj.T))

        pm0 = s.phi[mu].copy()
        loss(s.energies, pm0)
        ge, gp = sol.adjoint(pkg.to_fortran(pj.T), s.n_v + s.n_c)
        ge, gp = ge.cpu().numpy(), gp.cpu().numpy()
        fe = np.empty_like(ge)
        for i in range(len(fe)):
            ep, em = s.energies.copy(), s.energies.copy()
            ep[i] += h
            em[i] -= h
            fe[i] = (loss(ep, pm0) - loss(em, pm0)) / (2 * h)
        rng = np.random.default_rng(5)
        picks = [(int(a), int(i)) for a, i in zip(rng.integers(0, 20, 24), rng.integers(0, 12, 24))]
        fp = np.empty(len(picks))
        for t, (a, i) in enumerate(picks):
            pp, pq = pm0.copy(), pm0.copy()
            pp[a, i] += h
            pq[a, i] -= h
            fp[t] = (loss(s.energies, pp) - loss(s.energies, pq)) / (2 * h)
        torch.cuda.synchronize()
    assert rel_fro(ge, fe) < 1e-6
    assert rel_fro(np.array([gp[a, i] for a, i in picks]), fp) < 1e-6


def test_autograd_function():
    """torch.autograd through the CUDA forward and adjoint equals the direct calls."""
    import torch
    import paper_2403_12340_gb300 as pkg

    s = small_system(12, 3, 9, n_mu=20, seed_index=75)
    pj = A.random_projector(20, seed=13)
    mu = np.asarray(s.mu_idx)
    _, ge_o, gp_o = _oracle(s, 0.0, pj)
    with pkg.IsdfSmw(s.n, s.cell) as sol:
        sol.fit(pkg.to_fortran(s.phi), s.n_v, s.n_c, mu)
        e = torch.tensor(s.energies, dtype=torch.float64, requires_grad=True)
        pm = pkg.to_fortran(s.phi[mu]).requires_grad_(True)
        W = pkg.screened_coulomb_basis(sol, e, pm, 0.0)
        loss = (W * torch.as_tensor(pj.T, device=W.device)).sum()
        loss.backward()
        torch.cuda.synchronize()
        assert rel_fro(e.grad.numpy(), ge_o) < TOL
        assert rel_fro(pm.grad.cpu().numpy(), gp_o) < TOL


def test_adjoint_states_and_errors():
    import paper_2403_12340_gb300 as pkg

    s = small_system(12, 3, 9, n_mu=20, seed_index=76)
    with pkg.IsdfSmw(s.n, s.cell) as sol:
        sol.fit(pkg.to_fortran(s.phi), s.n_v, s.n_c, s.mu_idx)
        sol.polarizability(s.energies, [0.0])
        with pytest.raises(pkg.IsdfError) as ei:
            sol.screened_basis(0)  # before smw_inverse
        assert ei.value.code == -9
        sol.smw(0)
        sol.set_point_orbitals(pkg.to_fortran(s.phi[np.asarray(s.mu_idx)]))
        with pytest.raises(pkg.IsdfError) as ei:
            sol.screened_basis(0)  # invalidated by the new samples
        assert ei.value.code == -9
        bad = s.phi[np.asarray(s.mu_idx)].copy()
        bad[3, 2] = np.nan
        with pytest.raises(pkg.IsdfError) as ei:
            sol.set_point_orbitals(pkg.to_fortran(bad))
        assert ei.value.code == -4


def test_adjoint_config_48():
    """48^3, N_v = 64, N_c = 448, N_mu = 1536, FP64 forward, static:
    W_P and both gradients of tr(W_P Pj), Pj = Q Q^T of a seeded
    1536 x 768 Gaussian, against the oracle adjoint."""
    s = synth.workload("isdf48")
    pj = A.random_projector(len(s.mu_idx), seed=13)
    w_o, ge_o, gp_o = _oracle(s, 0.0, pj)
    w_g, ge_g, gp_g = _gpu(s, 0.0, pj)
    assert rel_fro(w_g, w_o) < TOL
    assert rel_fro(ge_g, ge_o) < TOL
    assert rel_fro(gp_g, gp_o) < TOL


# ---- through the fit: dL/dPhi over the whole grid -------------------------

def _gpu_fit(s, omega, pj):
    import torch
    import paper_2403_12340_gb300 as pkg

    phi = pkg.to_fortran(s.phi)  # the fit keeps reading it: it must outlive the backward
    with pkg.IsdfSmw(s.n, s.cell) as sol:
        sol.fit(phi, s.n_v, s.n_c, s.mu_idx)
        sol.polarizability(s.energies, [omega])
        sol.smw(0)
        ge, gphi = sol.adjoint_fit(pkg.to_fortran(pj.T), s.n_v + s.n_c)
        torch.cuda.synchronize()
        return ge.cpu().numpy(), gphi.cpu().numpy()


FIT_CASES = [  # (grid, n_v, n_c, n_mu, seed index, omega)
    (12, 3, 9, 20, 71, 0.0),
    ((10, 12, 9), 2, 10, 16, 72, 0.35),
    (16, 4, 12, 40, 73, 1.5),
]


@pytest.mark.parametrize("case", FIT_CASES, ids=[f"{c[0]}-{c[1]}-{c[2]}-{c[3]}-w{c[5]}" for c in FIT_CASES])
def test_adjoint_fit_matches_oracle(case):
    n, n_v, n_c, n_mu, seed, omega = case
    s = small_system(n, n_v, n_c, n_mu=n_mu, seed_index=seed)
    pj = A.random_projector(n_mu, seed=13)
    ge_o, gp_o = A.fit_loss_grad(s.phi, s.energies, s.n_v, s.mu_idx, s.n, s.cell, pj.T, omega)
    ge_g, gp_g = _gpu_fit(s, omega, pj)
    assert rel_fro(ge_g, ge_o) < TOL
    assert rel_fro(gp_g, gp_o) < TOL


def test_adjoint_fit_autograd_and_rank_check():
    """torch.autograd through screened_coulomb_fit equals the direct call;
    a rank-deficient fit is refused."""
    import torch
    import paper_2403_12340_gb300 as pkg

    s = small_system(12, 3, 9, n_mu=20, seed_index=77)
    pj = A.random_projector(20, seed=13)
    ge_o, gp_o = A.fit_loss_grad(s.phi, s.energies, s.n_v, s.mu_idx, s.n, s.cell, pj.T, 0.2)
    with pkg.IsdfSmw(s.n, s.cell) as sol:
        phi = pkg.to_fortran(s.phi).requires_grad_(True)
        e = torch.tensor(s.energies, dtype=torch.float64, requires_grad=True)
        W = pkg.screened_coulomb_fit(sol, phi, e, s.n_v, s.mu_idx, 0.2)
        (W * torch.as_tensor(pj.T, device=W.device)).sum().backward()
        torch.cuda.synchronize()
        assert rel_fro(phi.grad.cpu().numpy(), gp_o) < TOL
        assert rel_fro(e.grad.numpy(), ge_o) < TOL
    d = small_system((8, 8, 8), 2, 3, 9, seed_index=78)  # 9 points > 6 pairs
    with pkg.IsdfSmw(d.n, d.cell) as sol:
        _, rank = sol.fit(pkg.to_fortran(d.phi), d.n_v, d.n_c, d.mu_idx)
        assert rank < 9
        sol.polarizability(d.energies, [0.0])
        sol.smw(0)
        with pytest.raises(pkg.IsdfError) as ei:
            sol.adjoint_fit(pkg.to_fortran(np.eye(9)), d.n_e)
        assert ei.value.code == -9


def test_adjoint_fit_config_48():
    """Config 5 (48^3, N_mu = 1536, FP64 forward, static): dL/dPhi over the
    grid and dL/de against the oracle, and central differences (h = 1e-6)
    of the CUDA forward on sampled orbital entries at interpolation points
    and elsewhere on the grid."""
    import torch
    import paper_2403_12340_gb300 as pkg

    s = synth.workload("isdf48")
    pj = A.random_projector(len(s.mu_idx), seed=13)
    ge_o, gp_o = A.fit_loss_grad(s.phi, s.energies, s.n_v, s.mu_idx, s.n, s.cell, pj.T, 0.0)
    ge_g, gp_g = _gpu_fit(s, 0.0, pj)
    assert rel_fro(ge_g, ge_o) < TOL
    assert rel_fro(gp_g, gp_o) < TOL
    h = 1e-6
    mu = np.asarray(s.mu_idx)
    rng = np.random.default_rng(5)
    rows = list(rng.choice(mu, 5, replace=False)) + list(rng.choice(np.setdiff1d(np.arange(s.n_r), mu), 5,
                                                                    replace=False))
    picks = [(int(a), int(i)) for a, i in zip(rows, rng.integers(0, s.n_e, 10))]
    pj_t = torch.as_tensor(pj.T, device="cuda")
    phi_d = pkg.to_fortran(s.phi)
    fd = []
    with pkg.IsdfSmw(s.n, s.cell) as sol:

        def loss():
            sol.fit(phi_d, s.n_v, s.n_c, mu)
            sol.polarizability(s.energies, [0.0])
            sol.smw(0)
            return float((sol.screened_basis(0) * pj_t).sum())

        for a, i in picks:
            v = float(s.phi[a, i])
            phi_d[a, i] = v + h
            lp = loss()
            phi_d[a, i] = v - h
            lm = loss()
            phi_d[a, i] = v
            fd.append((lp - lm) / (2 * h))
    err = rel_fro(np.array([gp_g[a, i] for a, i in picks]), np.array(fd))
    print(f"\nisdf48 dL/dPhi through the fit: vs oracle {rel_fro(gp_g, gp_o):.2e}, sampled central differences {err:.2e}")
    assert err < 1e-6
