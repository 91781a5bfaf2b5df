"""GPU parity of the full-frequency (batched) path: every frequency's
polarizability, Cholesky factors, triangular inverses and SMW products in
batched launches (smw_inverse_all), against the FP64 oracle frequency by
frequency and against the one-frequency-at-a-time path.

Tolerances as for the single-frequency paths: 1e-10 (FP64), 1e-6 (mixed)
relative Frobenius error of eps^-1 X against the oracle."""
import numpy as np
import pytest

import oracle as O
import synth
from helpers import rel_fro, small_system

pytestmark = pytest.mark.gpu

TOL = {0: 1e-10, 1: 1e-6}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2403_12340_gb300 as pkg

    pkg.load_library()


def _run(s, omegas, x, prec, batched=True):
    import torch
    import paper_2403_12340_gb300 as pkg

    with pkg.IsdfSmw(s.n, s.cell) as sol:
        sol.fit(pkg.to_fortran(s.phi), s.n_v, s.n_c, s.mu_idx, prec=prec)
        sol.polarizability(s.energies, list(omegas))
        X = pkg.to_fortran(x)
        if batched:
            K = sol.smw_all(len(omegas), want_K=True)
            ks = [K[k].cpu().numpy() for k in range(len(omegas))]
        else:
            ks = [sol.smw(k, want_K=True).cpu().numpy() for k in range(len(omegas))]
        ys = [sol.apply(X, k).cpu().numpy() for k in range(len(omegas))]
        torch.cuda.synchronize()
    return ks, ys


CASES = [  # grid, n_v, n_c, n_mu, seed, number of frequencies
    (16, 4, 12, 40, 81, 5),
    ((12, 15, 10), 3, 9, 24, 82, 3),
    (18, 5, 20, 96, 83, 8),
]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}-{c[1]}-{c[2]}-{c[3]}-w{c[5]}" for c in CASES])
def test_batched_frequencies_match_oracle(case, prec):
    n, n_v, n_c, n_mu, seed, nw = case
    s = small_system(n, n_v, n_c, n_mu=n_mu, seed_index=seed)
    omegas, _ = synth.gauss_legendre_frequencies(nw)
    x = synth.probe_block(s.n_r, 4)
    ks, ys = _run(s, omegas, x, prec)
    ks1, _ = _run(s, omegas, x, prec, batched=False)
    for k, w in enumerate(omegas):
        ref = O.isdf_smw_solve(s.phi, s.energies, s.n_v, s.mu_idx, s.n, s.cell, x, omega=float(w))
        assert rel_fro(ys[k], ref.y) < TOL[prec], (k, w)
        assert rel_fro(ks[k], ks1[k]) < TOL[prec] * 10, (k, w)


def test_batched_config4_systems_sampled():
    """The two smallest systems of the 16-system full-frequency set, all 32
    Gauss-Legendre frequencies (mixed path), every fourth checked against the
    oracle."""
    omegas, _ = synth.gauss_legendre_frequencies(32)
    for i in (0, 1):
        s = synth.batch_system(i)
        x = synth.probe_block(s.n_r, 4)
        _, ys = _run(s, omegas, x, 1)
        for k in range(0, 32, 4):
            ref = O.isdf_smw_solve(s.phi, s.energies, s.n_v, s.mu_idx, s.n, s.cell, x, omega=float(omegas[k]))
            assert rel_fro(ys[k], ref.y) < TOL[1], (i, k)


def test_batched_config4_largest_system_two_frequencies():
    """The largest system of the 16-system set (60^3, N_v = 160, N_c = 1120,
    N_mu = 1920): every one of the 32 frequencies through the batched mixed
    path (smw_inverse_all), the first and the last checked against the
    oracle (fit and G once, B and K per frequency)."""
    omegas, _ = synth.gauss_legendre_frequencies(32)
    s = synth.batch_system(len(synth.BATCH_SYSTEMS) - 1)
    x = synth.probe_block(s.n_r, 4)
    _, ys = _run(s, omegas, x, 1)
    theta, rank = O.isdf_fit(s.phi, s.n_v, s.mu_idx)
    assert rank == s.n_mu
    g = O.coulomb_in_basis(theta, s.n, s.cell)
    pm = s.phi[np.asarray(s.mu_idx)]
    for k in (0, len(omegas) - 1):
        kk = O.capacitance(g, O.polarizability(pm, s.energies, s.n_v, float(omegas[k])))
        ref = O.apply_eps_inv(theta, kk, x, s.n, s.cell)
        assert rel_fro(ys[k], ref) < TOL[1], k


def test_smw_inverse_all_state_errors():
    import paper_2403_12340_gb300 as pkg

    s = small_system(12, 3, 9, n_mu=20, seed_index=84)
    with pkg.IsdfSmw(s.n, s.cell) as sol:
        sol.fit(pkg.to_fortran(s.phi), s.n_v, s.n_c, s.mu_idx)
        with pytest.raises(pkg.IsdfError) as ei:
            sol.smw_all(1)
        assert ei.value.code == -9


def test_batch_runner_many_systems():
    """isdf_batch_*: three systems of different sizes, four frequencies, two
    host workers; every system's eps^-1 X at every frequency against the
    oracle, and a second run of the same batch gives the same K."""
    import torch
    import paper_2403_12340_gb300 as pkg

    systems = [small_system(16, 4, 12, n_mu=40, seed_index=85), small_system((12, 15, 10), 3, 9, n_mu=24, seed_index=86),
               small_system(18, 5, 20, n_mu=96, seed_index=87)]
    omegas, _ = synth.gauss_legendre_frequencies(4)
    for s in systems:
        s.phi_dev = pkg.to_fortran(s.phi)
    for prec in (0, 1):
        batch = pkg.IsdfBatch(systems, prec=prec, n_workers=2)
        lat, svc, tot = batch.run(omegas)
        assert np.all(lat > 0) and np.all(svc > 0) and np.all(svc <= lat + 1e-6) and tot >= lat.max()
        for i, s in enumerate(systems):
            ctx, rank = batch.context(i)
            x = synth.probe_block(s.n_r, 3)
            X = pkg.to_fortran(x)
            Y = pkg.fortran_empty(s.n_r, 3, X.device)
            for k, w in enumerate(omegas):
                pkg.apply_eps_inv(ctx, k, X, Y, s.n_r)
                ref = O.isdf_smw_solve(s.phi, s.energies, s.n_v, s.mu_idx, s.n, s.cell, x, omega=float(w))
                assert rel_fro(Y.cpu().numpy(), ref.y) < TOL[prec], (prec, i, k)
        batch.run(omegas)
        torch.cuda.synchronize()
        batch.close()


def test_batch_graph_replay():
    """isdf_batch_capture / isdf_batch_replay: one CUDA graph of three
    systems' fits, all-frequency polarizabilities and SMW; the replay matches
    the oracle, and after the orbitals in the device buffers are replaced by
    other orbitals of the same shape a second replay matches the oracle for
    those (the graph recomputes from the buffers)."""
    import torch
    import paper_2403_12340_gb300 as pkg

    shapes = [(16, 4, 12, 32, 88), ((12, 15, 10), 3, 9, 18, 89), (18, 5, 20, 64, 90)]
    systems = [small_system(n, v, c, n_mu=m, seed_index=sd) for n, v, c, m, sd in shapes]
    omegas, _ = synth.gauss_legendre_frequencies(3)
    for s in systems:
        s.phi_dev = pkg.to_fortran(s.phi)
    for prec in (0, 1):
        for s in systems:  # the first orbitals again (the previous precision's replay replaced them)
            s.phi_dev.copy_(pkg.to_fortran(s.phi))
        batch = pkg.IsdfBatch(systems, prec=prec, n_workers=2)
        batch.capture(omegas)
        for rep in range(2):
            phis = []
            for i, s in enumerate(systems):
                if rep == 0:
                    phis.append(s.phi)
                else:  # other orbitals, same shape, same points and energies
                    n, v, c, m, sd = shapes[i]
                    phi2 = small_system(n, v, c, n_mu=m, seed_index=sd + 50).phi
                    s.phi_dev.copy_(pkg.to_fortran(phi2))
                    phis.append(phi2)
            torch.cuda.synchronize()
            lat, tot = batch.replay()
            assert np.all(lat > 0) and tot > 0
            for i, s in enumerate(systems):
                ctx, rank = batch.context(i)
                x = synth.probe_block(s.n_r, 3)
                X = pkg.to_fortran(x)
                Y = pkg.fortran_empty(s.n_r, 3, X.device)
                for k, w in enumerate(omegas):
                    pkg.apply_eps_inv(ctx, k, X, Y, s.n_r)
                    ref = O.isdf_smw_solve(phis[i], s.energies, s.n_v, s.mu_idx, s.n, s.cell, x, omega=float(w))
                    assert rel_fro(Y.cpu().numpy(), ref.y) < TOL[prec], (prec, rep, i, k)
        batch.close()


def test_batch_graph_needs_full_rank():
    """A system whose fit needs pivoting (N_mu above the pair count) cannot
    be captured: ISDF_ERR_STATE, and the eager run still works."""
    import paper_2403_12340_gb300 as pkg

    systems = [small_system(16, 4, 12, n_mu=32, seed_index=91), small_system(12, 2, 4, n_mu=12, seed_index=92)]
    for s in systems:
        s.phi_dev = pkg.to_fortran(s.phi)
    batch = pkg.IsdfBatch(systems, prec=0, n_workers=1)
    with pytest.raises(pkg.IsdfError) as ei:
        batch.capture([0.0])
    assert ei.value.code == -9
    with pytest.raises(pkg.IsdfError) as ei:
        batch.replay()
    assert ei.value.code == -9
    batch.run([0.0])
    batch.close()
