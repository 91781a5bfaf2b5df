"""Run one ISDF-SMW solve through the C ABI on the GPU (tests only)."""
import numpy as np

import paper_2403_12340_gb300 as pkg


def run_gpu(system, x, omegas=(0.0,), want=False, in_place=False, prec=0):
    """Fit, polarizability, SMW and apply for every frequency; returns host arrays."""
    import torch

    out = {}
    with pkg.IsdfSmw(system.n, system.cell) as s:
        phi = pkg.to_fortran(system.phi)
        theta, rank = s.fit(phi, system.n_v, system.n_c, system.mu_idx, prec=prec)
        D, G = s.polarizability(system.energies, list(omegas), want_D=want, want_G=want)
        ys, ks = [], []
        X = pkg.to_fortran(x)
        for k in range(len(omegas)):
            K = s.smw(k, want_K=want)
            if in_place:
                Y = pkg.to_fortran(X)
                s.apply(Y, k, Y)
            else:
                Y = s.apply(X, k)
            ys.append(Y.cpu().numpy())
            if want:
                ks.append(K.cpu().numpy())
        piv, L = s.factor(want_L=True)
        torch.cuda.synchronize()
        out["rank"] = rank
        out["y"] = ys
        out["piv"] = piv
        out["L"] = L.cpu().numpy()
        out["theta"] = theta.cpu().numpy() if want else None
        if want:
            out["D"] = D.cpu().numpy()
            out["G"] = G.cpu().numpy()
            out["K"] = ks
    return out
