"""Python binding of the ISDF-SMW C ABI (include/isdf_smw.h).

Argument marshalling only: every step of the computation runs in the CUDA
library `lib/libisdf_smw.so` (built by `build.py`).  There is no CPU or
PyTorch fallback: if the library is missing or fails to load, every call
raises.  PyTorch is used for device memory and streams.

Matrices are column-major (grid index fastest), as in the C ABI: a
N_r x k matrix is a float64 CUDA tensor of shape (N_r, k) with strides
(1, N_r); `fortran_empty` / `to_fortran` make such tensors.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libisdf_smw.so")

ISDF_OK = 0
ERRORS = {
    -1: "ISDF_ERR_ARG", -2: "ISDF_ERR_SHAPE", -3: "ISDF_ERR_INDEX", -4: "ISDF_ERR_NONFINITE",
    -5: "ISDF_ERR_ORDER", -6: "ISDF_ERR_NOT_SPD", -7: "ISDF_ERR_TIMEOUT", -8: "ISDF_ERR_CUDA",
    -9: "ISDF_ERR_STATE", -10: "ISDF_ERR_NOMEM",
}
ISDF_PREC_FP64 = 0
ISDF_PREC_MIXED = 1
ISDF_PREC_MIXED_PAIRS = 2

EXPORTED = ["isdf_create", "isdf_destroy", "isdf_fit", "build_polarizability", "smw_inverse",
            "apply_eps_inv", "isdf_fit_factor", "isdf_last_error", "isdf_version",
            "isdf_set_profiling", "isdf_read_profile", "isdf_phase_name", "isdf_launch_count",
            "apply_eps_inv_noalloc", "isdf_dgemm_split", "isdf_dgemm_split_error",
            "isdf_read_kernel_profile", "isdf_kernel_family_name", "isdf_set_point_orbitals",
            "isdf_screened_basis", "isdf_adjoint", "smw_inverse_all", "isdf_batch_create",
            "isdf_batch_destroy", "isdf_batch_run", "isdf_batch_context", "isdf_batch_last_error",
            "build_polarizability_contour", "isdf_contour_nodes", "isdf_cohsex", "isdf_batch_capture",
            "isdf_batch_replay", "isdf_set_autotune", "isdf_autotune_size", "isdf_autotune_entry",
            "isdf_autotune_clear", "isdf_device_allocations", "isdf_check_device_wait",
            "isdf_adjoint_fit", "isdf_read_kernel_trace", "isdf_set_refinement",
            "isdf_pair_weight_bounds", "isdf_ns_schedule"]
NUM_PHASES = 9
NUM_KERNEL_FAMILIES = 6


class IsdfError(RuntimeError):
    def __init__(self, code: int, message: str):
        self.code = code
        self.name = ERRORS.get(code, str(code))
        super().__init__(f"{self.name}: {message}")


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the CUDA library (once).  Raises if it is missing: no fallback."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"ISDF-SMW CUDA library not built: {path} is missing "
                          "(run __graft_entry__.build() or paper_2403_12340_gb300/build.py)")
    lib = ctypes.CDLL(path)
    P, I, D, L = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
    lib.isdf_create.argtypes = [ctypes.POINTER(P), I, I, I, D, D, D, P]
    lib.isdf_destroy.argtypes = [P]
    lib.isdf_fit.argtypes = [P, P, I, I, P, I, I, P, ctypes.POINTER(I)]
    lib.build_polarizability.argtypes = [P, P, P, I, P, P]
    lib.smw_inverse.argtypes = [P, I, P]
    lib.apply_eps_inv.argtypes = [P, I, P, I, P]
    lib.isdf_fit_factor.argtypes = [P, P, P]
    lib.isdf_last_error.argtypes = [P]
    lib.isdf_last_error.restype = ctypes.c_char_p
    lib.isdf_version.argtypes = []
    lib.isdf_version.restype = ctypes.c_char_p
    LL = ctypes.c_longlong
    lib.isdf_dgemm_split.argtypes = [I, I, I, D, P, LL, P, LL, D, P, LL, I, P]
    lib.isdf_dgemm_split.restype = I
    lib.isdf_dgemm_split_error.argtypes = []
    lib.isdf_dgemm_split_error.restype = ctypes.c_char_p
    lib.apply_eps_inv_noalloc.argtypes = [P, I, P, I, P]
    lib.apply_eps_inv_noalloc.restype = I
    lib.isdf_set_profiling.argtypes = [P, I]
    lib.isdf_read_profile.argtypes = [P, P, P]
    lib.isdf_phase_name.argtypes = [I]
    lib.isdf_phase_name.restype = ctypes.c_char_p
    lib.isdf_batch_create.argtypes = [P, P, I, I, I]
    lib.isdf_batch_destroy.argtypes = [P]
    lib.isdf_batch_run.argtypes = [P, P, I, I, P, P, P]
    lib.isdf_batch_context.argtypes = [P, I, P, P]
    lib.isdf_set_autotune.argtypes = [I]
    lib.isdf_autotune_size.argtypes = []
    lib.isdf_autotune_entry.argtypes = [I, P, P, P]
    lib.isdf_autotune_clear.argtypes = []
    lib.isdf_autotune_clear.restype = None
    lib.isdf_batch_capture.argtypes = [P, P, I]
    lib.isdf_batch_replay.argtypes = [P, P, P]
    for name in ["isdf_batch_create", "isdf_batch_destroy", "isdf_batch_run", "isdf_batch_context",
                 "isdf_batch_capture", "isdf_batch_replay"]:
        getattr(lib, name).restype = I
    lib.isdf_batch_last_error.argtypes = [P]
    lib.isdf_batch_last_error.restype = ctypes.c_char_p
    lib.build_polarizability_contour.argtypes = [P, P, I, P, P]
    lib.build_polarizability_contour.restype = I
    lib.isdf_contour_nodes.argtypes = [P, I, I, D]
    lib.isdf_contour_nodes.restype = I
    lib.isdf_pair_weight_bounds.argtypes = [P, I, I, D, ctypes.POINTER(D), ctypes.POINTER(D)]
    lib.isdf_pair_weight_bounds.restype = I
    lib.isdf_ns_schedule.argtypes = [D, I, P, P]
    lib.isdf_ns_schedule.restype = I
    lib.isdf_cohsex.argtypes = [P, P, P, P]
    lib.isdf_cohsex.restype = I
    lib.smw_inverse_all.argtypes = [P, P]
    lib.smw_inverse_all.restype = I
    lib.isdf_set_point_orbitals.argtypes = [P, P, LL]
    lib.isdf_screened_basis.argtypes = [P, I, P]
    lib.isdf_adjoint.argtypes = [P, I, P, P, P]
    lib.isdf_adjoint_fit.argtypes = [P, I, P, P, P]
    for name in ["isdf_set_point_orbitals", "isdf_screened_basis", "isdf_adjoint", "isdf_adjoint_fit"]:
        getattr(lib, name).restype = I
    lib.isdf_read_kernel_trace.argtypes = [P, I, P, P, P, P, P, P]
    lib.isdf_read_kernel_trace.restype = I
    lib.isdf_read_kernel_profile.argtypes = [P, P, P, P]
    lib.isdf_read_kernel_profile.restype = I
    lib.isdf_kernel_family_name.argtypes = [I]
    lib.isdf_kernel_family_name.restype = ctypes.c_char_p
    lib.isdf_launch_count.argtypes = []
    lib.isdf_launch_count.restype = ctypes.c_longlong
    lib.isdf_set_refinement.argtypes = [P, I]
    lib.isdf_set_refinement.restype = I
    lib.isdf_check_device_wait.argtypes = [P, ctypes.c_longlong]
    lib.isdf_check_device_wait.restype = I
    lib.isdf_device_allocations.argtypes = []
    lib.isdf_device_allocations.restype = ctypes.c_longlong
    for name in ["isdf_create", "isdf_destroy", "isdf_fit", "build_polarizability", "smw_inverse",
                 "apply_eps_inv", "isdf_fit_factor", "isdf_set_profiling", "isdf_read_profile"]:
        getattr(lib, name).restype = I
    _lib = lib
    return lib


def _check(rc: int, ctx) -> None:
    if rc != ISDF_OK:
        msg = load_library().isdf_last_error(ctx)
        raise IsdfError(rc, msg.decode() if msg else "")


def _dev_ptr(t, rows: Optional[int] = None, cols: Optional[int] = None, name: str = "tensor") -> int:
    """Device pointer of a float64 CUDA tensor laid out column-major."""
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float64:
        raise TypeError(f"{name} must be float64")
    if t.dim() == 1:
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    elif t.dim() == 2:
        r, c = t.shape
        if c > 1 and t.stride() != (1, r):
            raise ValueError(f"{name} must be column-major (strides (1, rows)); use to_fortran()")
        if c == 1 and t.stride(0) != 1:
            raise ValueError(f"{name} must have unit row stride")
        if rows is not None and r != rows:
            raise ValueError(f"{name} has {r} rows, expected {rows}")
        if cols is not None and c != cols:
            raise ValueError(f"{name} has {c} columns, expected {cols}")
    else:
        raise ValueError(f"{name} must be 1-D or 2-D")
    return t.data_ptr()


def fortran_empty(rows: int, cols: int, device="cuda"):
    import torch

    return torch.empty((cols, rows), dtype=torch.float64, device=device).t()


def to_fortran(a, device="cuda"):
    """Column-major float64 CUDA copy of a 2-D numpy array or tensor."""
    import torch

    t = torch.as_tensor(np.asarray(a) if not isinstance(a, torch.Tensor) else a, dtype=torch.float64)
    out = fortran_empty(t.shape[0], t.shape[1], device)
    out.copy_(t.to(device))
    return out


def version() -> str:
    return load_library().isdf_version().decode()


def isdf_last_error(ctx) -> str:
    msg = load_library().isdf_last_error(ctx)
    return msg.decode() if msg else ""


def isdf_create(n: Sequence[int], cell: Sequence[float], stream=None):
    """Create a context on the current CUDA device; returns an opaque handle."""
    lib = load_library()
    h = ctypes.c_void_p()
    s = ctypes.c_void_p(0 if stream is None else int(stream))
    _check(lib.isdf_create(ctypes.byref(h), int(n[0]), int(n[1]), int(n[2]), float(cell[0]),
                           float(cell[1]), float(cell[2]), s), None)
    return h


def isdf_destroy(ctx) -> None:
    _check(load_library().isdf_destroy(ctx), None)


def _is_cuda_tensor(t) -> bool:
    return type(t).__module__.startswith("torch") and getattr(t, "is_cuda", False)


def isdf_fit(ctx, phi, n_v: int, n_c: int, mu_idx, theta, n_r: int, prec: int = ISDF_PREC_FP64) -> int:
    """ISDF fit; writes theta (N_r x N_mu) and returns the numerical rank.
    mu_idx: host indices (anything numpy takes) or a contiguous int64 CUDA
    tensor, which the library reads from device memory."""
    if _is_cuda_tensor(mu_idx):
        import torch

        if mu_idx.dtype != torch.int64 or mu_idx.dim() != 1 or not mu_idx.is_contiguous():
            raise TypeError("mu_idx on the device must be a contiguous 1-D int64 tensor")
        pm, n_mu, keep = mu_idx.data_ptr(), int(mu_idx.shape[0]), mu_idx
    else:
        keep = np.ascontiguousarray(np.asarray(mu_idx, dtype=np.int64))
        pm, n_mu = keep.ctypes.data, int(keep.shape[0])
    pp = _dev_ptr(phi, n_r, n_v + n_c, "phi")
    pt = _dev_ptr(theta, n_r, n_mu, "theta")
    rank = ctypes.c_int(0)
    _check(load_library().isdf_fit(ctx, pp, int(n_v), int(n_c), pm, n_mu, int(prec), pt, ctypes.byref(rank)), ctx)
    del keep
    return rank.value


def build_polarizability(ctx, energies, omega, D_out=None, G_out=None) -> None:
    e = np.ascontiguousarray(np.asarray(energies, dtype=np.float64))
    w = np.ascontiguousarray(np.atleast_1d(np.asarray(omega, dtype=np.float64)))
    pd = 0 if D_out is None else _dev_ptr(D_out.reshape(-1), name="D_out")
    pg = 0 if G_out is None else _dev_ptr(G_out.reshape(-1), name="G_out")
    _check(load_library().build_polarizability(ctx, e.ctypes.data, w.ctypes.data, int(w.shape[0]), pd, pg),
           ctx)


def build_polarizability_contour(ctx, energies, n_nodes: int, D_out=None, G_out=None) -> None:
    e = np.ascontiguousarray(np.asarray(energies, dtype=np.float64))
    pd = 0 if D_out is None else _dev_ptr(D_out.reshape(-1), name="D_out")
    pg = 0 if G_out is None else _dev_ptr(G_out.reshape(-1), name="G_out")
    _check(load_library().build_polarizability_contour(ctx, e.ctypes.data, int(n_nodes), pd, pg), ctx)


def isdf_set_autotune(on) -> int:
    """Turn the tensor-core GEMM tile autotuner on (1) or off (0), or record
    the narrowest tiles without timing (2); returns the previous setting."""
    return int(load_library().isdf_set_autotune(2 if on == 2 else (1 if on else 0)))


def isdf_autotune_table():
    """The autotuner's table: a list of dicts (shape key, chosen tile width
    and splits, best and heuristic ms per call)."""
    lib = load_library()
    out = []
    key = (ctypes.c_int * 8)()
    ch = (ctypes.c_int * 2)()
    ms = (ctypes.c_double * 2)()
    for i in range(lib.isdf_autotune_size()):
        if lib.isdf_autotune_entry(i, key, ch, ms) != 0:
            break
        out.append({"M": key[0], "N": key[1], "Kp": key[2], "slices": key[3], "lower": key[4], "tri_b": key[5],
                    "count": key[6], "max_split": key[7], "bn": ch[0], "splits": ch[1], "ms_best": ms[0],
                    "ms_heuristic": ms[1]})
    return out


def isdf_autotune_clear() -> None:
    load_library().isdf_autotune_clear()


def isdf_contour_nodes(energies, n_v: int, n_c: int, tol: float) -> int:
    e = np.ascontiguousarray(np.asarray(energies, dtype=np.float64))
    n = load_library().isdf_contour_nodes(e.ctypes.data, int(n_v), int(n_c), float(tol))
    if n < 0:
        raise IsdfError(n, "isdf_contour_nodes: bad arguments or no gap")
    return n


def pair_weight_bounds(energies, n_v: int, n_c: int, w: float):
    """(wmin, wmax) of the pair weights 2 d / (d^2 + w^2), d = e_c - e_v (host only)."""
    e = np.ascontiguousarray(np.asarray(energies, dtype=np.float64))
    lo, hi = ctypes.c_double(), ctypes.c_double()
    rc = load_library().isdf_pair_weight_bounds(e.ctypes.data, int(n_v), int(n_c), float(w), ctypes.byref(lo),
                                                ctypes.byref(hi))
    if rc != 0:
        raise IsdfError(rc, "isdf_pair_weight_bounds")
    return lo.value, hi.value


def ns_schedule(kappa: float):
    """(beta, slices) of the Newton-Schulz steps for a spectrum in [1, kappa],
    or None when the route would take more than 12 steps (host only)."""
    beta = np.zeros(12, dtype=np.float64)
    slices = np.zeros(12, dtype=np.int32)
    n = load_library().isdf_ns_schedule(float(kappa), 12, beta.ctypes.data, slices.ctypes.data)
    if n < 0:
        raise IsdfError(n, "isdf_ns_schedule")
    return None if n == 0 else (beta[:n].copy(), slices[:n].copy())


def isdf_cohsex(ctx_vc, ctx_vn, ctx_nn, n_e: int, device="cuda"):
    """(SEX_X, X, COH) band self-energies (n_e each, device tensors)."""
    import torch

    sig = torch.empty(3 * n_e, dtype=torch.float64, device=device)
    _check(load_library().isdf_cohsex(ctx_vc, ctx_vn, ctx_nn, _dev_ptr(sig, name="sigma")), ctx_vc)
    return sig[:n_e], sig[n_e:2 * n_e], sig[2 * n_e:]


def smw_inverse(ctx, omega_index: int = 0, K_out=None) -> None:
    pk = 0 if K_out is None else _dev_ptr(K_out.reshape(-1), name="K_out")
    _check(load_library().smw_inverse(ctx, int(omega_index), pk), ctx)


def smw_inverse_all(ctx, K_out=None) -> None:
    pk = 0 if K_out is None else _dev_ptr(K_out.reshape(-1), name="K_out")
    _check(load_library().smw_inverse_all(ctx, pk), ctx)


def apply_eps_inv(ctx, omega_index: int, X, Y, n_r: int) -> None:
    n_rhs = X.shape[1] if X.dim() == 2 else 1
    px = _dev_ptr(X, n_r, None, "X")
    py = _dev_ptr(Y, n_r, n_rhs, "Y")
    _check(load_library().apply_eps_inv(ctx, int(omega_index), px, int(n_rhs), py), ctx)


def isdf_set_point_orbitals(ctx, phimu, n_mu: int, n_e: int) -> None:
    """Replace the orbital samples at the points (n_mu x n_e, column-major)."""
    _check(load_library().isdf_set_point_orbitals(ctx, _dev_ptr(phimu, n_mu, n_e, "phimu"), int(n_mu)), ctx)


def isdf_screened_basis(ctx, omega_index: int, W_out, n_mu: int) -> None:
    _check(load_library().isdf_screened_basis(ctx, int(omega_index), _dev_ptr(W_out, n_mu, n_mu, "W_out")), ctx)


def isdf_adjoint(ctx, omega_index: int, W_bar, grad_e, grad_phimu, n_mu: int, n_e: int) -> None:
    _check(load_library().isdf_adjoint(ctx, int(omega_index), _dev_ptr(W_bar, n_mu, n_mu, "W_bar"),
                                       _dev_ptr(grad_e, name="grad_energies"),
                                       _dev_ptr(grad_phimu, n_mu, n_e, "grad_phimu")), ctx)


def isdf_adjoint_fit(ctx, omega_index: int, W_bar, grad_e, grad_phi, n_mu: int, n_r: int, n_e: int) -> None:
    _check(load_library().isdf_adjoint_fit(ctx, int(omega_index), _dev_ptr(W_bar, n_mu, n_mu, "W_bar"),
                                           _dev_ptr(grad_e, name="grad_energies"),
                                           _dev_ptr(grad_phi, n_r, n_e, "grad_phi")), ctx)


def isdf_fit_factor(ctx, n_mu: int, L_out=None):
    """Pivot order (host int32 array) of the last fit; fills L_out if given."""
    piv = np.zeros(n_mu, dtype=np.int32)
    pl = 0 if L_out is None else _dev_ptr(L_out.reshape(-1), name="L_out")
    _check(load_library().isdf_fit_factor(ctx, piv.ctypes.data, pl), ctx)
    return piv


def isdf_set_refinement(ctx, steps: int) -> None:
    _check(load_library().isdf_set_refinement(ctx, int(steps)), ctx)


def isdf_set_profiling(ctx, on: bool) -> None:
    _check(load_library().isdf_set_profiling(ctx, 1 if on else 0), ctx)


def isdf_read_profile(ctx):
    """{phase name: (milliseconds, intervals)} since the last read (syncs the stream)."""
    ms = np.zeros(NUM_PHASES, dtype=np.float64)
    cnt = np.zeros(NUM_PHASES, dtype=np.int32)
    _check(load_library().isdf_read_profile(ctx, ms.ctypes.data, cnt.ctypes.data), ctx)
    lib = load_library()
    return {lib.isdf_phase_name(i).decode(): (float(ms[i]), int(cnt[i])) for i in range(NUM_PHASES)}


def isdf_read_kernel_profile(ctx):
    """{(family, phase): (milliseconds, launches, work)} of the timed kernel
    launches since the last read (syncs the device); work is flops for the
    GEMM / Cholesky families and bytes for "fft" and "slice"."""
    n = NUM_KERNEL_FAMILIES * NUM_PHASES
    ms = np.zeros(n, dtype=np.float64)
    cnt = np.zeros(n, dtype=np.int32)
    work = np.zeros(n, dtype=np.float64)
    lib = load_library()
    _check(lib.isdf_read_kernel_profile(ctx, ms.ctypes.data, cnt.ctypes.data, work.ctypes.data), ctx)
    out = {}
    for f in range(NUM_KERNEL_FAMILIES):
        for p in range(NUM_PHASES):
            i = f * NUM_PHASES + p
            if cnt[i]:
                out[(lib.isdf_kernel_family_name(f).decode(), lib.isdf_phase_name(p).decode())] = (
                    float(ms[i]), int(cnt[i]), float(work[i]))
    return out


def isdf_read_kernel_trace(ctx, max_records: int = 100000):
    """Launch-by-launch record of the timed kernels since the last read:
    a list of (start_ms, end_ms, family, phase, work, stream)."""
    lib = load_library()
    t0 = np.zeros(max_records)
    t1 = np.zeros(max_records)
    fam = np.zeros(max_records, dtype=np.int32)
    ph = np.zeros(max_records, dtype=np.int32)
    wk = np.zeros(max_records)
    st = np.zeros(max_records, dtype=np.int32)
    n = lib.isdf_read_kernel_trace(ctx, int(max_records), t0.ctypes.data, t1.ctypes.data, fam.ctypes.data,
                                   ph.ctypes.data, wk.ctypes.data, st.ctypes.data)
    if n < 0:
        raise IsdfError(n, isdf_last_error(ctx))
    fn = [lib.isdf_kernel_family_name(i).decode() for i in range(NUM_KERNEL_FAMILIES)]
    pn = [lib.isdf_phase_name(i).decode() for i in range(NUM_PHASES)]
    return [(float(t0[i]), float(t1[i]), fn[fam[i]], pn[ph[i]] if 0 <= ph[i] < NUM_PHASES else "?", float(wk[i]),
             int(st[i])) for i in range(n)]


def isdf_dgemm_split(A, B, C, alpha=1.0, beta=0.0, nslices=3, stream=None) -> None:
    """C = alpha A B^T + beta C on the tensor cores (float64 CUDA tensors,
    column-major: A M x K, B N x K, C M x N)."""
    import torch

    M, K = A.shape
    N = B.shape[0]
    pa = _dev_ptr(A, M, K, "A")
    pb = _dev_ptr(B, N, K, "B")
    pc = _dev_ptr(C, M, N, "C")
    s = torch.cuda.current_stream().cuda_stream if stream is None else int(stream)
    lib = load_library()
    rc = lib.isdf_dgemm_split(M, N, K, float(alpha), pa, max(M, 1), pb, max(N, 1), float(beta), pc, max(M, 1),
                              int(nslices), ctypes.c_void_p(s))
    if rc != ISDF_OK:
        raise IsdfError(rc, lib.isdf_dgemm_split_error().decode())


def isdf_launch_count() -> int:
    return int(load_library().isdf_launch_count())


def isdf_check_device_wait(ctx, limit_ns: int) -> int:
    """Run the library's bounded grid barrier on a barrier that never
    completes; returns the status code (ISDF_ERR_TIMEOUT, -7, when the bound
    works) without raising."""
    return int(load_library().isdf_check_device_wait(ctx, int(limit_ns)))


def isdf_device_allocations() -> int:
    """Device allocations the library has made in this process so far."""
    return int(load_library().isdf_device_allocations())


class IsdfSmw:
    """One context bound to one grid; thin convenience over the C ABI."""

    def __init__(self, n, cell, stream=None):
        import torch

        self.n = tuple(int(v) for v in n)
        self.cell = tuple(float(v) for v in cell)
        self.n_r = int(np.prod(self.n))
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.ctx = isdf_create(self.n, self.cell, self.stream.cuda_stream)
        self.n_mu = 0
        self.rank = 0

    def close(self):
        if self.ctx is not None:
            isdf_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def fit(self, phi, n_v, n_c, mu_idx, theta=None, prec=ISDF_PREC_FP64):
        mu = mu_idx if _is_cuda_tensor(mu_idx) else np.asarray(mu_idx, dtype=np.int64)
        if theta is None:
            theta = fortran_empty(self.n_r, mu.shape[0], phi.device)
        self.rank = isdf_fit(self.ctx, phi, n_v, n_c, mu, theta, self.n_r, prec)
        self.n_mu = int(mu.shape[0])
        self.phi = phi  # the library reads the orbitals again after the fit
        self.theta = theta
        return theta, self.rank

    def polarizability(self, energies, omega=(0.0,), want_D=False, want_G=False):
        import torch

        w = np.atleast_1d(np.asarray(omega, dtype=np.float64))
        dev = self.theta.device
        D = torch.empty((w.shape[0], self.n_mu, self.n_mu), dtype=torch.float64, device=dev) if want_D else None
        G = torch.empty((self.n_mu, self.n_mu), dtype=torch.float64, device=dev) if want_G else None
        build_polarizability(self.ctx, energies, w, D, G)
        return D, G

    def polarizability_contour(self, energies, n_nodes, want_D=False, want_G=False):
        """Static D by the contour integral of Algorithm 2 (one frequency, w = 0)."""
        import torch

        dev = self.theta.device
        D = torch.empty((1, self.n_mu, self.n_mu), dtype=torch.float64, device=dev) if want_D else None
        G = torch.empty((self.n_mu, self.n_mu), dtype=torch.float64, device=dev) if want_G else None
        build_polarizability_contour(self.ctx, energies, n_nodes, D, G)
        return D, G

    def smw(self, omega_index=0, want_K=False):
        import torch

        K = torch.empty((self.n_mu, self.n_mu), dtype=torch.float64, device=self.theta.device) if want_K else None
        smw_inverse(self.ctx, omega_index, K)
        return K

    def smw_all(self, n_omega, want_K=False):
        """K for every frequency of the last polarizability (batched)."""
        import torch

        K = (torch.empty((n_omega, self.n_mu, self.n_mu), dtype=torch.float64, device=self.theta.device)
             if want_K else None)
        smw_inverse_all(self.ctx, K)
        return K

    def apply(self, X, omega_index=0, Y=None):
        if Y is None:
            Y = fortran_empty(self.n_r, X.shape[1], X.device)
        apply_eps_inv(self.ctx, omega_index, X, Y, self.n_r)
        return Y

    def set_point_orbitals(self, phimu):
        """Orbital samples at the points (n_mu x n_e) for the next polarizability."""
        t = phimu if phimu.stride() == (1, self.n_mu) else to_fortran(phimu, phimu.device)
        isdf_set_point_orbitals(self.ctx, t, self.n_mu, t.shape[1])

    def screened_basis(self, omega_index=0):
        """W_P = P^T eps^-1 V P (n_mu x n_mu, points order) for one frequency."""
        W = fortran_empty(self.n_mu, self.n_mu, self.theta.device)
        isdf_screened_basis(self.ctx, omega_index, W, self.n_mu)
        return W

    def adjoint(self, W_bar, n_e, omega_index=0):
        """(dL/de, dL/dphi_mu) for dL/dW_P = W_bar."""
        import torch

        wb = W_bar if (W_bar.dim() == 2 and W_bar.stride() == (1, self.n_mu)) else to_fortran(W_bar, W_bar.device)
        ge = torch.empty(n_e, dtype=torch.float64, device=self.theta.device)
        gp = fortran_empty(self.n_mu, n_e, self.theta.device)
        isdf_adjoint(self.ctx, omega_index, wb, ge, gp, self.n_mu, n_e)
        return ge, gp

    def adjoint_fit(self, W_bar, n_e, omega_index=0):
        """(dL/de, dL/dPhi over the grid) for dL/dW_P = W_bar, with the ISDF
        vectors differentiated through the fit."""
        import torch

        wb = W_bar if (W_bar.dim() == 2 and W_bar.stride() == (1, self.n_mu)) else to_fortran(W_bar, W_bar.device)
        ge = torch.empty(n_e, dtype=torch.float64, device=self.theta.device)
        gphi = fortran_empty(self.n_r, n_e, self.theta.device)
        isdf_adjoint_fit(self.ctx, omega_index, wb, ge, gphi, self.n_mu, self.n_r, n_e)
        return ge, gphi

    def factor(self, want_L=False):
        import torch

        L = torch.empty((self.n_mu, self.n_mu), dtype=torch.float64, device=self.theta.device) if want_L else None
        piv = isdf_fit_factor(self.ctx, self.n_mu, L)
        # the library writes L column-major; the transposed view is L itself
        return piv, (L.t() if L is not None else None)


def _autograd_function():
    import torch

    class ScreenedCoulombBasis(torch.autograd.Function):
        """W_P(e, phi_mu) = P^T eps^-1(i w) V P with the ISDF vectors of a
        fitted IsdfSmw held fixed (the checkpoint).  forward runs the CUDA
        polarizability, SMW and projection; backward runs the CUDA adjoint.
        Between a forward and its backward the solver must not be used for
        another polarizability."""

        @staticmethod
        def forward(fctx, solver, energies, phi_mu, omega):
            solver.set_point_orbitals(phi_mu.detach())
            solver.polarizability(energies.detach().cpu().numpy(), [float(omega)])
            solver.smw(0)
            W = solver.screened_basis(0)
            fctx.solver = solver
            fctx.n_e = phi_mu.shape[1]
            fctx.e_device = energies.device
            return W

        @staticmethod
        def backward(fctx, gW):
            ge, gp = fctx.solver.adjoint(gW, fctx.n_e, 0)
            return None, ge.to(fctx.e_device), gp, None

    return ScreenedCoulombBasis


def _fit_autograd_function():
    import torch

    class ScreenedCoulombFit(torch.autograd.Function):
        """W_P(Phi, e) = P^T eps^-1(i w) V P with P refitted from the orbitals
        on the whole grid (FP64).  forward runs the CUDA fit, polarizability,
        SMW and projection; backward runs the CUDA adjoint through the fit,
        which recomputes what it needs from theta (the checkpoint).  Between
        a forward and its backward the solver must not be refitted."""

        @staticmethod
        def forward(fctx, solver, phi, energies, n_v, mu_idx, omega):
            solver.fit(phi.detach(), n_v, phi.shape[1] - n_v, mu_idx)
            solver.polarizability(energies.detach().cpu().numpy(), [float(omega)])
            solver.smw(0)
            fctx.solver = solver
            fctx.n_e = phi.shape[1]
            fctx.e_device = energies.device
            return solver.screened_basis(0)

        @staticmethod
        def backward(fctx, gW):
            ge, gphi = fctx.solver.adjoint_fit(gW, fctx.n_e, 0)
            return None, gphi, ge.to(fctx.e_device), None, None, None

    return ScreenedCoulombFit


def screened_coulomb_fit(solver, phi, energies, n_v, mu_idx, omega=0.0):
    """Differentiable W_P = P^T eps^-1 V P as a function of the orbitals on
    the grid (column-major N_r x N_e CUDA tensor) and the energies."""
    return _fit_autograd_function().apply(solver, phi, energies, n_v, mu_idx, omega)


def screened_coulomb_basis(solver, energies, phi_mu, omega=0.0):
    """Differentiable W_P = P^T eps^-1 V P (torch.autograd) on a fitted solver."""
    return _autograd_function().apply(solver, energies, phi_mu, omega)


class _System(ctypes.Structure):
    _fields_ = [("n1", ctypes.c_int), ("n2", ctypes.c_int), ("n3", ctypes.c_int),
                ("L1", ctypes.c_double), ("L2", ctypes.c_double), ("L3", ctypes.c_double),
                ("phi", ctypes.c_void_p), ("n_v", ctypes.c_int), ("n_c", ctypes.c_int),
                ("mu_idx", ctypes.c_void_p), ("n_mu", ctypes.c_int), ("energies", ctypes.c_void_p)]


class IsdfBatch:
    """Many systems, all frequencies (isdf_batch_* of the C ABI).  systems:
    objects with n, cell, n_v, n_c, mu_idx, energies and a column-major
    float64 CUDA tensor `phi_dev` (N_r x N_e), kept alive here."""

    def __init__(self, systems, prec=ISDF_PREC_FP64, n_workers=4):
        lib = load_library()
        self._keep = []
        arr = (_System * len(systems))()
        for i, s in enumerate(systems):
            mu = np.ascontiguousarray(np.asarray(s.mu_idx, dtype=np.int64))
            e = np.ascontiguousarray(np.asarray(s.energies, dtype=np.float64))
            n_r = int(np.prod(s.n))
            pp = _dev_ptr(s.phi_dev, n_r, s.n_v + s.n_c, "phi_dev")
            self._keep += [mu, e, s.phi_dev]
            arr[i] = _System(s.n[0], s.n[1], s.n[2], s.cell[0], s.cell[1], s.cell[2], pp, s.n_v, s.n_c,
                             mu.ctypes.data, mu.shape[0], e.ctypes.data)
        h = ctypes.c_void_p()
        rc = lib.isdf_batch_create(ctypes.byref(h), ctypes.cast(arr, ctypes.c_void_p), len(systems), int(prec),
                                   int(n_workers))
        if rc != ISDF_OK:
            raise IsdfError(rc, (lib.isdf_batch_last_error(None) or b"").decode())
        self.h = h
        self.n = len(systems)

    def run(self, omega, n_workers=0):
        """(latency_ms, service_ms, total_ms) of one run over all systems
        (n_workers 0: the number given at creation)."""
        lib = load_library()
        w = np.ascontiguousarray(np.atleast_1d(np.asarray(omega, dtype=np.float64)))
        lat = np.zeros(self.n)
        svc = np.zeros(self.n)
        tot = ctypes.c_double(0.0)
        rc = lib.isdf_batch_run(self.h, w.ctypes.data, int(w.shape[0]), int(n_workers), lat.ctypes.data,
                                svc.ctypes.data, ctypes.byref(tot))
        if rc != ISDF_OK:
            raise IsdfError(rc, (lib.isdf_batch_last_error(self.h) or b"").decode())
        return lat, svc, tot.value

    def capture(self, omega):
        """Eager run at omega, then one CUDA graph of every system's device
        work (isdf_batch_capture)."""
        lib = load_library()
        w = np.ascontiguousarray(np.atleast_1d(np.asarray(omega, dtype=np.float64)))
        self._graph_omega = w
        rc = lib.isdf_batch_capture(self.h, w.ctypes.data, int(w.shape[0]))
        if rc != ISDF_OK:
            raise IsdfError(rc, (lib.isdf_batch_last_error(self.h) or b"").decode())

    def replay(self):
        """(latency_ms per system, total_ms) of one launch of the captured graph."""
        lib = load_library()
        lat = np.zeros(self.n)
        tot = ctypes.c_double(0.0)
        rc = lib.isdf_batch_replay(self.h, lat.ctypes.data, ctypes.byref(tot))
        if rc != ISDF_OK:
            raise IsdfError(rc, (lib.isdf_batch_last_error(self.h) or b"").decode())
        return lat, tot.value

    def context(self, i):
        """(context handle, rank) of system i."""
        c = ctypes.c_void_p()
        r = ctypes.c_int(0)
        lib = load_library()
        rc = lib.isdf_batch_context(self.h, int(i), ctypes.byref(c), ctypes.byref(r))
        if rc != ISDF_OK:
            raise IsdfError(rc, (lib.isdf_batch_last_error(self.h) or b"").decode())
        return c, r.value

    def close(self):
        if getattr(self, "h", None) is not None:
            load_library().isdf_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
