#!/usr/bin/env python
"""Throughput of the ISDF-SMW inverse dielectric matrix on GB300.

One step = one full solve of the hot path on one synthetic system: ISDF fit
(isdf_fit), polarizability and Coulomb operators in the ISDF basis
(build_polarizability, static w = 0), SMW capacitance (smw_inverse) and the
application of eps^-1 to 16 probe vectors (apply_eps_inv), all through the C
ABI.  Workload: the 48^3 grid (N_r = 110592), N_v = 64, N_c = 448,
N_mu = 1536 system of the synthetic generator (random combinations of the
lowest 1024 real plane waves, Lowdin-orthonormalised; occupied energies
uniform in [-10, -2] eV, unoccupied in [0, 20] eV; QRCP points).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

Under torchrun (N > 1) every rank solves its own copy of the system on its
own GPU (independent replicas, no data-path collective; barrier and
max-over-ranks timing only), so `value` is the whole-job solves/s.
`--impl reference` times the FP64 CPU oracle (the only reference there is:
the paper ships no code) on this host's cores, rank 0 only.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "ε^-1 (ISDF-SMW) solves/s and TFLOP/s vs plain FP64 GPU path at stated error"
WORKLOAD = "isdf48"
N_RHS = 16

# Peak of the FP64 pipe (the FP64 path has no tensor-core form on GB300):
# 152 SMs x 4 FP64 flop/clk (2 DFMA) x 2070 MHz maximum SM clock.  A DFMA
# throughput microbenchmark on this machine measured 1.20 TFLOP/s at ~1.97 GHz.
FP64_PEAK_TFLOPS = 152 * 4 * 2.070e9 / 1e12
# double-float products on the FP32 pipe: 128 lanes per SM, 12 FP32
# instructions per product (1 mul, 3 fma, 8 add / sub), 2 flops counted
DF_PEAK_TFLOPS = 152 * 128 * 2.070e9 / 12 * 2 / 1e12


def measured_peaks():
    """HBM copy bandwidth and BF16 dense GEMM rate measured on this GPU type
    (MEASURED_PEAKS.json beside this file), else the stated fallback."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]), "source": "of measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "of fallback"}


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) of
# the kernel a roofline cell names, from one ncu capture of this workload
# (profiles/tc_gemm_isdf48.md, one launch each of k_tc_gemm); absent until
# captured or once the kernel has changed since.
NCU_DRAM_BYTES = {
    "tc_gemm:coulomb_syrk": 1.444847e9 + 0.139929e9,
    "tc_gemm:fit_trsm": 1.677543e9 + 3.342264e9,
    "tc_gemm:fit_gram": 0.347267e9 + 0.964097e9,
    "tc_gemm:polar_d": 0.321547e9 + 0.021572e9,
}


def dominant_cell(cells):
    """The roofline cell: the tensor-core GEMM cell with the most time per
    step (k_tc_gemm takes the largest share of the serialised launch list,
    profiles/); the factorisation chains beside it run on other streams and
    their timers count the time their blocks wait for SMs.  Without a
    tensor-core cell, the cell with the most time per step."""
    tc = [c for c in cells if c["kernel"].startswith("tc_gemm:")]
    pool = tc or cells
    return max(pool, key=lambda c: c["ms_per_step"]) if pool else None

# BF16 slice products per FP32-grade product on the tensor-core path
# (three slices, pairs i + j < 3)
SLICE_PRODUCTS = 6


def kernel_roofline(fam, phase, ms, cnt, work, steps, peaks, workload="isdf48"):
    """Roofline of one (kernel family, phase) cell of the library's kernel
    timing: work per launch / average launch time against the peak of the
    unit that bounds the family."""
    sec = ms / 1e3
    cell = {"kernel": f"{fam}:{phase}", "launches_per_step": round(cnt / steps, 2),
            "ms_per_launch": round(ms / cnt, 4), "ms_per_step": round(ms / steps, 4)}
    if fam == "tc_gemm":
        # the library counts the BF16 MMA flops it issues (six slice products
        # per FP32-grade product); the roofline counts the method's own
        # flops only, one product per term
        issued = work / sec / 1e12
        ach = issued / SLICE_PRODUCTS
        cell.update({"bound": "tensor", "achieved": round(ach, 2), "peak": peaks["bf16_tflops"],
                     "unit": "TFLOP/s", "frac": round(ach / peaks["bf16_tflops"], 4),
                     "peak_source": f"bf16 dense burst {peaks['source']}",
                     "work": "algorithmic flops of the product (one per term; the split-precision slice "
                             "products are not counted)",
                     "issued_tflops": round(issued, 2), "issued_frac": round(issued / peaks["bf16_tflops"], 4),
                     "issued_work": f"BF16 MMA flops of the {SLICE_PRODUCTS} slice products"})
    elif fam in ("fp64_gemm", "chol_diag"):
        ach = work / sec / 1e12
        cell.update({"bound": "alu", "achieved": round(ach, 4), "peak": round(FP64_PEAK_TFLOPS, 4),
                     "unit": "TFLOP/s", "frac": round(ach / FP64_PEAK_TFLOPS, 4),
                     "peak_source": "derived: 152 SMs x 4 FP64 flop/clk x 2070 MHz (FP64 pipe)",
                     "work": "FP64 flops"})
    elif fam == "df_gemm":
        ach = work / sec / 1e12
        cell.update({"bound": "alu", "achieved": round(ach, 4), "peak": round(DF_PEAK_TFLOPS, 4),
                     "unit": "TFLOP/s", "frac": round(ach / DF_PEAK_TFLOPS, 4),
                     "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2070 MHz / 12 FP32 instructions per "
                                    "double-float product x 2 flops (FP32 pipe)",
                     "work": "flops of the FP64 update, carried in double-float"})
    else:
        ach = work / sec / 1e9
        cell.update({"bound": "hbm", "achieved": round(ach, 1), "peak": peaks["hbm_gbs"],
                     "unit": "GB/s", "frac": round(ach / peaks["hbm_gbs"], 4),
                     "peak_source": f"HBM copy {peaks['source']}",
                     "work": "algorithmic bytes (input read + output write)"})
    # the captures are of the isdf48 solve: another workload's cell of the same
    # name moves other bytes, so it has no traffic figure
    cell["traffic"] = NCU_DRAM_BYTES.get(cell["kernel"]) if workload == "isdf48" else None
    return cell


def algorithmic_flops(n_r, n_e, pairs, r, n_rhs, n_half2):
    """Flops each phase performs by the arithmetic of the method (not counting
    padding, wasted tile work or the extra products of the split precision):
    a GEMM m x n x k counts 2 m n k, a SYRK (lower triangle) m^2 k, a
    triangular solve m n^2, a Cholesky n^3 / 3 and a real 3-D FFT of length
    N 2.5 N log2 N per column (half of the complex 5 N log2 N)."""
    log2nr = math.log2(n_r)
    return {
        "points_chol": 2.0 * r * r * n_e + r ** 3 / 3.0,
        "fit_gram": 2.0 * n_r * r * n_e,
        "fit_trsm": float(n_r) * r * r,
        "coulomb_fft": 2.5 * n_r * log2nr * r,
        "coulomb_syrk": float(n_half2) * r * r,
        "polar_d": float(pairs) * r * r,
        "whiten_d": 2.0 * r ** 3,
        "smw": (2.0 / 3.0 + 4.0 + 1.0 + 1.0) * r ** 3,
        "apply": 4.0 * n_r * r * n_rhs + 2.0 * r * r * n_rhs + 5.0 * n_r * log2nr * n_rhs,
    }


# ----------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.tmp = None

    def start(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.tmp, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.tmp.flush()
        self.tmp.seek(0)
        rows = [ln.strip().split(",") for ln in self.tmp.read().splitlines() if ln.strip()]
        self.tmp.close()
        os.unlink(self.tmp.name)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for row in rows:
            row = [c.strip() for c in row]
            if len(row) < 9:
                continue
            try:
                sm.append(float(row[1]))
                smax = float(row[2])
            except ValueError:
                continue
            for nm, v in zip(names, row[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ helpers

def max_over_ranks(ms: float, device=None) -> float:
    """Largest value over all ranks (the job is as slow as its slowest rank)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms
    t = torch.tensor([ms], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world_size: int, steps: int, ms_total_max: float) -> float:
    """Whole-job solves/s: every rank solved `steps` systems in at most ms_total_max."""
    return world_size * steps / (ms_total_max / 1e3)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def make_system():
    import synth

    return synth.workload(WORKLOAD)


def oracle_solve(s, x):
    import oracle

    t0 = time.perf_counter()
    res = oracle.isdf_smw_solve(s.phi, s.energies, s.n_v, s.mu_idx, s.n, s.cell, x)
    return res, time.perf_counter() - t0


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def workload_config(s, extra=None):
    cfg = {
        "workload": (f"{WORKLOAD}: {s.n[0]}^3 grid (N_r={s.n_r}), N_v={s.n_v}, N_c={s.n_c}, "
                     f"N_mu={s.n_mu}, static omega=0, {N_RHS} probe vectors"),
        "n_r": s.n_r, "n_v": s.n_v, "n_c": s.n_c, "n_mu": s.n_mu, "n_rhs": N_RHS,
        "precision": "fp64",
        "l2": "inputs larger than L2 (phi 453 MB, theta 1.36 GB per solve)",
        "data": "seeded synthetic Gamma-point orbitals (stand-in for the paper's KSSOLV systems)",
    }
    if extra:
        cfg.update(extra)
    return cfg


# ------------------------------------------------------------- native arm

PREC = {"fp64": 0, "mixed": 1}
PREC_DETAIL = {
    "fp64": "every step in float64 on the FP64 pipe",
    "mixed": ("large contractions on tcgen05 tensor cores with operands cut into 3 BF16 slices "
              "(FP32 accumulation, FP64 sums over K blocks), FFT of theta in FP32; Cholesky "
              "factorisations and triangular inverses in FP64, their trailing updates in "
              "double-float (FP32 pairs, about 2^-46 relative)"),
}


def run_native(args):
    import torch
    import torch.distributed as dist

    import paper_2403_12340_gb300 as pkg

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    s = make_system()
    import synth

    x = synth.probe_block(s.n_r, N_RHS)

    # CPU baseline first (rank 0, one GPU): the oracle as it stands, one full solve
    cpu = None
    ref_y = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        res, t = oracle_solve(s, x)
        ref_y = res.y
        cpu = {"value": 1.0 / t, "unit": "solves/s", "cores": cpu_cores(), "kind": "oracle",
               "sample": f"one full {WORKLOAD} solve (fit, B, G, K, eps^-1 on {N_RHS} probes), "
                         f"{t:.1f} s, numpy/scipy FP64 with BLAS on all host cores"}

    pkg.load_library()
    stream = torch.cuda.current_stream(dev)
    phi = pkg.to_fortran(s.phi, dev)
    X = pkg.to_fortran(x, dev)
    theta = pkg.fortran_empty(s.n_r, s.n_mu, dev)
    Y = pkg.fortran_empty(s.n_r, N_RHS, dev)
    ctx = pkg.IsdfSmw(s.n, s.cell, stream)

    prec = PREC[args.prec]

    def step(phi_d, X_d, Y_d, p=None):
        ctx.fit(phi_d, s.n_v, s.n_c, s.mu_idx, theta, prec=prec if p is None else p)
        ctx.polarizability(s.energies, [0.0])
        ctx.smw(0)
        ctx.apply(X_d, 0, Y_d)

    def rel_err():
        if ref_y is None:
            return None
        y = Y.cpu().numpy()
        return float(np.linalg.norm(y - ref_y) / np.linalg.norm(ref_y))

    # the plain FP64 path on the same system, for the speedup at the stated error
    fp64 = None
    if prec != 0 and not args.no_fp64_compare:
        for _ in range(max(1, min(args.warmup, 2))):
            step(phi, X, Y, 0)
        torch.cuda.synchronize(dev)
        err64 = rel_err()
        k64 = max(1, min(args.steps, 3))
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(k64):
            step(phi, X, Y, 0)
        f1.record(stream)
        torch.cuda.synchronize(dev)
        ms64 = max_over_ranks(f0.elapsed_time(f1), dev)
        fp64 = {"value": round(job_throughput(ws, k64, ms64), 4), "unit": "solves/s",
                "ms_per_step": round(ms64 / k64, 3), "steps": k64, "rel_err_vs_oracle": err64}

    # tile autotuner: the first warm-up step times the GEMM tile candidates
    if args.autotune == "on":
        pkg.isdf_set_autotune(1)
    for _ in range(args.warmup):
        step(phi, X, Y)
    torch.cuda.synchronize(dev)
    pkg.isdf_set_autotune(0)
    tuned = pkg.isdf_autotune_table()
    err = rel_err()

    # ---- device-timed region: inputs resident in HBM
    sampler = None
    if rank == 0:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        sampler = ClockSampler(uuid if uuid.startswith("GPU-") else f"GPU-{uuid}")
    pkg.isdf_set_profiling(ctx.ctx, True)
    pkg.isdf_read_profile(ctx.ctx)
    pkg.isdf_read_kernel_profile(ctx.ctx)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    if sampler:
        sampler.start()
    n0 = pkg.isdf_launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step(phi, X, Y)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    launches = pkg.isdf_launch_count() - n0
    clocks = sampler.stop() if sampler else None
    prof = pkg.isdf_read_profile(ctx.ctx)
    kprof = pkg.isdf_read_kernel_profile(ctx.ctx)
    pkg.isdf_set_profiling(ctx.ctx, False)
    rank_r = ctx.rank
    ms_total = max_over_ranks(e0.elapsed_time(e1), dev)
    if ws > 1:
        dist.barrier()
    ms_step = ms_total / args.steps
    value = job_throughput(ws, args.steps, ms_total)

    # ---- end to end through the C ABI with host buffers (pinned), copies timed
    e2e = None
    if not args.no_e2e:
        phi_h = torch.from_numpy(np.ascontiguousarray(s.phi.T)).pin_memory()   # (N_e, N_r) = column-major phi
        x_h = torch.from_numpy(np.ascontiguousarray(x.T)).pin_memory()
        y_h = torch.empty((N_RHS, s.n_r), dtype=torch.float64).pin_memory()
        phi_t = torch.empty((s.n_e, s.n_r), dtype=torch.float64, device=dev)
        x_t = torch.empty((N_RHS, s.n_r), dtype=torch.float64, device=dev)
        k_e2e = max(1, min(args.steps, args.e2e_steps))

        def e2e_step():
            phi_t.copy_(phi_h, non_blocking=True)
            x_t.copy_(x_h, non_blocking=True)
            step(phi_t.t(), x_t.t(), Y)
            y_h.copy_(Y.t(), non_blocking=True)

        e2e_step()
        torch.cuda.synchronize(dev)
        if ws > 1:
            dist.barrier()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(k_e2e):
            e2e_step()
        a1.record(stream)
        torch.cuda.synchronize(dev)
        ms_e2e = max_over_ranks(a0.elapsed_time(a1), dev)
        e2e = {"value": job_throughput(ws, k_e2e, ms_e2e), "unit": "solves/s",
               "h2d_bytes_per_step": int(phi_h.numel() * 8 + x_h.numel() * 8 + s.mu_idx.nbytes + s.energies.nbytes + 8),
               "d2h_bytes_per_step": int(y_h.numel() * 8), "steps": k_e2e}

    # ---- roofline of the dominant kernel, timed per launch on its own stream
    n_half2 = 2 * (s.n[0] // 2 + 1) * s.n[1] * s.n[2]
    fl = algorithmic_flops(s.n_r, s.n_e, s.n_v * s.n_c, rank_r, N_RHS, n_half2)
    phases = {name: round(ms / args.steps, 3) for name, (ms, cnt) in prof.items() if cnt}
    flops_step = sum(fl.values())
    peaks = measured_peaks()
    cells = [kernel_roofline(f, p, ms, cnt, w, args.steps, peaks)
             for (f, p), (ms, cnt, w) in kprof.items() if cnt and ms > 0]
    cells.sort(key=lambda c: -c["ms_per_step"])
    roof = dominant_cell(cells)
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 4), "unit": "solves/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.prec == "fp64" else "bf16x3 (f32 accumulate) + f64",
            "data": "synthetic",
            "config": workload_config(s, {"parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                                          "rank": rank_r, "precision": args.prec,
                                          "precision_detail": PREC_DETAIL[args.prec],
                                          "autotune": autotune_summary(args, tuned)}),
            "flops_per_step": flops_step,
            "kernels": cells[:8], "phases_ms": phases,
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
            "clocks": clocks,
            # the figures a reader of the end of this line needs most come last
            "tflops": round(flops_step * value / 1e12, 4),
            "fp64_path": fp64,
            "speedup_vs_fp64": (round(value / fp64["value"], 3) if fp64 else None),
            "rel_err_vs_oracle": err,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        dist.destroy_process_group()


def autotune_summary(args, table):
    """How many GEMM shapes the tile autotuner timed and how many it moved
    off the built-in heuristic (tile width or split count)."""
    if args.autotune != "on":
        return "off"
    moved = [t for t in table if t["ms_best"] < t["ms_heuristic"]]
    saved = sum(t["ms_heuristic"] - t["ms_best"] for t in moved)
    return {"shapes": len(table), "changed": len(moved), "ms_saved_per_call_sum": round(saved, 3),
            "tiles_64": sum(1 for t in table if t["bn"] == 64)}


# ------------------------------------------------ full-frequency batch arm

BATCH_OMEGAS = 32


def _gen_batch_system(i):
    import synth

    return synth.batch_system(i)


def batch_systems():
    """The 16-system full-frequency set, generated in spawned host processes."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor

    import synth

    n = len(synth.BATCH_SYSTEMS)
    workers = max(1, min(8, cpu_cores() // 4))
    with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_gen_batch_system, range(n)))


# The bounded CPU sample of the full-frequency set: (system index, number of
# frequencies, None = all) -- the three smallest systems at every frequency
# and one of middle size (45^3, N_v 89) at two; about 15-30 s of oracle work
BATCH_CPU_SAMPLE = ((0, None), (1, None), (2, None), (8, 2))


def batch_system_flops(s, n_omega):
    """Algorithmic flops of one system of the set at n_omega frequencies: the
    fit and G once, D(w), its whitening and K(w) per frequency."""
    n_half2 = 2 * (s.n[0] // 2 + 1) * s.n[1] * s.n[2]
    fl = algorithmic_flops(s.n_r, s.n_e, s.n_v * s.n_c, s.n_mu, 0, n_half2)
    return (fl["points_chol"] + fl["fit_gram"] + fl["fit_trsm"] + fl["coulomb_fft"] + fl["coulomb_syrk"]
            + n_omega * (fl["polar_d"] + fl["whiten_d"] + fl["smw"]))


def oracle_batch_baseline(systems, omegas, sample=BATCH_CPU_SAMPLE, timer=None):
    """The oracle's rate on the whole set from a bounded sample of it: the
    sample's (system, frequency) units are timed, and the set's time is
    taken as the set's algorithmic flops at the sample's flop rate (the
    sample alone would overstate solves/s: its systems are the small ones).
    Returns (solves/s of the set, seconds timed, units timed, flop rate)."""
    timer = timer or oracle_batch_sample
    t = f_sample = 0.0
    units = 0
    for i, nw in sample:
        s = systems[min(i, len(systems) - 1)]
        om = omegas if nw is None else omegas[:nw]
        t += timer(s, om)
        f_sample += batch_system_flops(s, len(om))
        units += len(om)
    rate = f_sample / t
    f_all = sum(batch_system_flops(s, len(omegas)) for s in systems)
    return len(systems) * len(omegas) * rate / f_all, t, units, rate


def oracle_batch_sample(s, omegas):
    """The FP64 oracle on one system at every frequency: fit and G once, then
    B(w) and K(w) per frequency (the units the batch counts)."""
    import oracle as O

    t0 = time.perf_counter()
    theta, _ = O.isdf_fit(s.phi, s.n_v, s.mu_idx)
    g = O.coulomb_in_basis(theta, s.n, s.cell)
    pm = s.phi[s.mu_idx]
    for w in omegas:
        O.capacitance(g, O.polarizability(pm, s.energies, s.n_v, float(w)))
    return time.perf_counter() - t0


def run_batch(args):
    """Config 4: every system of the set at 32 imaginary frequencies per step,
    K(w) of every (system, frequency) pair; throughput and per-system latency."""
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2403_12340_gb300 as pkg
    import synth

    ws, rank, local = dist_env()
    systems = batch_systems()  # before CUDA starts (spawned processes)
    if ws > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    omegas, _ = synth.gauss_legendre_frequencies(BATCH_OMEGAS)
    for s in systems:
        s.phi_dev = pkg.to_fortran(s.phi, dev)
    n_sys = len(systems)
    batch = pkg.IsdfBatch(systems, prec=PREC[args.prec], n_workers=args.batch_workers)
    if args.autotune == "on":
        pkg.isdf_set_autotune(1)
    batch.run(omegas, n_workers=1)  # sizes every workspace; tunes the GEMM tiles one system at a time
    pkg.isdf_set_autotune(0)
    tuned = pkg.isdf_autotune_table()
    n0 = pkg.isdf_launch_count()
    batch.run(omegas)
    launches_per_run = pkg.isdf_launch_count() - n0
    graph = args.batch_mode == "graph"
    if graph:
        batch.capture(omegas)  # one eager run, then the graph of every system's device work
    for _ in range(max(1, args.warmup)):
        if graph:
            batch.replay()
        else:
            batch.run(omegas)

    # parity sample: the smallest system, first and last frequency, 4 probes
    err = None
    if rank == 0:
        import oracle as O

        s0 = systems[0]
        ctx0, _ = batch.context(0)
        x = synth.probe_block(s0.n_r, 4)
        X = pkg.to_fortran(x, dev)
        Y = pkg.fortran_empty(s0.n_r, 4, dev)
        errs = []
        for k in (0, BATCH_OMEGAS - 1):
            pkg.apply_eps_inv(ctx0, k, X, Y, s0.n_r)
            ref = O.isdf_smw_solve(s0.phi, s0.energies, s0.n_v, s0.mu_idx, s0.n, s0.cell, x, omega=float(omegas[k]))
            errs.append(float(np.linalg.norm(Y.cpu().numpy() - ref.y) / np.linalg.norm(ref.y)))
        err = max(errs)

    ctxs = [batch.context(i)[0] for i in range(n_sys)]
    sampler = None
    if rank == 0:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        sampler = ClockSampler(uuid if uuid.startswith("GPU-") else f"GPU-{uuid}")
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    if sampler:
        sampler.start()
    n0 = pkg.isdf_launch_count()
    lats, svcs, tot_ms = [], [], 0.0
    for _ in range(args.steps):
        if graph:
            lat, tot = batch.replay()
            svc = lat
        else:
            lat, svc, tot = batch.run(omegas)
        lats.append(lat)
        svcs.append(svc)
        tot_ms += tot
    torch.cuda.synchronize(dev)
    # a replay issues the kernels recorded in its graph: those of one eager run
    launches = launches_per_run * args.steps if graph else pkg.isdf_launch_count() - n0
    clocks = sampler.stop() if sampler else None
    ms_max = max_over_ranks(tot_ms, dev)
    # kernel timing: one more run with a single worker, so that no other
    # system's kernels share the GPU with the launch being timed
    for c in ctxs:
        pkg.isdf_set_profiling(c, True)
        pkg.isdf_read_profile(c)
        pkg.isdf_read_kernel_profile(c)
    _, _, prof_ms = batch.run(omegas, n_workers=1)
    kprof = {}
    for c in ctxs:
        for key, (ms, cnt, w) in pkg.isdf_read_kernel_profile(c).items():
            a = kprof.get(key, (0.0, 0, 0.0))
            kprof[key] = (a[0] + ms, a[1] + cnt, a[2] + w)
        pkg.isdf_set_profiling(c, False)
    solves = ws * n_sys * BATCH_OMEGAS * args.steps
    value = solves / (ms_max / 1e3)
    lat_all = np.concatenate(lats)
    svc_all = np.concatenate(svcs)

    flops_run = sum(batch_system_flops(s, BATCH_OMEGAS) for s in systems)
    peaks = measured_peaks()
    cells = [kernel_roofline(f, ph, ms, cnt, w, 1, peaks, workload="batch16")
             for (f, ph), (ms, cnt, w) in kprof.items() if cnt and ms > 0]
    cells.sort(key=lambda c: -c["ms_per_step"])
    for c in cells:
        c["timed_in"] = f"a one-worker run after the timed runs ({prof_ms:.0f} ms for the whole batch)"

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        v, t, units, rate = oracle_batch_baseline(systems, omegas)
        picked = ", ".join(f"{systems[min(i, n_sys - 1)].n[0]}^3/{systems[min(i, n_sys - 1)].n_v} at "
                           f"{BATCH_OMEGAS if nw is None else nw}" for i, nw in BATCH_CPU_SAMPLE)
        cpu = {"value": round(v, 4), "unit": "solves/s", "cores": cpu_cores(), "kind": "oracle",
               "sample": (f"{units} (system, frequency) units of the set (grid^3/N_v at frequencies: {picked}), "
                          f"fit and G once per system, B(w) and K(w) per frequency, {t:.1f} s of numpy/scipy "
                          f"FP64 at {rate / 1e9:.1f} GFLOP/s algorithmic; the value is the whole set's "
                          f"{n_sys * BATCH_OMEGAS} solves at that rate")}
    if rank == 0:
        sizes = ", ".join(f"{s.n[0]}^3/{s.n_v}" for s in systems)
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.prec == "fp64" else "bf16x3 (f32 accumulate) + f64", "data": "synthetic",
            "config": {"workload": (f"batch16: 16 systems (grid^3/N_v: {sizes}), N_c = 7 N_v, N_mu = 12 N_v, "
                                    f"{BATCH_OMEGAS} Gauss-Legendre imaginary frequencies each; a solve is "
                                    "K(w) of one (system, frequency)"),
                       "precision": args.prec, "precision_detail": PREC_DETAIL[args.prec],
                       "host_workers": args.batch_workers, "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                       "mode": ("one CUDA graph of every system's fit, polarizability and SMW at all frequencies, "
                                "one launch per step" if graph else "host worker threads, eager calls"),
                       "autotune": autotune_summary(args, tuned),
                       "l2": "inputs larger than L2 (phi 0.05-2.2 GB per system)",
                       "timing": "host wall clock around each run; a run returns after every system's GPU work"},
            "tflops": round(flops_run * args.steps * ws / (ms_max / 1e3) / 1e12, 3),
            "flops_per_step": flops_run,
            "latency_ms": {"p50": round(float(np.percentile(lat_all, 50)), 2),
                           "p99": round(float(np.percentile(lat_all, 99)), 2),
                           "kind": ("per system, from the start of the run to its last K(w)" if not graph else
                                    "per system, from the start of the graph to the end of its branch "
                                    "(events recorded inside the graph)")},
            "service_ms": {"p50": round(float(np.percentile(svc_all, 50)), 2),
                           "p99": round(float(np.percentile(svc_all, 99)), 2),
                           "kind": ("per system, from the start of its fit to its last K(w)" if not graph else
                                    "the graph starts every system at once: equal to the latency")},
            "kernels": cells[:8], "roofline": dominant_cell(cells),
            "cpu_baseline": cpu, "e2e": None,
            "e2e_note": "not measured for the batch: the default bench line carries the end-to-end number",
            "gpu_launches": int(launches), "clocks": clocks,
            "rel_err_vs_oracle": err,
        }
        print(json.dumps(line), flush=True)
    batch.close()
    if ws > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------- reference arm

def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return  # rank 0 alone runs the CPU oracle; the other ranks exit without work
    import synth

    s = make_system()
    x = synth.probe_block(s.n_r, N_RHS)
    for _ in range(args.warmup):
        oracle_solve(s, x)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_solve(s, x)
    t = time.perf_counter() - t0
    value = args.steps / t
    sample = (f"each step one full {WORKLOAD} solve (fit, B, G, K, eps^-1 on {N_RHS} probes) by the "
              f"FP64 numpy/scipy oracle")
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": "solves/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * t / args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(s, {"parallelism": "host cores, rank 0 only"}),
        "cpu_baseline": {"value": round(value, 5), "unit": "solves/s", "cores": cpu_cores(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 5), "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--prec", choices=["mixed", "fp64"], default="mixed",
                    help="mixed: split-BF16 tensor-core contractions (the headline); fp64: FP64 pipe only")
    ap.add_argument("--no-fp64-compare", action="store_true",
                    help="skip timing the plain FP64 path next to the mixed one")
    ap.add_argument("--workload", choices=["isdf48", "batch16"], default="isdf48",
                    help="isdf48: one 48^3 system (the default line); batch16: 16 systems x 32 frequencies")
    ap.add_argument("--batch-workers", type=int, default=4, help="host threads of the batch runner")
    ap.add_argument("--batch-mode", choices=["graph", "threads"], default="graph",
                    help="batch16: replay one captured CUDA graph per step, or drive eager calls from host threads")
    ap.add_argument("--autotune", choices=["on", "off"], default="on",
                    help="time the tensor-core GEMM tile candidates during the warm-up")
    args = ap.parse_args(argv)
    if args.warmup < 0 or args.steps < 1:
        ap.error("need --steps >= 1 and --warmup >= 0")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch16":
        run_batch(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
