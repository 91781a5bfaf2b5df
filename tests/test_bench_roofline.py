"""Host logic of bench.py's roofline cells: each kernel family is measured
against the peak of the unit that bounds it, achieved = work per launch /
average launch time, frac = achieved / peak.  CPU only."""
import pytest

import bench

PEAKS = {"hbm_gbs": 6779.0, "bf16_tflops": 1936.2, "source": "of measured"}


@pytest.mark.parametrize("fam,bound,unit,peak", [
    ("tc_gemm", "tensor", "TFLOP/s", PEAKS["bf16_tflops"]),
    ("fp64_gemm", "alu", "TFLOP/s", bench.FP64_PEAK_TFLOPS),
    ("chol_diag", "alu", "TFLOP/s", bench.FP64_PEAK_TFLOPS),
    ("df_gemm", "alu", "TFLOP/s", bench.DF_PEAK_TFLOPS),
    ("fft", "hbm", "GB/s", PEAKS["hbm_gbs"]),
    ("slice", "hbm", "GB/s", PEAKS["hbm_gbs"]),
])
def test_cell_units_and_fraction(fam, bound, unit, peak):
    # 20 launches over 2 steps, 10 ms in all, 3e12 flops (or 3e10 bytes) of work
    work = 3e12 if unit == "TFLOP/s" else 3e10
    c = bench.kernel_roofline(fam, "smw", 10.0, 20, work, 2, PEAKS)
    assert c["kernel"] == f"{fam}:smw"
    assert c["bound"] == bound and c["unit"] == unit
    assert c["launches_per_step"] == 10.0 and c["ms_per_step"] == 5.0 and c["ms_per_launch"] == 0.5
    achieved = work / 0.010 / (1e12 if unit == "TFLOP/s" else 1e9)
    if fam == "tc_gemm":
        # the library's work for this family is the issued BF16 MMA flops of the
        # slice products; the cell reports the method's flops (one product per
        # term) as achieved / frac and the issued rate beside them
        assert c["issued_tflops"] == pytest.approx(achieved, rel=1e-3)
        assert c["issued_frac"] == pytest.approx(achieved / peak, rel=1e-3)
        achieved /= bench.SLICE_PRODUCTS
    assert c["achieved"] == pytest.approx(achieved, rel=1e-3)
    assert c["peak"] == pytest.approx(peak, rel=1e-4)
    assert c["frac"] == pytest.approx(achieved / peak, rel=1e-3)
    assert c["traffic"] is None


def test_derived_peaks():
    # 152 SMs at 2070 MHz: 4 FP64 flop/clk; 128 FP32 lanes / 12 instructions x 2 flops
    assert bench.FP64_PEAK_TFLOPS == pytest.approx(1.2586, rel=1e-4)
    assert bench.DF_PEAK_TFLOPS == pytest.approx(6.7123, rel=1e-4)


def test_dominant_cell_prefers_tensor_gemm():
    """The roofline cell is the tensor-core GEMM cell with the most time per
    step, even when a factorisation chain's cell (timed on its own stream,
    waits included) reads longer; without a tensor-core cell, the longest
    cell.  Its traffic comes from the ncu table when the kernel is in it."""
    import bench

    peaks = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "of test"}
    cells = [bench.kernel_roofline("df_gemm", "points_chol", 30.0, 92, 1e10, 10, peaks),
             bench.kernel_roofline("tc_gemm", "fit_trsm", 28.0, 10, 1e13, 10, peaks),
             bench.kernel_roofline("tc_gemm", "coulomb_syrk", 20.0, 10, 1e13, 10, peaks)]
    roof = bench.dominant_cell(cells)
    assert roof["kernel"] == "tc_gemm:fit_trsm"
    assert roof["traffic"] == bench.NCU_DRAM_BYTES["tc_gemm:fit_trsm"]
    # the captured bytes are the isdf48 solve's: no figure for another workload's cell
    other = bench.kernel_roofline("tc_gemm", "fit_trsm", 28.0, 10, 1e13, 10, peaks, workload="batch16")
    assert other["traffic"] is None
    assert bench.dominant_cell(cells[:1])["kernel"] == "df_gemm:points_chol"
    assert bench.dominant_cell([]) is None


def test_batch_cpu_baseline_scales_the_sample_to_the_set():
    """The full-frequency set's CPU baseline: the sampled units are timed,
    and the set's time is its algorithmic flops at the sample's flop rate."""
    from types import SimpleNamespace

    import synth

    systems = [SimpleNamespace(n=(n, n, n), n_r=n ** 3, n_v=nv, n_c=7 * nv, n_e=8 * nv, n_mu=12 * nv)
               for n, nv in synth.BATCH_SYSTEMS]
    omegas = list(range(32))
    calls = []

    def timer(s, om):  # an oracle that runs at exactly 10 GFLOP/s
        calls.append((s.n[0], len(om)))
        return bench.batch_system_flops(s, len(om)) / 1e10

    v, t, units, rate = bench.oracle_batch_baseline(systems, omegas, timer=timer)
    assert calls == [(24, 32), (27, 32), (30, 32), (45, 2)]
    assert units == 3 * 32 + 2
    assert rate == pytest.approx(1e10)
    f_all = sum(bench.batch_system_flops(s, 32) for s in systems)
    assert v == pytest.approx(16 * 32 / (f_all / 1e10))
    # the sample alone would claim far more: its systems are the small ones
    assert units / t > 5 * v
    # a set smaller than the sample's indices takes its last system
    v2, _, _, _ = bench.oracle_batch_baseline(systems[:4], omegas, timer=timer)
    assert calls[-1] == (32, 2)
    assert v2 > v
