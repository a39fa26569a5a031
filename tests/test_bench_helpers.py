"""bench.py's per-step bookkeeping on the CPU: launches per step of each
step form and FFT length, and the roofline entry's kernel names, bounds and
traffic lookup (the per-phase times here are made up; only the bookkeeping
is checked)."""
import bench


def test_launches_per_step_of_each_form():
    # register path (N' <= 1024): row FFT, convolution, row kernel, and the
    # y sweep (GS form) or one launch of both sweep GEMMs (dense form)
    assert bench.launches_per_step(1024, dense=False) == 4
    assert bench.launches_per_step(1024, dense=True) == 4
    # shared-memory engine: the GS form's y sweep is transpose, row solve and
    # transpose with leapfrog; at N' = 8192 the convolution is three passes
    assert bench.launches_per_step(4096, dense=False) == 6
    assert bench.launches_per_step(4096, dense=True) == 4
    assert bench.launches_per_step(8192, dense=False) == 8
    assert bench.launches_per_step(8192, dense=True) == 6


def test_roofline_names_bounds_and_traffic():
    phase_ms = [0.019, 0.057, 0.044, 0.077]
    r = bench.roofline_of(phase_ms, 1023, 1024, True, 3, "n1023")
    assert list(r["kernels"]) == ["kr_rows_r2c", "kr_cols_conv", "kr_rows_solve<dense>", "k_tc_gemm(x+y)"]
    # the dominant phase is the merged sweep GEMM: it runs none of the
    # method's FFT flops, so its roofline is HBM on the method's 24 B per point
    # (x sweep 8, y sweep and leapfrog 16); the tensor work is a labelled
    # dense equivalent beside it
    assert r["kernel"] == "k_tc_gemm(x+y)" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["traffic"] == bench.NCU_TRAFFIC[("n1023", "k_tc_gemm(x+y)")]
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    pts = 3 * 1023 ** 2
    assert abs(r["achieved"] - 24 * pts / 77e-6 / 1e9) < 1e-6 * r["achieved"]
    assert r["peak"] == bench.peaks_of()["hbm_gbs"]
    de = r["dense_equivalent"]
    assert abs(de["tflops"] - 12.0 * 1023 ** 3 * 3 / 77e-6 / 1e12) < 1e-6 * de["tflops"]
    # the FFT kernels' intensities (~4, ~10 and ~3 flop/B) sit below the ridge
    # FP32 peak / HBM peak (~12 flop/B): HBM-bound
    for nm in ("kr_rows_r2c", "kr_cols_conv", "kr_rows_solve<dense>"):
        k = r["kernels"][nm]
        assert k["intensity_flop_per_byte"] < r["ridge_flop_per_byte"] and k["bound"] == "hbm", nm
    # the shared-memory engine's names; no capture -> no traffic; the GS row
    # solve (inverse FFT + Algorithm 1, ~28 flop/B at N' = 8192) is above the ridge
    r8 = bench.roofline_of([0.68, 1.82, 2.68, 2.24], 8191, 8192, False, 1, "n8191")
    assert list(r8["kernels"]) == ["k_rows_r2c", "k_conv3_a+b+c", "k_rows_solve",
                                  "k_transpose+k_rows_gs+k_transpose_leapfrog"]
    assert r8["kernel"] == "k_rows_solve" and r8["bound"] == "alu" and r8["unit"] == "TFLOP/s"
    assert r8["traffic"] is None
    r4 = bench.roofline_of([0.15, 0.41, 0.30, 0.58], 4095, 4096, True, 1, "n4095")
    assert "k_cols_conv" in r4["kernels"] and r4["kernel"] == "k_tc_gemm(x+y)"


def test_roofline_names_at_fft_length_2048():
    # N' = 2048: the dense form's FFT part runs on the register path, the GS
    # form on the shared-memory engine (y sweep on the transpose)
    phase_ms = [0.027, 0.068, 0.080, 0.100]
    rd = bench.roofline_of(phase_ms, 2047, 2048, True, 1, None)
    assert list(rd["kernels"]) == ["kr_rows_r2c", "kr_cols_conv", "kr_rows_solve<dense>", "k_tc_gemm(x+y)"]
    rg = bench.roofline_of(phase_ms, 2047, 2048, False, 1, None)
    assert list(rg["kernels"]) == ["k_rows_r2c", "k_cols_conv", "k_rows_solve",
                                  "k_transpose+k_rows_gs+k_transpose_leapfrog"]
    assert rd["traffic"] is None and rg["traffic"] is None
