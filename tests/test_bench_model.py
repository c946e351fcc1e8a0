"""CPU checks of the bench line's rating arithmetic: the dominant-kernel roofline on the H
application's algorithmic bytes, its ALU share of the nominal FFT flops, the side-stream
ratings against one SM, and the tensor-core GEMM fractions, on hand-made stage timings of
the gs96 geometry (N = 96, |S| = 115,313, 128 states)."""
import math

import bench

GEO = dict(N=96, nG=115313, nstates=128, batch=128, ncols=0, yrows=61)
PK = dict(hbm=6800.0, bf16=1931.2, bf16_sus=1717.6, sm_max_mhz=2070.0, src="measured")


def test_hpsi_algorithmic_bytes_and_fft_flops():
    # packed psi in and H psi out (complex64) for every state, plus V (float) once
    assert bench.hpsi_algorithmic_bytes(GEO) == 2 * 115313 * 8 * 128 + 96 ** 3 * 4 == 239699968
    # two full 3D FFTs per state at 5 n log2 n
    assert math.isclose(bench.hpsi_fft_flops(GEO), 128 * 2 * 5 * 96 ** 3 * math.log2(96 ** 3))


def test_roofline_picks_the_main_stream_kernel_with_most_time():
    steps = 10
    entries = {"apply_h": (10.0, 10), "plane": (6.2, 10), "zinv": (1.1, 10), "zfwd": (1.4, 10),
               "rr_step": (8.8, 10), "cholesky": (2.1, 10), "gram": (1.4, 20), "rotate": (2.5, 20)}
    rl, name, side = bench.roofline(entries, GEO, PK, steps)
    # rr_step has more time but runs on the side stream: not the dominant main-stream kernel
    assert name == "plane" and rl["kernel"] == "plane"
    ms = 6.2 / 10
    assert math.isclose(rl["achieved"], 239699968 / (ms * 1e-3) / 1e9)
    assert math.isclose(rl["frac"], rl["achieved"] / PK["hbm"])
    assert rl["bound"] == "hbm" and rl["unit"] == "GB/s" and rl["peak"] == PK["hbm"]
    # the plane kernel's share (x and y passes: two thirds) of the nominal FFT flops
    flops = 2.0 / 3.0 * bench.hpsi_fft_flops(GEO)
    assert math.isclose(rl["alu"]["achieved"], flops / (ms * 1e-3) / 1e12)
    assert math.isclose(rl["alu"]["frac"], rl["alu"]["achieved"] / bench.FP32_PROBE_TFLOPS)
    # the side stream's one-CTA stages are rated against one SM's share of the peak
    sides = {s["kernel"]: s for s in side}
    assert set(sides) == {"rr_step", "cholesky"}
    assert all(math.isclose(s["peak"], bench.FP32_PEAK_TFLOPS / 152) for s in side)


def test_tensor_gemm_fractions():
    steps = 10
    entries = {"gram": (1.36, 20), "proj_gemm": (1.03, 10), "rotate": (2.50, 20)}
    out = bench.tensor_gemms(entries, GEO, PK, steps, 256)
    n, K = 128, 115313
    gram = out["gram"]
    assert gram["launches_per_step"] == 2 and gram["split_products"] == 3
    assert math.isclose(gram["flops_tensor_per_step"], 3 * 2 * 8.0 * n * n * K)
    assert math.isclose(gram["tflops_tensor"], gram["flops_tensor_per_step"] / (0.136e-3) / 1e12)
    assert math.isclose(gram["frac_of_bf16_peak"], gram["tflops_tensor"] / PK["bf16"])
    proj = out["proj_gemm"]
    assert math.isclose(proj["flops_algorithmic_per_step"], 8.0 * 256 * n * K)
    rot = out["rotate"]
    assert rot["split_products"] == 4
    assert math.isclose(rot["flops_tensor_per_step"], 4 * 2 * 8.0 * n * 2 * n * K)
    # a stage that did not run is left out
    assert "rotate" not in bench.tensor_gemms({"gram": (1.0, 20)}, GEO, PK, steps, 256)
