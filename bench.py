#!/usr/bin/env python
"""Benchmark of the Kohn-Sham hot path on one GB300 (N GPUs: independent replicas).

Workload ``gs96`` (the ground-state block-iteration cell): L = 30 bohr, 96^3 grid,
|S| = 115,313 plane waves (20 Ha), 128 states, 64 atoms on a perturbed fcc lattice,
Gaussian V_loc (depth -3 Ha, width 0.8 bohr), 4 KB projectors per atom.  One step is one
steepest-descent block iteration through the C ABI: CholQR (Gram GEMM, FP64 Cholesky,
rotation) -> H psi for all 128 states -> Rayleigh-Ritz (GEMM, eigensolver, two
rotations) -> SD update.  Mixed precision (complex64 states and FFTs).

value = 128 * 96^3 state-gridpoints per step / step time (device CUDA events, L2 flushed
between timed steps).  Extra keys: H psi alone, the all-FP64 GPU path, a real-time ETRS
step of the 128^3 / 512-state cell, the live per-kernel roofline, the CPU oracle timed on
a bounded sample, and the end-to-end figure with host buffers.

--impl reference times the FP64 CPU oracle (plain numpy, tests' reference) on the same
workload, one block iteration on a bounded sample of the states per step.
"""
import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Hψ state·gridpts/s & %HBM roofline, mixed vs FP64; TD steps/s; serve p50/p99"
UNIT = "state·gridpts/s"
WORKLOAD = "gs96"
CPU_SAMPLE_STATES = 4
BASE_SERVE_SEED = 20210612
SERVE_WORKERS = 32


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return dict(hbm=d["hbm_gbs"], bf16=d["bf16_tflops"], bf16_sus=d["bf16_tflops_sustained"],
                    sm_max_mhz=d.get("sm_max_mhz", 2070.0), src="measured")
    return dict(hbm=6800.0, bf16=1900.0, bf16_sus=1700.0, sm_max_mhz=2070.0, src="fallback")


# ------------------------------------------------------------------------------------------------
# CPU leg: the oracle as it stands, on a bounded sample (runs in a child process, 1 thread)
# ------------------------------------------------------------------------------------------------
def cpu_leg(nsteps, warmup, nsample):
    from oracle import ks_oracle as ko
    from paper_2106_03872_gb300 import inputs
    cell = inputs.cell(WORKLOAD)
    ref = ko.Cell(cell)
    c = inputs.random_coeffs(cell["seed"], cell["nstates"], ref.nG)[:nsample]
    for _ in range(warmup):
        ko.block_iteration(ref, c, 1)
    times = []
    for _ in range(nsteps):
        t0 = time.perf_counter()
        ko.block_iteration(ref, c, 1)
        times.append(time.perf_counter() - t0)
    return dict(times=times, nsample=nsample, N=ref.N)


def cpu_td_leg(nsample=2):
    """The oracle's real-time step on the td128 cell (ETRS + Taylor 4 with Hartree + Slater,
    dt = 0.05) for a sample of its states, one step, one thread; the full 512-state step time
    is extrapolated by the state count (the H applications and the density are per state; the
    per-step potential, counted once per sample, makes this an upper estimate).  Opt-in
    (--cpu-td-leg): a full-size oracle step takes hours."""
    from oracle import ks_oracle as ko
    from paper_2106_03872_gb300 import inputs
    cell = inputs.cell("td128")
    ref = ko.Cell(cell)
    q, _ = ko.cholqr(inputs.random_coeffs(cell["seed"], nsample, ref.nG))
    t0 = time.perf_counter()
    ko.td_run(ref, q, 0.05, 1, "etrs", True)
    dt = time.perf_counter() - t0
    return {"cell": "td128", "sample_states": nsample, "s_per_sample_step": dt,
            "extrapolated_s_per_step": dt / nsample * cell["nstates"], "nstates": cell["nstates"], "threads": 1,
            "kind": "oracle", "host": platform.machine()}


def run_cpu_leg(nsteps, warmup, nsample):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-leg", "--steps", str(nsteps), "--warmup", str(warmup),
           "--sample", str(nsample)]
    r = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=1800)
    if r.returncode != 0:
        raise RuntimeError("cpu leg failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def run_cpu_leg_all(nsteps, warmup, nsample, nproc=None):
    """The same bounded sample on every host core: nproc independent 1-thread oracle processes
    at once (the block iterations of different samples are independent problems); returns the
    legs of all of them."""
    nproc = nproc or os.cpu_count() or 1
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-leg", "--steps", str(nsteps), "--warmup", str(warmup),
           "--sample", str(nsample)]
    procs = [subprocess.Popen(cmd, env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)
             for _ in range(nproc)]
    legs = []
    for p in procs:
        out, err = p.communicate(timeout=1800)
        if p.returncode != 0:
            raise RuntimeError("cpu leg failed: " + err[-2000:])
        legs.append(json.loads(out.strip().splitlines()[-1]))
    return legs


def cpu_baseline_obj(leg, legs_all=None):
    t = sum(leg["times"]) / len(leg["times"])
    one = {"value": leg["nsample"] * leg["N"] ** 3 / t, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": "one block iteration (CholQR, H psi, Rayleigh-Ritz, SD update) of %d of the 128 states of "
                     "the %s cell, FP64 numpy oracle, 1 thread; mean of %d steps" % (
                         leg["nsample"], WORKLOAD, len(leg["times"]))}
    if not legs_all:
        return one
    value = sum(l["nsample"] * l["N"] ** 3 / (sum(l["times"]) / len(l["times"])) for l in legs_all)
    return {"value": value, "unit": UNIT, "cores": len(legs_all), "kind": "oracle",
            "sample": "%d concurrent 1-thread oracle processes (one per host core, nproc = %d), each one block "
                      "iteration of %d of the 128 states of the %s cell per step; throughputs summed" % (
                          len(legs_all), os.cpu_count() or 1, leg["nsample"], WORKLOAD),
            "one_core": one}


# ------------------------------------------------------------------------------------------------
# Clock sampling during the timed region
# ------------------------------------------------------------------------------------------------
class Clocks:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------------------------------
# Roofline of the dominant kernel (stage timings from the library's CUDA events)
# ------------------------------------------------------------------------------------------------
# ALU peaks from unit counts and clocks: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz; FP64 is
# GB300's nominal 1.25 TFLOP/s (an FMA probe measured 69.5 and 1.195 TFLOP/s)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
FP64_PEAK_TFLOPS = 1.25


def max_over_ranks(ms, dist, device):
    """Job time of replicas: the slowest rank's time (every rank must call this)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def replica_throughput(world, units_per_rank, job_ms):
    """Whole-job throughput: units every rank processed / the job time (weak scaling)."""
    return world * units_per_rank / (job_ms * 1e-3)


def stage_model(name, geo, pk, fp32_tflops):
    """(bound, algorithmic amount per launch, peak, unit) for a timed stage, or None."""
    N, nG, ns, ncols = geo["N"], geo["nG"], geo["nstates"], geo.get("ncols", 0)
    c64 = 8
    if name == "eigh":
        # Householder tridiagonalisation (16/3) n^3 + back-transformation 8 n^3 real flops
        # (complex), Newton-Schulz/bisection/twisted factorisation are lower order
        return "alu", (16.0 / 3.0 + 8.0) * ns ** 3, FP32_PEAK_TFLOPS, "TFLOP/s"
    if name == "rr_step":
        # eigh above, plus the triangular subspace products conj(M) (H_raw M^T) and C = Vt M
        # (three products of n^3/2 complex MACs: 12 n^3 flop)
        return "alu", (16.0 / 3.0 + 8.0 + 12.0) * ns ** 3, FP32_PEAK_TFLOPS, "TFLOP/s"
    if name == "cholesky":
        # two FP32 passes, each a complex Cholesky + triangular inverse (2 x n^3/6 complex
        # MACs = 8 n^3 / 3 flop), plus FP64 triangular products (n^3 complex MACs, 8 n^3 flop)
        return "alu", 2 * 8.0 * ns ** 3 / 3.0 + 8.0 * ns ** 3, FP32_PEAK_TFLOPS, "TFLOP/s"
    if name == "apply_h":
        # packed psi in + packed H psi out per state (the per-state algorithmic bytes of H psi)
        return "hbm", 2 * nG * c64 * ns + N ** 3 * 4, pk["hbm"], "GB/s"
    if name == "fft_lines":
        # one launch = one 1D-FFT pass over a batch of grids; bytes = read + write of the batch
        return "hbm", 2 * geo["batch"] * N ** 3 * c64, pk["hbm"], "GB/s"
    if name == "plane":
        # FFT flops (5 n log2 n per complex line of n) of the y- and x-lines each plane
        # transforms, inverse and forward: (2 x_r + 1) y-lines and N x-lines per direction
        import math
        lines = 2 * (geo["yrows"] + N)
        return "alu", ns * N * lines * 5.0 * N * math.log2(N), FP32_PEAK_TFLOPS, "TFLOP/s"
    if name in ("zinv", "zfwd"):
        return "hbm", ns * (ncols * N + 2 * nG) * c64, pk["hbm"], "GB/s"
    if name == "gram":
        # complex Psi^H Psi: 8 real flops per complex MAC
        return "tensor", 8.0 * ns * ns * nG, pk["bf16"], "TFLOP/s"
    if name == "rotate":
        return "tensor", 8.0 * ns * ns * nG, pk["bf16"], "TFLOP/s"
    return None


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch on the gs96 cell, from
# one ncu capture, with the hash of the kernel sources it was taken on: the bench reports the
# figure only while the sources are unchanged (otherwise traffic is null until re-captured).
NCU_TRAFFIC_GS96 = {"sources": "fd9ce299d9550286", "bytes": {"plane": 357760256 + 243112448}}
KERNEL_SOURCES = ("paper_2106_03872_gb300/csrc/fused.cu", "paper_2106_03872_gb300/csrc/fft_device.cuh")


def kernel_sources_hash():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(name):
    if NCU_TRAFFIC_GS96["sources"] != kernel_sources_hash():
        return None
    return NCU_TRAFFIC_GS96["bytes"].get(name)


# Stages that run as single-CTA kernels on the side stream, concurrently with the main stream's
# whole-GPU kernels: rated against one SM's share of the peak, not chosen as the dominant kernel
SIDE_STREAM = ("cholesky", "subspace", "eigh", "rr_step", "rot_prep", "ritz_values")


def _rate(name, ms, count, geo, pk, peak_scale=1.0):
    model = stage_model(name, geo, pk, None)
    per_launch_ms = ms / max(count, 1)
    out = {"kernel": name, "launch_ms": per_launch_ms, "launches": count}
    if model is None:
        out.update({"bound": "unknown", "achieved": None, "peak": None, "unit": None, "frac": None})
        return out
    bound, amount, peak, unit = model
    peak = peak * peak_scale
    if unit == "GB/s":
        achieved = amount / (per_launch_ms * 1e-3) / 1e9
    else:
        achieved = amount / (per_launch_ms * 1e-3) / 1e12
    out.update({"bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
                "peak_src": "derived: unit counts x max SM clock" if bound == "alu" else pk["src"]})
    return out


# FP32 CUDA-core rate measured by an FMA-chain probe over all 152 SMs (the derived 80.5 TFLOP/s
# assumes every lane issues an FMA every cycle at the maximum clock)
FP32_PROBE_TFLOPS = 69.5
HPSI_STAGES = ("plane", "zinv", "zfwd", "proj_gemm", "nl_values")


def hpsi_algorithmic_bytes(geo):
    """Algorithmic bytes of one H psi of the block: packed psi in and packed H psi out (complex64,
    2 |S| 8 B per state) plus the potential (N^3 4 B per call)."""
    return 2 * geo["nG"] * 8 * geo["nstates"] + geo["N"] ** 3 * 4


def hpsi_fft_flops(geo):
    """Nominal FFT flops of one H psi of the block: two full 3D FFTs per state at 5 n log2 n per
    length-n transform (5 N^3 log2(N^3) each), however much of the grid the pruned kernels skip."""
    import math
    N = geo["N"]
    return geo["nstates"] * 2 * 5.0 * N ** 3 * math.log2(N ** 3)


def tensor_gemms(entries, geo, pk, steps, nprojtot):
    """Tensor-core GEMM stages of one block iteration: their tensor work (split-BF16: three bf16
    products per real product for the overlaps, four for the rotations) over their device time,
    against the measured bf16 peak.  The stage timers cover every launch of the stage (the split-K
    reductions included), so the fraction is a lower bound of the MMA pipe's busy time."""
    n, K = geo["nstates"], geo["nG"]
    # algorithmic flops per launch: 8 real flops per complex MAC
    model = {"gram": (8.0 * n * n * K, 3, 2),            # S and H_raw: two launches per step
             "proj_gemm": (8.0 * nprojtot * n * K, 3, 1),  # projections onto the projector block
             "rotate": (8.0 * n * 2 * n * K, 4, 2)}        # psi and H psi rotated from [psi; H psi; H^2 psi]
    out = {}
    for name, (alg, split, per_step) in model.items():
        if name not in entries:
            continue
        ms = entries[name][0] / steps
        tens = alg * split * per_step
        out[name] = {"ms_per_step": ms, "launches_per_step": per_step, "flops_algorithmic_per_step": alg * per_step,
                     "split_products": split, "flops_tensor_per_step": tens,
                     "tflops_tensor": tens / (ms * 1e-3) / 1e12,
                     "frac_of_bf16_peak": tens / (ms * 1e-3) / 1e12 / pk["bf16"], "peak_src": pk["src"]}
    return out


def roofline(entries, geo, pk, steps):
    """The dominant kernel: the main-stream stage with the most device time.  A stage of the H psi
    pipeline is rated against HBM on the algorithmic bytes of the whole H psi it serves (one launch
    processes the block's states), with its share of the nominal FFT flops against the measured
    FP32 rate beside it; other stages by their own model.  Returns it, its name, and the
    side-stream single-SM stages rated against one SM's share of the peak."""
    leaf = {k: v for k, v in entries.items() if k != "apply_h" and k not in SIDE_STREAM}
    if not leaf:
        return None, None, []
    name = max(leaf, key=lambda k: leaf[k][0])
    ms, count = leaf[name]
    launch_s = ms / max(count, 1) * 1e-3
    if name in HPSI_STAGES:
        # the H application runs its kernels over batches of states (column buffers resident in
        # L2): rate the kernel's time per H psi call, its launches of all batches together
        calls = entries.get("apply_h", (0.0, count))[1]
        call_s = ms / max(calls, 1) * 1e-3
        nbytes = hpsi_algorithmic_bytes(geo)
        achieved = nbytes / call_s / 1e9
        # x and y passes of both 3D FFTs for the plane kernel (2/3 of the FFT flops), z passes
        # (1/3) for zinv + zfwd together (1/6 each); the projections carry none
        share = {"plane": 2.0 / 3.0, "zinv": 1.0 / 6.0, "zfwd": 1.0 / 6.0}.get(name, 0.0)
        flops = share * hpsi_fft_flops(geo)
        out = {"kernel": name, "launch_ms": launch_s * 1e3, "launches": count, "ms_per_hpsi": call_s * 1e3,
               "hpsi_calls": calls, "bound": "hbm",
               "achieved": achieved, "peak": pk["hbm"], "unit": "GB/s", "frac": achieved / pk["hbm"],
               "peak_src": pk["src"], "algorithmic_bytes_per_hpsi": nbytes,
               "basis": "algorithmic bytes of one H psi of the %d-state block (packed psi in, packed H psi "
                        "out, complex64, plus V) / this kernel's device time per H psi (its launches over "
                        "the L2-sized state batches together)" % geo["nstates"],
               "traffic": measured_traffic(name),
               "alu": {"flops_per_hpsi": flops, "achieved": flops / call_s / 1e12 if flops else None,
                       "peak": FP32_PROBE_TFLOPS, "unit": "TFLOP/s",
                       "frac": flops / call_s / 1e12 / FP32_PROBE_TFLOPS if flops else None,
                       "peak_src": "measured FP32 FMA probe",
                       "basis": "this kernel's share of the nominal FFT flops of H psi "
                                "(2 x 5 N^3 log2 N^3 per state)"}}
    else:
        out = _rate(name, ms, count, geo, pk)
        out["traffic"] = None
    side = [dict(_rate(k, entries[k][0], entries[k][1], geo, pk, 1.0 / 152), peak_note="one SM of 152")
            for k in SIDE_STREAM if k in entries and stage_model(k, geo, pk, None) is not None]
    return out, name, side


# ------------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------------
def main_gpu(args):
    import numpy as np
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    cpu = cpu_all = None
    if rank == 0 and not args.no_cpu:
        cpu = run_cpu_leg(args.cpu_steps, 1, CPU_SAMPLE_STATES)     # before any CUDA work
        cpu_all = run_cpu_leg_all(args.cpu_steps, 1, CPU_SAMPLE_STATES)

    torch.cuda.set_device(local)
    from paper_2106_03872_gb300 import inputs, ks
    pk = peaks()
    stream = torch.cuda.Stream()
    cell = inputs.cell(WORKLOAD)
    N, ns = cell["N"], cell["nstates"]
    nG = ks.count_gvectors(cell["L"], N, cell["ecut"])
    c0 = inputs.random_coeffs(cell["seed"], ns, nG)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def timed_steps(g, nsteps, warmup, fn, profile=False):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        if profile:
            g.profile(2)
            g.profile(1)
        launches0 = ks.kernel_launches()
        times = []
        for _ in range(nsteps):
            with torch.cuda.stream(stream):
                flush.zero_()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            fn()
            ev1.record(stream)
            ev1.synchronize()
            times.append(ev0.elapsed_time(ev1))
        torch.cuda.synchronize()
        launches = ks.kernel_launches() - launches0
        entries = g.profile_entries() if profile else {}
        if profile:
            g.profile(0)
        return times, launches, entries

    # ---- main arm: mixed precision block iteration
    g = ks.Grid(cell, prec="bf16x3")
    g.set_states(c0)
    g.orthonormalize()
    geo = dict(N=N, nG=g.nG, nstates=ns, batch=ns, ncols=0,
               yrows=2 * int(cell["ecut"] ** 0.5 * 2 ** 0.5 * cell["L"] / (2 * 3.141592653589793)) + 1)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    # K steps are timed as one call of K block iterations: one iteration touches psi, H psi
    # and H^2 psi (354 MB, more than the 126 MB L2), so consecutive steps find no operand in
    # L2; the L2 is flushed once before the timed call
    with Clocks(local) as clk:
        for _ in range(args.warmup):
            g.block_iteration(1, stream)
        torch.cuda.synchronize()
        g.profile(2)
        g.profile(1)
        launches0 = ks.kernel_launches()
        with torch.cuda.stream(stream):
            flush.zero_()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        g.block_iteration(args.steps, stream)
        ev1.record(stream)
        ev1.synchronize()
        times = [ev0.elapsed_time(ev1)]
        launches = ks.kernel_launches() - launches0
        entries = g.profile_entries()
        g.profile(0)
    total_ms = max_over_ranks(sum(times), dist, "cuda")
    ms_per_step = total_ms / args.steps
    value = replica_throughput(world, ns * N ** 3 * args.steps, total_ms)

    rl, rl_name, rl_side = roofline(entries, geo, pk, args.steps)
    tgemm = tensor_gemms(entries, geo, pk, args.steps, int(np.asarray(cell["pos"]).reshape(-1, 3).shape[0]) * cell["nproj"])

    # ---- H psi alone (device buffers)
    psi = torch.from_numpy(c0).to("cuda", torch.complex64)
    hpsi = torch.empty_like(psi)
    h_times, _, h_entries = timed_steps(g, args.steps, 2,
                                        lambda: g.apply_h(psi.data_ptr(), hpsi.data_ptr(), ns, stream), profile=True)
    h_ms = statistics.median(h_times)
    h_bytes = 2 * g.nG * 8 * ns + N ** 3 * 4
    hpsi_only = {"value": ns * N ** 3 / (h_ms * 1e-3), "unit": UNIT, "ms": h_ms,
                 "hbm_frac_algorithmic": h_bytes / (h_ms * 1e-3) / 1e9 / pk["hbm"],
                 "stages_ms_per_call": {k: v[0] / args.steps for k, v in h_entries.items() if v[0] > 0}}

    # ---- end to end through the public API with host buffers: every step copies the states in
    # from pinned host memory, runs one block iteration and copies the updated states (the
    # iteration's result) and the Ritz values back
    pinned = torch.empty((ns, g.nG), dtype=torch.complex128, pin_memory=True)
    pinned.numpy()[:] = c0
    pin_np = pinned.numpy()
    pinned_out = torch.empty((ns, g.nG), dtype=torch.complex128, pin_memory=True)
    out_np = pinned_out.numpy()
    e2e_times = []
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.set_states(pin_np)
        eig = g.block_iteration(1, stream)
        g.get_states(out=out_np)
        t1 = time.perf_counter()
        if i >= args.warmup:
            e2e_times.append(t1 - t0)
    e2e_ms = max_over_ranks(1e3 * statistics.mean(e2e_times), dist, "cuda")
    e2e = {"value": replica_throughput(world, ns * N ** 3, e2e_ms), "unit": UNIT, "ms_per_step": e2e_ms,
           "h2d_bytes_per_step": ns * g.nG * 16, "d2h_bytes_per_step": ns * g.nG * 16 + ns * 8,
           "note": "ks_set_states (pinned complex128 host -> device) + one block iteration + ks_get_states "
                   "(updated states, device -> pinned complex128 host) + Ritz values to host"}
    assert np.all(np.isfinite(eig)) and np.all(np.isfinite(out_np[0]))

    # ---- the 24^3 parity cell (8 states, FP64 and mixed): microseconds per H psi call through the
    # C ABI, device buffers (stream-ordered, timed on the device) and host buffers (wall clock)
    small = small_cell_timing(ks, inputs, stream, args.steps)

    # ---- the precision plan with FP64 Cholesky and FP64 Rayleigh-Ritz inside the timed iteration
    # (KS_OPT_FP64_SUBSPACE): same workload, the states and their GEMMs mixed
    fp64_sub = None
    if not args.no_fp64:
        gf = ks.Grid(cell, prec="bf16x3")
        gf.set_option(ks.KS_OPT_FP64_SUBSPACE, 1)
        gf.set_states(c0)
        gf.orthonormalize()
        tf_, _, ef_ = timed_steps(gf, 3, 1, lambda: gf.block_iteration(1, stream), profile=True)
        msf = statistics.mean(tf_)
        fp64_sub = {"workload": "gs96 block iteration, mixed states and GEMMs with the Cholesky factor, subspace "
                                "products and Rayleigh-Ritz eigensolver in FP64 (one-CTA FP64 kernels)",
                    "value": ns * N ** 3 / (msf * 1e-3), "ms_per_step": msf,
                    "stages_ms_per_step": {k: v[0] / len(tf_) for k, v in ef_.items() if v[0] > 0}}
        gf.close()

    # ---- all-FP64 GPU path, same workload
    fp64 = None
    if not args.no_fp64:
        g64 = ks.Grid(cell, prec="fp64")
        g64.set_states(c0)
        g64.orthonormalize()
        t64, _, e64 = timed_steps(g64, max(2, args.steps // 5), 1, lambda: g64.block_iteration(1, stream),
                                  profile=True)
        ms64 = statistics.mean(t64)
        fp64 = {"value": ns * N ** 3 / (ms64 * 1e-3), "ms_per_step": ms64, "speedup_mixed_vs_fp64": ms64 / ms_per_step,
                "stages_ms_per_step": {k: v[0] / len(t64) for k, v in e64.items() if v[0] > 0}}
        g64.close()

    # ---- real-time ETRS step of the 128^3 / 512-state cell (Hartree + Slater each step)
    td = None
    if not args.no_td:
        tcell = inputs.cell("td128")
        gt = ks.Grid(tcell, prec="bf16x3")
        ntg = gt.nG
        gt.set_states(inputs.random_coeffs(tcell["seed"], tcell["nstates"], ntg))
        gt.orthonormalize()
        gt.kick((0.01, 0.0, 0.0))
        tt, _, te = timed_steps(gt, 2, 1, lambda: gt.td_step(0.05, 1, "etrs", True, stream, dipoles=True),
                                profile=True)
        tms = statistics.mean(tt)
        td = {"workload": "td128: L=40, N=128, 512 states, 128 atoms, kick 0.01 bohr^-1 along x at t=0, then "
                          "ETRS + Taylor 4 with Hartree + Slater and the dipole recorded each step, dt=0.05",
              "steps_per_s": 1e3 / tms, "ms_per_step": tms,
              "stages_ms_per_step": {k: v[0] / len(tt) for k, v in te.items() if v[0] > 0}}
        gt.close()

    # ---- self-consistent field on the gs96 cell: 4 SCF iterations per call, each with
    # V[n_in], 2 block iterations, CholQR, the output density and Broyden mixing (the
    # paper's default)
    scf = None
    if not args.no_scf:
        gs = ks.Grid(cell, prec="bf16x3")
        gs.set_states(c0)
        SCF_IT, SCF_EIG = 4, 2
        ts, _, se = timed_steps(gs, 2, 1, lambda: gs.scf(SCF_IT, eig_iters=SCF_EIG, mix=0.3, stream=stream,
                                                         mixer="broyden", history=4), profile=True)
        sms = statistics.mean(ts)
        scf = {"workload": "gs96, %d SCF iterations per call, %d block iterations each, Broyden mixing 0.3 "
                           "with 4 history pairs (the call's initial CholQR and density included)" % (SCF_IT, SCF_EIG),
               "ms_per_scf_iteration": sms / SCF_IT, "ms_per_call": sms,
               "stages_ms_per_call": {k: v[0] / len(ts) for k, v in se.items() if v[0] > 0}}
        gs.close()

    # ---- Teter-preconditioned steepest descent on the gs96 cell (non-pipelined: CholQR, H psi,
    # Rayleigh-Ritz and the preconditioned update in order)
    teter = None
    forces = None
    if not args.no_scf:
        gp = ks.Grid(cell, prec="bf16x3")
        gp.set_states(c0)
        tp, _, pe = timed_steps(gp, 3, 1, lambda: gp.block_iteration(1, stream, precond="teter"), profile=True)
        tf, _, fe = timed_steps(gp, 2, 1, lambda: gp.forces(stream), profile=False)
        forces = {"workload": "gs96, forces on the 64 atoms from the 128 states (Eq. 11): 4 full-grid transforms "
                              "per state, real-space projections, separable local term",
                  "ms_per_call": statistics.mean(tf)}
        teter = {"workload": "gs96, one Teter-preconditioned block iteration per call",
                 "ms_per_iteration": statistics.mean(tp),
                 "stages_ms_per_iteration": {k: v[0] / len(tp) for k, v in pe.items() if v[0] > 0}}
        gp.close()

    # ---- Ehrenfest dynamics on the gs96 cell: per step the ETRS step, the ionic potential and
    # projectors rebuilt at the new positions, and the forces of the new states
    ehrenfest = None
    if not args.no_td:
        ge = ks.Grid(cell, prec="bf16x3")
        ge.set_states(c0)
        ge.orthonormalize()
        na = cell["pos"].shape[0]
        mass = np.full(na, 28.0855 * 1822.888)                          # silicon, electron masses
        vel = inputs.thermal_velocities(cell["seed"], mass)
        EH_STEPS = 2
        tE, _, eE = timed_steps(ge, 2, 1, lambda: ge.ehrenfest(0.05, EH_STEPS, mass, vel, stream=stream),
                                profile=True)
        ems = statistics.mean(tE)
        ehrenfest = {"workload": "gs96, 64 atoms of silicon mass with 300 K velocities, %d Ehrenfest steps per "
                                 "call (dt=0.05; each: ETRS step with Hartree + Slater, V_loc and projectors "
                                 "rebuilt at R(t+dt), forces of the new states), plus the call's initial "
                                 "forces" % EH_STEPS,
                     "ms_per_call": ems, "ms_per_step": ems / EH_STEPS,
                     "stages_ms_per_call": {k: v[0] / len(tE) for k, v in eE.items() if v[0] > 0}}
        ge.close()

    serve = None if args.no_serve else serve_bench(ks, inputs, args.serve_requests, args.serve_load_requests)

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c64", "data": "synthetic",
        "config": {"workload": "gs96: L=30 bohr, N=96, |S|=%d, 128 states, 64 atoms (perturbed fcc), 4 KB "
                               "projectors/atom, one SD block iteration per step (CholQR + H psi + Rayleigh-Ritz + "
                               "update), mixed precision" % g.nG,
                   "global_batch": ns * world, "grid": N, "parallelism": "replicas" if world > 1 else "single",
                   "l2": "flushed (256 MB device write) before the timed call of K steps; one step's working set "
                         "(psi, H psi, H^2 psi: 354 MB) exceeds the 126 MB L2"},
        "roofline": rl, "side_stream_roofline": rl_side, "tensor_gemms": tgemm,
        "cpu_baseline": cpu_baseline_obj(cpu, cpu_all) if cpu else None, "e2e": e2e,
        "gpu_launches": launches, "clocks": clk.summary(), "hpsi_only": hpsi_only, "fp64_gpu": fp64, "fp64_subspace": fp64_sub, "td": td,
        "small_cell": small, "autotune": ks.autotune_report(),
        "scf": scf, "teter": teter, "forces": forces, "ehrenfest": ehrenfest, "serve": serve,
        "stages_ms_per_step": {k: v[0] / args.steps for k, v in entries.items() if v[0] > 0},
    }
    print(json.dumps(line), flush=True)


def small_cell_timing(ks, inputs, stream, nsteps):
    import numpy as np
    import torch
    cell = inputs.cell("small")
    out = {"workload": "small: L=10, N=24, |S|=4,337, 8 states, 4 atoms, FP64 and mixed H psi"}
    for prec, cdt in (("fp64", torch.complex128), ("bf16x3", torch.complex64)):
        g = ks.Grid(cell, prec=prec)
        c = inputs.random_coeffs(cell["seed"], cell["nstates"], g.nG)
        psi = torch.from_numpy(c).to("cuda", cdt)
        h = torch.empty_like(psi)
        reps = 200
        for _ in range(10):
            g.apply_h(psi.data_ptr(), h.data_ptr(), cell["nstates"], stream)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(reps):
            g.apply_h(psi.data_ptr(), h.data_ptr(), cell["nstates"], stream)
        ev1.record(stream)
        ev1.synchronize()
        dev_us = 1e3 * ev0.elapsed_time(ev1) / reps
        t = []
        for _ in range(max(5, nsteps)):
            t0 = time.perf_counter()
            g.apply_h_host(c)
            t.append(time.perf_counter() - t0)
        out[prec] = {"us_per_call_device": dev_us, "us_per_call_host_buffers": 1e6 * statistics.median(t)}
        g.close()
    return out


def serve_bench(ks, inputs, nreq, nreq_load):
    """Continuous-batching server on the serving workload's shape (grids {32,48,64,96}^3 at
    h = 0.3125 bohr, 8-256 states, 4-64 atoms, half 10 block iterations and half 50 ETRS steps with
    Hartree + Slater): saturated throughput over nreq requests submitted at once, then Poisson
    arrivals at 50/80/95 % of that rate over the first nreq_load of them, with p50/p99 latency
    (submit to finish)."""
    import numpy as np

    reqs = inputs.serve_requests(BASE_SERVE_SEED, nreq)

    def run(rate, sub):
        srv = ks.Server(0, workers=SERVE_WORKERS)
        t0 = time.perf_counter()
        tickets = []
        arrival = 0.0
        rng = np.random.default_rng(BASE_SERVE_SEED + 1)
        for r in sub:
            if rate:
                arrival += rng.exponential(1.0 / rate)
                delay = t0 + arrival - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
            tickets.append(srv.submit(r, r["kind"], r["count"], r["dt"], prec="bf16x3"))
        lat = []
        for t in tickets:
            while True:
                st, res, _, l = srv.poll(t, 1000)
                if st == ks.KS_OK:
                    lat.append(l)
                    break
                if st not in (ks.KS_PENDING, ks.KS_ERR_TIMEOUT):
                    raise RuntimeError("serving request failed: %s" % ks.load().ks_last_error())
        span = time.perf_counter() - t0
        stats = srv.stats()
        srv.close()
        return span, np.array(lat), stats

    span, lat, stats = run(None, reqs)
    sat = nreq / span
    loads = []
    sub = reqs[:nreq_load]
    for frac in (0.5, 0.8, 0.95):
        sp, la, _ = run(frac * sat, sub)
        loads.append({"load": frac, "rate_req_per_s": frac * sat, "requests": len(sub),
                      "p50_s": float(np.percentile(la, 50)), "p99_s": float(np.percentile(la, 99)),
                      "throughput_req_per_s": len(sub) / sp})
    gp = sum(r["nstates"] * r["N"] ** 3 * r["count"] for r in reqs)
    return {"requests": nreq, "workers": SERVE_WORKERS, "saturated_req_per_s": sat,
            "saturated_state_gridpts_steps_per_s": gp / span, "saturated_s": span,
            "saturated_p50_s": float(np.percentile(lat, 50)), "saturated_p99_s": float(np.percentile(lat, 99)),
            "saturated_worker_stats": stats, "loads": loads,
            "workload": "seeded requests of the serving workload: N in {32,48,64,96} (L = 0.3125 N), 8-256 "
                        "states, 4-64 atoms at uniform positions, half 10 block iterations and half 50 ETRS "
                        "steps (dt 0.05, Hartree + Slater), mixed precision; %d requests at saturation, the "
                        "first %d at each Poisson load" % (nreq, nreq_load)}


def main_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    leg = cpu_leg(args.steps, args.warmup, CPU_SAMPLE_STATES)
    base = cpu_baseline_obj(leg)
    t = sum(leg["times"]) / len(leg["times"])
    line = {"impl": "reference", "metric": METRIC, "value": base["value"], "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "gs96 (bounded sample: %d of 128 states per step)" % CPU_SAMPLE_STATES},
            "cpu_baseline": base, "e2e": {"value": base["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                                          "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-leg", action="store_true")
    ap.add_argument("--cpu-td-leg", action="store_true",
                    help="time the oracle's td128 real-time step on a sample of states (one thread) and exit")
    ap.add_argument("--sample", type=int, default=CPU_SAMPLE_STATES)
    ap.add_argument("--cpu-steps", type=int, default=2)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-td", action="store_true")
    ap.add_argument("--no-scf", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=300)
    ap.add_argument("--serve-load-requests", type=int, default=120)
    args = ap.parse_args()
    if args.cpu_leg:
        print(json.dumps(cpu_leg(args.steps, args.warmup, args.sample)))
        return
    if args.cpu_td_leg:
        print(json.dumps(cpu_td_leg()))
        return
    if args.impl == "reference":
        main_reference(args)
        return
    main_gpu(args)


if __name__ == "__main__":
    main()
