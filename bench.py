"""Benchmark: SO(3) FFT forward + inverse transforms per second on the GB300.

One step = one forward transform (2-D FFTs + DWT) and one inverse transform
(iDWT + 2-D FFTs) of one band-limited function at bandwidth B, through the C
ABI.  Default workload: B = 256 in FP64 (512^3 complex128 grid, 2 GiB;
coefficients complex Gaussian scaled by 1/(l+1)).  Below B = 256 the inputs
rotate over enough distinct grids/coefficient vectors that one pass over them
exceeds the 129 MB L2; from B = 256 up one input alone exceeds it.

Printed JSON line (rank 0):
  value        device-timed fwd+inv pairs/s over the timed steps (CUDA events)
  e2e          the same through soft_forward_host / soft_inverse_host with
               pinned host buffers, host<->device copies inside the timing
  roofline     dominant kernel (the FP64 DWT or iDWT) against the FP64 pipe
  rel_l2       the timed outputs against the FP64 oracle: forward coefficients
               of sampled order pairs (all lengths), inverse values at sampled
               grid points, each computed one by one by the oracle; and the
               whole forward output against the input coefficients (the grids
               are their FP64 inverse in every mode), which within_bound uses
  modes        (default workload, one GPU) the same measurement for B = 128,
               256, 512 in each precision mode (fp64, fp64_tc, bf16x3, tf32):
               pairs/s, per-phase ms, FP64-pipe fraction, tensor TFLOP/s and
               rel-L2 against the oracle, on identical inputs per B
  cpu_baseline the FP64 CPU oracle on all host cores (OpenMP over order pairs
               and slices) at the workload's B, plus a single-thread figure;
               a full round trip when it fits the time budget, else a timed
               sample of every stride-th row of order pairs and slice,
               extrapolated (labelled)

Multi-GPU (torchrun): the transforms are independent, so every rank runs its
own replica of the workload (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (B, dtype, coefficient kind, description)
    "b16": (16, "fp64", "uniform", "FP64 SOFT forward+inverse, B=16, 32^3 complex128 grid, U(-1,1) coefficients"),
    "b64": (64, "fp64", "gauss_decay", "FP64 SOFT forward+inverse, B=64, 128^3 complex128 grid (32 MiB), "
                                       "complex Gaussian coefficients x 1/(l+1)"),
    "b128": (128, "fp64", "gauss_decay", "FP64 SOFT forward+inverse, B=128, 256^3 complex128 grid (256 MiB)"),
    "b256": (256, "fp64", "gauss_decay", "FP64 SOFT forward+inverse, B=256, 512^3 complex128 grid (2 GiB)"),
    "b512": (512, "fp64", "gauss_decay", "FP64 SOFT forward+inverse, B=512, 1024^3 complex128 grid (16 GiB)"),
}
for _B in (64, 128, 256, 512):
    for _m, _d in (("bf16x3", "split-BF16x3"), ("tf32", "TF32")):
        WORKLOADS[f"b{_B}_{_m}"] = (_B, _m, "gauss_decay",
                                    f"mixed SOFT forward+inverse, B={_B}, {_d} contraction on tcgen05 tensor cores, "
                                    f"FP64 Wigner-d recurrence, FP32 2-D FFTs; complex128 in/out")
    WORKLOADS[f"b{_B}_real"] = (_B, "fp64_real", "gauss_decay",
                                f"FP64 SOFT forward+inverse of a real function, B={_B}: soft_forward_real / "
                                f"soft_inverse_real on a real (2B)^3 float64 grid, one partner of each conjugate "
                                f"pair contracted")
    WORKLOADS[f"b{_B}_fp64tc_real"] = (_B, "fp64_tc_real", "gauss_decay",
                                       f"FP64-accurate SOFT forward+inverse of a real function, B={_B}: "
                                       f"soft_forward_real / soft_inverse_real on an FP64-TC plan (tensor-core "
                                       f"contraction of one partner per conjugate pair, double-float half-spectrum FFT)")
    WORKLOADS[f"b{_B}_clenshaw"] = (_B, "fp64_clenshaw", "gauss_decay",
                                    f"FP64 SOFT forward+inverse, B={_B}, inverse DWT by Clenshaw's algorithm "
                                    f"(backward summation over the degrees, the iDWT's last tile-shape variant)")
    WORKLOADS[f"b{_B}_fp64tc"] = (_B, "fp64_tc", "gauss_decay",
                                  f"FP64-accurate SOFT forward+inverse, B={_B}: FP64 Wigner-d recurrence, S and "
                                  f"2-D FFTs, contraction on tcgen05 tensor cores as exact base-128 BF16 digit "
                                  f"products (7 digits per operand)")
# Batches of same-B transforms through soft_batched_forward / soft_batched_inverse:
# mixed plans share one DWT launch per group of 8 (N = 16 x 8 tensor-core columns).
BATCHED = {}
for _B, _nb in ((64, 8), (128, 8), (256, 8), (512, 4)):
    for _m in ("bf16x3", "fp64"):
        _name = f"b{_B}_{_m}_x{_nb}"
        WORKLOADS[_name] = (_B, _m, "gauss_decay",
                            f"{_nb} {'mixed BF16x3' if _m == 'bf16x3' else 'FP64'} SOFT forward+inverse transforms "
                            f"at B={_B} per step through the batched, graph-captured API")
        BATCHED[_name] = [_B] * _nb
# FP64-TC batches: each entry's own kernels, captured in the batch's graph.
for _B, _nb in ((64, 8), (128, 8), (256, 4)):
    _name = f"b{_B}_fp64tc_x{_nb}"
    WORKLOADS[_name] = (_B, "fp64_tc", "gauss_decay",
                        f"{_nb} FP64-accurate (FP64-TC) SOFT forward+inverse transforms at B={_B} per step through "
                        f"the batched, graph-captured API (each transform's own DWT / iDWT launches in one graph)")
    BATCHED[_name] = [_B] * _nb
# Mixed bandwidths in one batch: the FP64 transforms share one persistent DWT
# and one persistent iDWT launch over all their (transform, cluster) items.
WORKLOADS["mix_fp64"] = (256, "fp64", "gauss_decay",
                         "8 FP64 SOFT forward+inverse transforms per step, B = 32, 64, 128, 256 (two each), through "
                         "the batched, graph-captured API: one persistent DWT and one persistent iDWT launch over "
                         "all (transform, cluster) items")
BATCHED["mix_fp64"] = [32, 64, 128, 256, 32, 64, 128, 256]
# Batched rotational matching: 64 correlation requests, B uniform over {8, 16, 32, 64, 128}.
CORR_WORKLOAD = ("corr64", "batched rotational matching: 64 correlation requests, B drawn uniformly from "
                 "{8,16,32,64,128}, SH coefficients complex Gaussian x 1/(l+1); per request: correlation "
                 "coefficients, FP64 inverse SOFT (one graph-captured persistent launch for all iDWTs), "
                 "arg-max over the (2B)^3 grid")
METRIC = "SOFT fwd+inv transforms/s"
UNIT = "fwd+inv pairs/s"
L2_BYTES = 129 * 2 ** 20

# FP64 pipe peak, derived: the GB300's nominal 1.25 TFLOP/s FP64 at the maximum
# SM clock of 2070 MHz over 152 SMs is 4 FP64 flops (2 DFMA) per SM per clock.
FP64_FLOPS_PER_SM_CLK = 4
N_SM = 152
SM_MAX_MHZ = 2070.0

# DRAM traffic per launch of the dominant kernels from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum), keyed by kernel and bandwidth,
# with the source file and the SHA-256 prefix of its code (comments and blank
# lines removed) that the capture was taken on; reported as null once that
# code has changed.
TRAFFIC = {
    ("dwt_forward_fp64_kernel", 64): (36_887_552 + 12_032, "dwt_fp64.cu", "1047c03e36d8df50"),
    ("dwt_forward_fp64_kernel", 256): (3_089_268_992 + 362_294_016, "dwt_fp64.cu", "eb315583bf94423f"),
    ("dwt_forward_tc_kernel", 128): (294_756_608 + 45_407_488, "dwt_fp64tc.cu", "c443e7c0222d361b"),
}


def kernel_source_sha(name: str = "dwt_fp64.cu") -> str:
    """SHA-256 prefix of a CUDA source's code: /* */ and // comments, trailing
    spaces and blank lines removed, so that comment edits keep a capture valid."""
    path = os.path.join(ROOT, "paper_1808_00896_gb300", "csrc", name)
    text = re.sub(r"/\*.*?\*/", "", open(path).read(), flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    code = "\n".join(line.rstrip() for line in text.splitlines() if line.strip())
    return hashlib.sha256(code.encode()).hexdigest()[:16]


def dwt_flops(B: int) -> dict:
    """Algorithmic FP64 flops of one DWT (or iDWT) launch at bandwidth B:
    contraction 8B per coefficient (2B real FMAs on re and im), plus the
    rescaled three-term recurrence, 2 FMAs = 4 flops per generated T entry;
    one T column block per symmetry cluster: sum over m = 0..B-1 of (m+1)
    clusters with B-m degrees and 2B samples."""
    nc = B * (4 * B * B - 1) // 3
    t_entries = 2 * B * sum((m + 1) * (B - m) for m in range(B))
    return {"contraction": 8 * B * nc, "recurrence": 4 * t_entries, "t_entries": t_entries}


class ClockSampler:
    """nvidia-smi samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_median": statistics.median(power) if power else None}


def busy_warmup(step, warmup: int, sync, min_seconds: float = 0.3) -> None:
    """Untimed steps: at least `warmup` of them, and more until `min_seconds`
    have passed, so the clock sampler is attached and the GPU is under load
    (not idling) when the timed region opens."""
    t0 = time.perf_counter()
    i = 0
    while i < warmup or time.perf_counter() - t0 < min_seconds:
        step(i)
        i += 1
        if i >= warmup:
            sync()


def max_over_ranks(x: float) -> float:
    """Max of a per-rank number over all ranks (identity without a process
    group).  CPU tensor on gloo, the current CUDA device otherwise."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = torch.device("cpu") if dist.get_backend() == "gloo" else torch.device("cuda", torch.cuda.current_device())
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


class OracleTimer:
    """Times the FP64 CPU oracle's forward+inverse round trip at bandwidth B on
    a given number of threads.  A full round trip at B >= 256 takes minutes on
    one core, so it can also take a timed SAMPLE: the oracle's strided runs
    process every stride-th row of order pairs and every stride-th beta slice
    plus the full run's fixed costs (the copies of the grid), and a run with a
    stride above 4B measures those fixed costs alone.  The full time is then
    extrapolated as fixed + stride x (sample - fixed)."""

    def __init__(self, B: int, coef, grid):
        import numpy as np

        import oracle
        self.oracle = oracle
        oracle.build()
        self.B = B
        self.coef = coef
        self.grid = grid
        self.gbuf = np.zeros_like(grid)
        self.cbuf = np.zeros_like(coef)

    def _round_trip(self, stride: int) -> float:
        t0 = time.perf_counter()
        if stride == 1:
            self.oracle.inverse(self.B, self.coef)
            self.oracle.forward(self.B, self.grid)
        else:
            self.oracle.inverse_strided(self.B, self.coef, stride, out=self.gbuf)
            self.oracle.forward_strided(self.B, self.grid, stride, out=self.cbuf)
        return time.perf_counter() - t0

    def fixed(self) -> float:
        return self._round_trip(1 << 30)

    def sampled(self, stride: int, fixed: float) -> float:
        """Extrapolated seconds of one full round trip from one strided run."""
        if stride <= 1:
            return self._round_trip(1)
        return fixed + stride * max(0.0, self._round_trip(stride) - fixed)

    def measure(self, threads: int, budget_s: float, allow_full: bool = True) -> dict:
        """Seconds per full round trip on `threads` threads within about
        budget_s of CPU time: a full run when the first sample's estimate
        fits, else the extrapolated sample at the smallest stride that fits."""
        prev = self.oracle.set_threads(threads)
        try:
            B = self.B
            rows = 2 * B - 1
            s0 = max(1, rows // 16)  # a first sample of 16 rows
            fixed = self.fixed()
            est = self.sampled(s0, fixed)
            if allow_full and est <= budget_s:
                t, stride, how = self._round_trip(1), 1, f"1 full B={B} round trip"
            else:
                stride = max(1, min(s0, math.ceil(est / max(1e-3, budget_s))))
                t = est if stride == s0 else self.sampled(stride, fixed)
                how = (f"B={B} round trip extrapolated from a timed sample of every {stride}-th row of order pairs "
                       f"and beta slice ({(rows + stride - 1) // stride} of {rows} rows): fixed costs "
                       f"{fixed:.2f} s + {stride} x the sampled per-row work")
            used = self.oracle.threads()
        finally:
            self.oracle.set_threads(prev)
        return {"seconds": t, "how": how, "threads": used, "stride": stride}


def cpu_baseline_oracle(B: int, kind: str, budget_s: float, seed: int) -> dict:
    """The FP64 oracle, as it stands, at bandwidth B: on all host cores
    (OpenMP) and on one thread, each as a full round trip when it fits the
    budget, else a timed sample extrapolated to the full round trip."""
    import oracle
    from paper_1808_00896_gb300 import synth
    oracle.build()
    coef = synth.coefficients(B, kind, seed=seed)
    grid = synth.random_grid(B, seed=seed + 1)  # the oracle's time does not depend on the values
    tm = OracleTimer(B, coef, grid)
    cores = host_cores()
    allc = tm.measure(cores, budget_s)
    one = tm.measure(1, budget_s / 2, allow_full=B <= 64)
    return {"value": 1.0 / allc["seconds"], "unit": UNIT, "cores": allc["threads"], "kind": "oracle",
            "sample": f"{allc['how']} on {allc['threads']} threads (OpenMP over order pairs and slices; "
                      f"nproc {cores})",
            "single_thread": {"value": 1.0 / one["seconds"], "unit": UNIT, "cores": 1, "sample": one["how"]},
            "omp_speedup": one["seconds"] / allc["seconds"]}


def workload_config(args, B: int, dtype: str, kind: str, world: int) -> dict:
    """The `config` dict of a workload, the same for both arms."""
    n = 2 * B
    grid_bytes = (8 if dtype in ("fp64_real", "fp64_tc_real") else 16) * n ** 3  # real grids: doubles
    coef_bytes = 16 * (B * (4 * B * B - 1) // 3)
    set_bytes = grid_bytes + coef_bytes
    # enough input sets that one pass over them is at least twice the L2
    R = max(1, math.ceil(2 * L2_BYTES / set_bytes))
    return {"workload": WORKLOADS[args.workload][3], "B": B, "mode": dtype, "coefficients": kind,
            "inputs_rotated": R, "tile_variants": None,
            "l2": f"{R} rotating input sets of {set_bytes / 2**20:.1f} MiB ({R * set_bytes / 2**20:.0f} MiB "
                  f"per pass, > 129 MB L2)" if R > 1 else "single input larger than L2",
            "parallelism": f"replicas x{world}"}


def run_reference(args) -> None:
    """--impl reference: the CPU oracle timed as it stands on this machine's host
    cores (OpenMP over order pairs and slices), on the same workload, metric,
    unit and config.  Each step is a bounded sample: the oracle's strided
    round trip over every stride-th row of order pairs and beta slice, with
    the stride picked so a step takes a few seconds, extrapolated to the full
    round trip as fixed + stride x (sample - fixed) (fixed costs measured once
    in the warm-up)."""
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    B, dtype, kind, desc = WORKLOADS[args.workload]
    import oracle
    from paper_1808_00896_gb300 import synth
    oracle.build()
    coef = synth.coefficients(B, kind, seed=synth.BASE_SEED + 7)
    grid = synth.random_grid(B, seed=synth.BASE_SEED + 8)
    tm = OracleTimer(B, coef, grid)
    cores = host_cores()
    oracle.set_threads(cores)
    fixed = tm.fixed()
    rows = 2 * B - 1
    s0 = max(1, rows // 16)
    est = tm.sampled(s0, fixed)  # warm-up and first estimate
    per_step = max(0.5, min(6.0, args.ref_seconds / max(1, args.steps + args.warmup)))
    stride = max(1, min(s0, math.ceil(est / per_step)))
    for _ in range(max(0, args.warmup - 1)):
        tm.sampled(stride, fixed)
    ts = [tm.sampled(stride, fixed) for _ in range(args.steps)]
    dt = sum(ts)
    value = args.steps / dt
    how = ("full round trips" if stride == 1 else
           f"round trips extrapolated from timed samples of every {stride}-th row of order pairs and beta slice "
           f"({(rows + stride - 1) // stride} of {rows} rows; fixed costs {fixed:.2f} s measured once)")
    sample = f"{args.steps} B={B} FP64 {how}, {oracle.threads()} threads (nproc {cores}), after {args.warmup} warm-up"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "executed_steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(args, B, dtype, kind, world),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_corr(args) -> None:
    """--workload corr64: batched correlations through soft_batched_correlate."""
    import numpy as np
    import torch

    from paper_1808_00896_gb300 import Plan, batched_correlate, capi, synth
    from paper_1808_00896_gb300 import build as build_mod

    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    build_mod.build()
    reqs = synth.correlation_requests(64, seed=synth.BASE_SEED + 4 + 1000 * rank)
    plans = [Plan(B, "fp64", device=dev) for B, _, _ in reqs]
    fs = [torch.from_numpy(f).to(dev) for _, f, _ in reqs]
    gs = [torch.from_numpy(g).to(dev) for _, _, g in reqs]
    grids = [p.empty_grid() for p in plans]
    bi = torch.empty(len(reqs), dtype=torch.int64, device=dev)
    bv = torch.empty(len(reqs), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        batched_correlate(plans, fs, gs, grids, bi, bv)
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(dev.index if world == 1 else local)
    if world > 1:
        torch.distributed.barrier()
    sampler.start()
    busy_warmup(lambda i: batched_correlate(plans, fs, gs, grids, bi, bv), 0, lambda: torch.cuda.synchronize(dev))
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n_launch0 = capi.soft_launch_count()
    ev0.record(stream)
    for _ in range(args.steps):
        batched_correlate(plans, fs, gs, grids, bi, bv)
    ev1.record(stream)
    gpu_launches = capi.soft_launch_count() - n_launch0
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    ms = max_over_ranks(ms)
    value = world * len(reqs) * 1000.0 / ms
    # e2e: SH coefficients host -> device, the batch, arg-max results device -> host.
    fh = [torch.from_numpy(f).pin_memory() for _, f, _ in reqs]
    gh = [torch.from_numpy(g).pin_memory() for _, _, g in reqs]
    bih = torch.empty(len(reqs), dtype=torch.int64, pin_memory=True)
    bvh = torch.empty(len(reqs), dtype=torch.float64, pin_memory=True)
    e2e_steps = max(3, min(args.steps, args.e2e_steps))
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        for a, b in zip(fs, fh):
            a.copy_(b, non_blocking=True)
        for a, b in zip(gs, gh):
            a.copy_(b, non_blocking=True)
        batched_correlate(plans, fs, gs, grids, bi, bv)
        bih.copy_(bi, non_blocking=True)
        bvh.copy_(bv, non_blocking=True)
        torch.cuda.synchronize(dev)
    e2e_dt = time.perf_counter() - t0
    h2d = sum(16 * B * B * 2 for B, _, _ in reqs)
    # Roofline: the batch's inverse DWT flops over the whole step (FFT, coefficient
    # build and arg-max included, so this understates the DWT kernel's own rate).
    algo = sum(dwt_flops(B)["contraction"] + dwt_flops(B)["recurrence"] for B, _, _ in reqs)
    peak_gflops = FP64_FLOPS_PER_SM_CLK * N_SM * SM_MAX_MHZ * 1e6 / 1e9
    achieved = algo / (ms * 1e-3) / 1e9
    if rank == 0:
        Bs = [B for B, _, _ in reqs]
        line = {
            "metric": "batched rotational correlations/s", "value": value, "unit": "correlations/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": CORR_WORKLOAD[1], "requests": len(reqs),
                       "bandwidth_counts": {str(b): Bs.count(b) for b in sorted(set(Bs))},
                       "parallelism": f"replicas x{world}", "l2": "per-step working set > 1 GB (> L2)"},
            "e2e": {"value": world * len(reqs) * e2e_steps / e2e_dt, "unit": "correlations/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 16 * len(reqs), "steps": e2e_steps},
            "gpu_launches": gpu_launches,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_gflops, "unit": "GFLOP/s",
                         "frac": achieved / peak_gflops, "traffic": None, "kernel": "idwt_fp64_persistent_kernel",
                         "note": "whole-step time (FFTs, coefficient build and arg-max included)"},
            "clocks": clocks, "cpu_baseline": None,
        }
        print(json.dumps(line), flush=True)
    for p in plans:
        p.close()


def run_batched(args) -> None:
    """Batched workloads: nb same-B transforms per step (forward + inverse)."""
    import torch

    from paper_1808_00896_gb300 import Plan, batched_forward, batched_inverse, capi, synth
    from paper_1808_00896_gb300 import build as build_mod

    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    build_mod.build()
    B, dtype, kind, desc = WORKLOADS[args.workload]
    Bs = BATCHED[args.workload]
    nb = len(Bs)
    plans = [Plan(b, dtype, device=dev) for b in Bs]
    coefs = [torch.from_numpy(synth.coefficients(b, kind, seed=synth.BASE_SEED + 100 * rank + i)).to(dev)
             for i, b in enumerate(Bs)]
    grids = batched_inverse(plans, coefs)
    coef_out = [p.empty_coef() for p in plans]
    grid_out = [p.empty_grid() for p in plans]
    stream = torch.cuda.current_stream(dev)

    def step():
        batched_forward(plans, grids, coef_out)
        batched_inverse(plans, coefs, grid_out)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(dev.index if world == 1 else local)
    if world > 1:
        torch.distributed.barrier()
    sampler.start()
    busy_warmup(lambda i: step(), 0, lambda: torch.cuda.synchronize(dev))
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n_launch0 = capi.soft_launch_count()
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    gpu_launches = capi.soft_launch_count() - n_launch0
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    ms = max_over_ranks(ms)
    value = world * nb * 1000.0 / ms
    # the same transforms one plan call at a time (no graph, no shared launch), for comparison
    def single():
        for p, g, c, go, co in zip(plans, grids, coefs, grid_out, coef_out):
            p.forward(g, out=co)
            p.inverse(c, out=go)
    for _ in range(2):
        single()
    torch.cuda.synchronize(dev)
    ev0.record(stream)
    for _ in range(args.steps):
        single()
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    ms_single = ev0.elapsed_time(ev1) / args.steps
    fl = dwt_flops(B)
    peak_gflops = FP64_FLOPS_PER_SM_CLK * N_SM * SM_MAX_MHZ * 1e6 / 1e9
    if dtype == "fp64":
        algo = 2 * sum(dwt_flops(b)["contraction"] + dwt_flops(b)["recurrence"] for b in Bs)
        note = ("whole-step time (FFTs included): the FP64 contraction + recurrence of the batch's DWTs and iDWTs "
                "(one persistent launch per direction)")
    elif dtype == "fp64_tc":
        algo = 2 * nb * fl["recurrence"]  # each transform's own recurrence, DWT and iDWT
        note = ("whole-step time (FFTs included): the FP64 recurrence of every transform's DWT and iDWT "
                "(per-transform launches inside the batch's graph)")
    else:
        algo = 2 * fl["recurrence"]  # one shared recurrence per batched DWT launch, 2 launches per step
        note = ("whole-step time (FFTs included): the FP64 recurrence of the 2 batched (i)DWT launches, "
                "shared by the nb transforms")
    kernel = {"fp64": "dwt_forward_fp64_kernel", "fp64_tc": "dwt_forward_tc_kernel"}.get(dtype, "dwt_forward_mixed_kernel")
    roofline = {"bound": "alu", "achieved": algo / (ms * 1e-3) / 1e9, "peak": peak_gflops, "unit": "GFLOP/s",
                "frac": algo / (ms * 1e-3) / 1e9 / peak_gflops, "traffic": None, "kernel": kernel, "note": note}
    if dtype != "fp64":
        # tensor-core products per real multiply-add: 3 (BF16x3), 28 (FP64-TC digit pairs)
        roofline["tensor_tflops_achieved"] = 2 * (28 if dtype == "fp64_tc" else 3) * nb * fl["contraction"] / (ms * 1e-3) / 1e12
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if dtype == "fp64" else dtype, "data": "synthetic",
            "config": {"workload": desc, "B": B if len(set(Bs)) == 1 else Bs, "mode": dtype, "batch": nb,
                       "coefficients": kind, "parallelism": f"replicas x{world}", "l2": "per-step working set > L2"},
            "e2e": None, "gpu_launches": gpu_launches, "roofline": roofline, "clocks": clocks, "cpu_baseline": None,
            "per_plan_calls": {"ms_per_step": ms_single, "value": world * nb * 1000.0 / ms_single,
                               "speedup_of_batch": ms_single / ms},
        }
        print(json.dumps(line), flush=True)
    for p in plans:
        p.close()


MODES = ("fp64", "fp64_tc", "bf16x3", "tf32")
MODE_BS = (128, 256, 512)
# stated rel-L2 bounds against the FP64 oracle, per mode
MODE_BOUND = {"fp64": 1e-10, "fp64_tc": 1e-10, "bf16x3": 5e-5, "tf32": 2e-3}
# tensor-core products per real multiply-add of the contraction: 3 split-BF16
# pairs, 1 TF32, or the 28 digit pairs (levels 0..6) of the FP64-accurate mode
TENSOR_MULT = {"bf16x3": 3, "tf32": 1, "fp64_tc": 28}
PEAK_FP64_GFLOPS = FP64_FLOPS_PER_SM_CLK * N_SM * SM_MAX_MHZ * 1e6 / 1e9
PEAK_SOURCE = "derived: nominal FP64 1.25 TFLOP/s = 4 flop/clk/SM x 152 SM x 2070 MHz"


def sample_pairs(B: int, seed: int, count: int = 16) -> list:
    """Order pairs whose runs span every length: the extreme cases, then
    random pairs on evenly spaced shells max(|m|,|m'|) = l0 <= B - 1."""
    import numpy as np
    rng = np.random.default_rng(seed)
    pairs = [(0, 0), (B - 1, B - 1), (1 - B, B - 1), (B // 2, -(B // 3))][:max(1, min(count, (2 * B - 1) ** 2))]
    want = min(count, (2 * B - 1) ** 2)
    k = 0
    while len(pairs) < want:
        l0 = min(B - 1, int(round((k % max(1, count - 4)) * (B - 1) / max(1, count - 5))))
        k += 1
        other = int(rng.integers(-l0, l0 + 1)) if l0 > 0 else 0
        sgn = 1 if rng.integers(0, 2) else -1
        pr = (sgn * l0, other) if rng.integers(0, 2) else (other, sgn * l0)
        if pr not in pairs:
            pairs.append(pr)
    return pairs


def sample_points(B: int, seed: int, count: int = 16) -> list:
    import numpy as np
    rng = np.random.default_rng(seed)
    n = 2 * B
    pts = [(0, 0, 0), (n - 1, n - 1, n - 1), (1, B, n - 2)]
    while len(pts) < count:
        pts.append(tuple(int(v) for v in rng.integers(0, n, size=3)))
    return pts  # (i, j, k)


class OracleRef:
    """The FP64 oracle's values for one bandwidth's inputs at sampled order
    pairs (forward coefficients, whole runs) and sampled grid points (inverse),
    each computed one by one; compares device outputs against them."""

    def __init__(self, B: int, grid_host, coef_host, seed: int, threads: int, real: bool = False):
        import numpy as np

        import oracle
        oracle.build()
        self.B = B
        self.pairs = sample_pairs(B, seed)
        self.pts = sample_points(B, seed + 1)
        prev = oracle.set_threads(threads)
        try:
            self.fwd = np.concatenate(oracle.forward_pairs(B, grid_host, self.pairs))
            self.inv = oracle.inverse_points(B, coef_host, self.pts)
        finally:
            oracle.set_threads(prev)
        if real:
            self.inv = self.inv.real
        from paper_1808_00896_gb300 import capi
        idx = []
        for m, mp in self.pairs:
            l0 = max(abs(m), abs(mp))
            o = capi.soft_coef_index(B, l0, m, mp)
            idx.extend(range(o, o + B - l0))
        n = 2 * B
        self.coef_idx = np.array(idx, dtype=np.int64)
        self.grid_idx = np.array([(j * n + i) * n + k for (i, j, k) in self.pts], dtype=np.int64)

    def errors(self, coef_dev, grid_dev) -> dict:
        import torch

        from paper_1808_00896_gb300 import synth
        ci = torch.from_numpy(self.coef_idx).to(coef_dev.device)
        gi = torch.from_numpy(self.grid_idx).to(grid_dev.device)
        f = coef_dev.reshape(-1)[ci].cpu().numpy()
        g = grid_dev.reshape(-1)[gi].cpu().numpy()
        return {"forward": synth.rel_l2(f, self.fwd), "inverse": synth.rel_l2(g, self.inv),
                "sample": f"{len(self.pairs)} order pairs ({len(self.coef_idx)} coefficients, every run length "
                          f"band) and {len(self.pts)} grid points vs the oracle's one-by-one forms"}


def roofline_numbers(B: int, dtype: str, phase_ms, phase_cnt) -> dict:
    """Dominant (i)DWT kernel's algorithmic FP64 rate from the library's events:
    contraction + recurrence for FP64 plans, half the contraction on real
    grids, the FP64 recurrence alone for the tensor-core modes (whose
    contraction runs on tcgen05; its TFLOP/s is reported beside)."""
    fl = dwt_flops(B)
    real = dtype == "fp64_real"  # FP64 real grids: half the contraction on the FP64 pipe
    fwd_ms = phase_ms[1] / max(1, phase_cnt[1])
    inv_ms = phase_ms[2] / max(1, phase_cnt[2])
    kname = {"fp64": "fp64", "fp64_real": "fp64", "fp64_clenshaw": "fp64", "fp64_tc": "tc",
             "fp64_tc_real": "tc"}.get(dtype, "mixed")
    inv_name = "idwt_clenshaw_fp64_kernel" if dtype == "fp64_clenshaw" else f"dwt_inverse_{kname}_kernel"
    dom, dom_ms = (f"dwt_forward_{kname}_kernel", fwd_ms) if phase_ms[1] >= phase_ms[2] else (inv_name, inv_ms)
    algo = fl["contraction"] + fl["recurrence"] if dtype in ("fp64", "fp64_clenshaw") else \
        fl["contraction"] / 2 + fl["recurrence"] if real else fl["recurrence"]
    achieved = algo / (dom_ms * 1e-3) / 1e9
    out = {"kernel": dom, "dom_ms": dom_ms, "algo": algo, "achieved": achieved, "frac": achieved / PEAK_FP64_GFLOPS,
           "phase_ms_per_launch": {"fft_forward": phase_ms[0] / max(1, phase_cnt[0]), "dwt_forward": fwd_ms,
                                   "dwt_inverse": inv_ms, "fft_inverse": phase_ms[3] / max(1, phase_cnt[3])}}
    if dtype in TENSOR_MULT or dtype == "fp64_tc_real":
        half = 0.5 if dtype == "fp64_tc_real" else 1.0  # one partner of each conjugate pair
        mult = TENSOR_MULT[dtype.replace("_real", "")]
        out["tensor_tflops"] = half * mult * fl["contraction"] / (dom_ms * 1e-3) / 1e12
    return out


def measure_mode(B: int, mode: str, grid_dev, coef_dev, ref: OracleRef, steps_max: int, warmup: int, dev,
                 target_s: float = 1.5) -> dict:
    """One (B, mode) record: forward(grid) + inverse(coef) pairs/s with CUDA
    events over K steps (K picked for about target_s of timed work, at least
    2), the library's per-phase events, and the timed outputs' rel-L2 against
    the oracle."""
    import torch

    from paper_1808_00896_gb300 import Plan, capi
    plan = Plan(B, mode, device=dev)
    try:
        coef_out = plan.empty_coef()
        grid_out = plan.empty_grid()
        stream = torch.cuda.current_stream(dev)

        def step():
            plan.forward(grid_dev, out=coef_out)
            plan.inverse(coef_dev, out=grid_out)

        t0 = time.perf_counter()
        for _ in range(warmup):
            step()
        plan.sync()
        tw = (time.perf_counter() - t0) / max(1, warmup)
        K = int(max(2, min(steps_max, math.ceil(target_s / max(tw, 1e-6)))))
        capi.soft_plan_read_timing(plan.handle)
        capi.soft_plan_enable_timing(plan.handle, True)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(K):
            step()
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        plan.sync()
        ms = ev0.elapsed_time(ev1) / K
        phase_ms, phase_cnt = capi.soft_plan_read_timing(plan.handle)
        capi.soft_plan_enable_timing(plan.handle, False)
        rf = roofline_numbers(B, mode, phase_ms, phase_cnt)
        err = ref.errors(coef_out, grid_out)
        full = float(torch.linalg.vector_norm(coef_out - coef_dev) / torch.linalg.vector_norm(coef_dev))
    finally:
        plan.close()
    rec = {"B": B, "mode": mode, "pairs_per_s": 1000.0 / ms, "ms_per_pair": ms, "steps": K,
           "phase_ms": {k: round(v, 4) for k, v in rf["phase_ms_per_launch"].items()},
           "kernel": rf["kernel"], "fp64_gflops": rf["achieved"], "frac": rf["frac"],
           "rel_l2_forward": err["forward"], "rel_l2_inverse": err["inverse"],
           "rel_l2_forward_vs_input_coef": full, "bound": MODE_BOUND[mode],
           # the stated bounds are over all coefficients (or grid values): the full
           # forward output against the input coefficients, which the oracle's
           # forward of the band-limited grid reproduces to ~1e-13 (the fp64 rows'
           # sampled error), and the sampled grid points, which weigh every region alike;
           # the sampled runs weigh the short high-order runs as much as the long ones
           "within_bound": bool(full <= MODE_BOUND[mode] and err["inverse"] <= MODE_BOUND[mode])}
    if "tensor_tflops" in rf:
        rec["tensor_tflops"] = rf["tensor_tflops"]
    return rec


def run_modes(Bs, args, dev) -> dict:
    """The per-(B, mode) table: for each B one band-limited input (complex
    Gaussian coefficients x 1/(l+1), grid = the FP64 GPU inverse of them),
    the oracle's sampled values, then every mode on the same inputs."""
    import torch

    from paper_1808_00896_gb300 import Plan, synth
    recs = []
    cores = host_cores()
    t_start = time.perf_counter()
    for B in Bs:
        seed = synth.BASE_SEED + 7 + B
        coef_h = synth.coefficients(B, "gauss_decay", seed=seed)
        coef_dev = torch.from_numpy(coef_h).to(dev)
        with Plan(B, "fp64", device=dev) as p:
            grid_dev = p.inverse(coef_dev)
            p.sync()
        grid_h = grid_dev.cpu().numpy()
        t0 = time.perf_counter()
        ref = OracleRef(B, grid_h, coef_h, seed, cores)
        t_oracle = time.perf_counter() - t0
        del grid_h
        per_b = []
        for mode in MODES:
            per_b.append(measure_mode(B, mode, grid_dev, coef_dev, ref, args.steps, args.warmup, dev))
            per_b[-1]["oracle_ref_s"] = round(t_oracle, 2)
        base = next(r["pairs_per_s"] for r in per_b if r["mode"] == "fp64")
        for r in per_b:
            r["speedup_vs_fp64"] = r["pairs_per_s"] / base
        recs.extend(per_b)
        del grid_dev, coef_dev
        torch.cuda.empty_cache()
    return {"records": recs, "inputs": "per B: coefficients complex Gaussian x 1/(l+1) (seed BASE_SEED+7+B), grid = "
                                      "FP64 GPU inverse of them; identical for every mode",
            "rel_l2": "timed outputs vs the FP64 oracle: whole runs of 16 sampled order pairs (forward) and 16 grid "
                      "points (inverse), the oracle's one-by-one forms on all host cores",
            "frac": "dominant (i)DWT kernel's algorithmic FP64 flops / duration vs the derived FP64 peak "
                    "(fp64: contraction + recurrence; tensor-core modes: the FP64 recurrence, tensor TFLOP/s beside)",
            "seconds": round(time.perf_counter() - t_start, 1)}


def run_ours(args) -> None:
    import numpy as np
    import torch

    from paper_1808_00896_gb300 import Plan, capi, synth
    from paper_1808_00896_gb300 import build as build_mod

    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    build_mod.build()

    B, dtype, kind, desc = WORKLOADS[args.workload]
    n = 2 * B
    grid_bytes = 16 * n ** 3
    coef_bytes = 16 * synth.num_coeffs(B)
    config = workload_config(args, B, dtype, kind, world)
    R = config["inputs_rotated"]

    real = dtype in ("fp64_real", "fp64_tc_real")  # real grids: soft_forward_real / soft_inverse_real
    plan = Plan(B, {"fp64_real": "fp64", "fp64_clenshaw": "fp64", "fp64_tc_real": "fp64_tc"}.get(dtype, dtype),
                device=dev)
    tuned = plan.tune() if args.tune else None
    if dtype == "fp64_clenshaw":
        plan.set_variant(1, plan.num_variants(1) - 1)  # the Clenshaw iDWT
    if tuned is not None:
        config["tile_variants"] = {"dwt": tuned["dwt"], "idwt": tuned["idwt"]}
    coefs = [torch.from_numpy(synth.coefficients(B, kind, seed=synth.BASE_SEED + 100 * rank + r)).to(dev)
             for r in range(R)]
    # the grids are the FP64 inverse of the coefficients in every mode: band
    # limited to them to ~1e-13, so the forward's whole output can be checked
    # against the coefficients as well as the sampled runs against the oracle
    gen = plan if dtype in ("fp64", "fp64_real", "fp64_clenshaw") else Plan(B, "fp64", device=dev)
    grids = [gen.inverse(c) for c in coefs]
    if gen is not plan:
        gen.close()
    if real:
        # a real grid per input set, and the coefficients of that real function
        grids = [g.real.contiguous() for g in grids]
        coefs = [plan.forward_real(g) for g in grids]
    coef_out = plan.empty_coef()
    grid_out = torch.empty((n, n, n), dtype=torch.float64, device=dev) if real else plan.empty_grid()
    stream = torch.cuda.current_stream(dev)

    def step(r):
        if real:
            plan.forward_real(grids[r], out=coef_out)
            plan.inverse_real(coefs[r], out=grid_out)
        else:
            plan.forward(grids[r], out=coef_out)
            plan.inverse(coefs[r], out=grid_out)

    for w in range(args.warmup):
        step(w % R)
    plan.sync()
    capi.soft_plan_read_timing(plan.handle)  # discard
    capi.soft_plan_enable_timing(plan.handle, True)

    sampler = ClockSampler(dev.index if world == 1 else local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    sampler.start()
    capi.soft_plan_enable_timing(plan.handle, False)
    busy_warmup(lambda i: step(i % R), 0, lambda: torch.cuda.synchronize(dev))
    capi.soft_plan_enable_timing(plan.handle, True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n_launch0 = capi.soft_launch_count()
    ev0.record(stream)
    for s_ in range(args.steps):
        step(s_ % R)
    ev1.record(stream)
    gpu_launches = capi.soft_launch_count() - n_launch0
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    ms_total = ev0.elapsed_time(ev1)
    ms_total = max_over_ranks(ms_total)
    plan.sync()
    phase_ms, phase_cnt = capi.soft_plan_read_timing(plan.handle)
    capi.soft_plan_enable_timing(plan.handle, False)
    last = (args.steps - 1) % R  # the input set of the last timed step: its outputs are checked below

    ms_per_step = ms_total / args.steps
    value = world * 1000.0 / ms_per_step

    # e2e with pinned host memory: through the host-buffer entry points, or
    # (real grids) explicit copies around the device calls, on one stream.
    e2e_steps = max(3, min(args.steps, int(args.e2e_steps)))
    g_host = torch.empty((n, n, n), dtype=grids[0].dtype, pin_memory=True)
    g_host.copy_(grids[0].cpu())
    c_host = torch.empty(synth.num_coeffs(B), dtype=torch.complex128, pin_memory=True)
    c_host.copy_(coefs[0].cpu())
    c_res = torch.empty_like(c_host, pin_memory=True)
    g_res = torch.empty_like(g_host, pin_memory=True)
    gh, ch, cr, gr = g_host.numpy(), c_host.numpy(), c_res.numpy(), g_res.numpy()
    g_dev, c_dev = torch.empty_like(grids[0]), plan.empty_coef()

    # rel-L2 of the timed outputs against the oracle (outside every timed region)
    rel = None
    if rank == 0:
        ref = OracleRef(B, np.ascontiguousarray(grids[last].cpu().numpy()).astype(np.complex128),
                        coefs[last].cpu().numpy(), synth.BASE_SEED + 11 + B, host_cores(), real=real)
        rel = ref.errors(coef_out, grid_out)
        rel["bound"] = MODE_BOUND.get("fp64" if dtype in ("fp64_real", "fp64_clenshaw", "fp64_tc_real") else dtype)
        fwd_err = rel["forward"]
        if not real:
            # the bound is over all coefficients: the whole forward output against
            # the input coefficients (the sampled runs weigh the short high-order
            # runs, whose small coefficients carry the FP32 FFT's absolute error,
            # as much as the long ones)
            fwd_err = float(torch.linalg.vector_norm(coef_out - coefs[last]) / torch.linalg.vector_norm(coefs[last]))
            rel["forward_vs_input_coef"] = fwd_err
        rel["within_bound"] = bool(fwd_err <= rel["bound"] and rel["inverse"] <= rel["bound"])

    def e2e_step():
        if real:
            g_dev.copy_(g_host, non_blocking=True)
            plan.forward_real(g_dev, out=coef_out)
            c_res.copy_(coef_out, non_blocking=True)
            c_dev.copy_(c_host, non_blocking=True)
            plan.inverse_real(c_dev, out=grid_out)
            g_res.copy_(grid_out, non_blocking=True)
            torch.cuda.synchronize(dev)
        else:
            plan.forward_host(gh, cr)
            plan.inverse_host(ch, gr)

    e2e_step()
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    e2e_dt = time.perf_counter() - t0
    e2e_dt = max_over_ranks(e2e_dt)
    gb = grid_bytes // 2 if real else grid_bytes
    e2e = {"value": world * e2e_steps / e2e_dt, "unit": UNIT,
           "h2d_bytes_per_step": gb + coef_bytes, "d2h_bytes_per_step": coef_bytes + gb,
           "steps": e2e_steps}

    # Roofline of the dominant kernel, from the library's CUDA events.
    rf = roofline_numbers(B, dtype, phase_ms, phase_cnt)
    tr = None if real else TRAFFIC.get((rf["kernel"], B))
    traffic = tr[0] if (tr and tr[2] == kernel_source_sha(tr[1])) else None
    roofline = {"bound": "alu", "achieved": rf["achieved"], "peak": PEAK_FP64_GFLOPS, "unit": "GFLOP/s",
                "frac": rf["frac"], "traffic": traffic, "kernel": rf["kernel"], "peak_source": PEAK_SOURCE,
                "algorithmic_flops_per_launch": rf["algo"], "phase_ms_per_launch": rf["phase_ms_per_launch"]}
    if "tensor_tflops" in rf:
        roofline["tensor_tflops_achieved"] = rf["tensor_tflops"]
        roofline["note"] = ("tensor-core contraction: frac is the FP64 Wigner-d recurrence (2 FMA per T entry) "
                            "against the FP64 pipe; tensor_tflops_achieved counts the contraction's tensor-core flops")
    plan.close()
    del grids, coefs, g_dev, c_dev, coef_out, grid_out
    torch.cuda.empty_cache()

    modes = None
    want_modes = args.modes != "off" and world == 1 and (args.modes != "auto" or args.workload == "b256")
    if want_modes:
        Bs = MODE_BS if args.modes == "auto" else tuple(int(x) for x in args.modes.split(","))
        modes = run_modes(Bs, args, dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_oracle(B, kind, args.cpu_seconds, synth.BASE_SEED + 7)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f64" if dtype in ("fp64", "fp64_real", "fp64_clenshaw") else dtype.replace("_real", ""),
            "data": "synthetic", "config": config, "e2e": e2e, "gpu_launches": gpu_launches, "roofline": roofline, "clocks": clocks,
            "rel_l2": rel, "cpu_baseline": cpu,
        }
        if modes is not None:
            line["modes"] = modes
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + [CORR_WORKLOAD[0]], default="b256")
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--cpu-seconds", type=float, default=30.0,
                    help="budget of the all-core oracle round trip (a full run when it fits, else a sample)")
    ap.add_argument("--ref-seconds", type=float, default=120.0)
    ap.add_argument("--modes", default="auto",
                    help="per-mode table: 'auto' (default workload on one GPU), 'off', or B list like '128,256'")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tune", action="store_true", help="autotune the DWT tile shapes before timing")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        ap.error("--warmup must be >= 3")
    if args.workload == CORR_WORKLOAD[0]:
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the batched correlation workload has no CPU "
                              "reference arm; the oracle checks it in tests/test_gpu_batched.py"}))
            return
        args.steps = args.steps or 20
        run_corr(args)
        return
    if args.workload in BATCHED:
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "batched workloads have no CPU reference arm"}))
            return
        args.steps = args.steps or {64: 200, 128: 40, 256: 6, 512: 2}[WORKLOADS[args.workload][0]]
        if len(set(BATCHED[args.workload])) > 1:
            args.steps = min(args.steps, 10)
        run_batched(args)
        return
    if args.steps is None:
        B = WORKLOADS[args.workload][0]
        args.steps = {"ours": {16: 2000, 64: 400, 128: 60, 256: 10, 512: 3},
                      "reference": {16: 50, 64: 20, 128: 4, 256: 1, 512: 1}}[args.impl][B]
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
