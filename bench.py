#!/usr/bin/env python
"""Benchmark of the voxel-gravity forward model on one GB300 (or N replicas).

Default workload: 464^3 = 99,897,344 voxels of 100 m (FP32 densities), a
layered 2600/2700/2900 kg/m^3 background with three seeded +-400 kg/m^3
ellipsoids, midpoint rule, 1024^2 surface stations -- the largest workload of
the paper's scale (about 1e8 voxels).  A timed step is one whole pass of the
path on resident inputs: the plan build (observer Morton keys, sort, box
tables, lists) and the forward solve (sources, upward sweep, M2L, downward
sweep, evaluation, near field, near+far combine), then the plan's release.
The mixed-precision FMM runs at a degree whose error against the FP64 oracle
stays below 1e-6 (relative L2 on a seeded observer sample); the plain FP64 FMM
and lower degrees are timed beside it on the same GPU.

Metric: effective interactions/s = N_sources * M_observers / step time, and
ms/solve of the forward with the plan built.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                  "sm_max_mhz": 2070.0}
N_SM = 152
FP32_LANES_PER_SM = 128          # FP32 FMA lanes per SM per clock
FP64_TFLOPS_NOMINAL = 1.25       # GB300 FP64 (vector and tensor) rate
FLOPS_PER_PAIR = 20.0            # the paper's count: 5 add, 7 mul, 1 sqrt ~ 20 mul-equivalents
F16_PER_BF16 = 1.0               # nominal dense FP16 / BF16 tensor rates
SFU_RSQRT_PER_SM = 16            # reciprocal square roots per SM per clock
# Throughput probes on a GB300 of this machine (FMA chains and MUFU rsqrt chains,
# 152 x 8 blocks of 256 threads, CUDA events): the denominators of the
# near field's secondary fractions.
FP32_TFLOPS_PROBE = 69.6
MUFU_RSQRT_PROBE = 4.63e12


# DRAM traffic per launch of the dominant kernel, from one ncu capture (the
# ncu summaries under profiles/), with the SHA-1 of the kernel's source files
# at capture time: once a source changes the figure no longer describes the
# kernel and the bench reports null.  The 464^3 figures are captures of
# the same recipe at 320^3 (the full size holds too much device memory for a
# multi-pass capture) scaled by the work units of a launch: near pairs for
# the evaluation (its near-field and far-field kernels together),
# interaction-list box pairs for the M2L.
NCU_TRAFFIC = {
    # evaluation: near-field and far-field kernels of one forward, scaled by the pairs
    ("eval", "layered_scale_464^3", 10): (round((7902720 + 0 + 23410176 + 0) * 596922624 / 280629504),
                                          ("paper_1107_5951_gb300/csrc/gf_fmm.cu",
                                           "paper_1107_5951_gb300/csrc/gf_simd.cuh",
                                           "paper_1107_5951_gb300/csrc/fmm_math.cuh"),
                                          "e6e19973d3feff22bec7f445f4c523b35d9d346b"),
    ("m2l", "layered_scale_464^3", 10): (round((19061248 + 0) * 1125279 / 510295),
                                         ("paper_1107_5951_gb300/csrc/gf_m2l.cu",),
                                         "06e97124d0ebb1d513f65faa28dd3a3ea34f260c"),
}


def sources_sha1(files):
    """SHA-1 of the concatenated sources a kernel is compiled from."""
    import hashlib
    h = hashlib.sha1()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def ncu_traffic(stage, workload, p, precision, m2l):
    key = (stage, workload, p)
    if precision != "mixed" or m2l != "auto" or key not in NCU_TRAFFIC:
        return None
    nbytes, srcs, sha = NCU_TRAFFIC[key]
    try:
        if sources_sha1(srcs) != sha:
            return None
    except OSError:
        return None
    return nbytes


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        d["_source"] = "measured"
        return d
    d = dict(PEAKS_FALLBACK)
    d["_source"] = "fallback"
    return d


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gf", "reference"], default="gf")
    ap.add_argument("--side", type=int, default=0, help="voxels per axis (0: the workload's own)")
    ap.add_argument("--stations", type=int, default=0, help="stations per axis (0: the workload's own)")
    ap.add_argument("--mode", default="auto", choices=["auto", "fmm", "direct"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--p", type=int, default=0, help="expansion degree (0: the workload's default)")
    ap.add_argument("--leaf-vox", type=int, default=0)
    ap.add_argument("--m2l", default="auto", choices=["auto", "simt"])
    ap.add_argument("--sample-obs", type=int, default=8192,
                    help="observers in the oracle's bounded sample")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--parallel", default="replicas", choices=["replicas", "sources"],
                    help="N > 1: independent replicas (weak scaling), or one solve with the sources "
                         "split over the ranks and one sum all-reduce of the field (strong scaling)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the FP64 FMM and the lower-degree runs beside the headline")
    ap.add_argument("--points", type=int, default=1 << 24, help="points: number of scattered points")
    ap.add_argument("--workload", default="scale",
                    choices=["volume", "scale", "serving", "adjoint", "sum_an", "topo_hex", "points"],
                    help="scale (default): 464^3 layered model, 1024^2 stations; volume: 128^3 random "
                         "field, stations + voxel centres; serving: a stream of uneven requests; adjoint: misfit "
                         "gradients of 16 models at 256^2 stations; sum_an: voxels integrated in closed form "
                         "(FMM: 128^3 random field at 512^2 stations; --mode direct: the 16^3 prism model); "
                         "topo_hex: terrain-following hexahedra (256 x 256 x 64 cells, 8 nodes each) at 512^2 "
                         "draped stations; points: 2^24 scattered points with volumes at 512^2 stations")
    ap.add_argument("--requests", type=int, default=512, help="serving: requests per pass")
    ap.add_argument("--slots", type=int, default=8, help="serving: requests on the device at once")
    ap.add_argument("--rate", type=float, default=0.0,
                    help="serving: Poisson arrival rate in requests/s (0: half the saturated rate)")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, enabled: bool):
        self.proc = None
        self.path = None
        self.gpu = gpu_index
        if not enabled:
            return
        try:
            # the raw samples go to $GF_CLOCKS_DIR (default: the system temp dir)
            out_dir = os.environ.get("GF_CLOCKS_DIR") or tempfile.gettempdir()
            os.makedirs(out_dir, exist_ok=True)
            self.path = os.path.join(out_dir, "clocks_bench_%d.csv" % os.getpid())
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
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
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ ranks
def max_over_ranks(x, world, device="cpu"):
    """The largest value of x over the ranks (a job's time is that of its
    slowest rank); x itself on one rank."""
    if world <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch
        torch.distributed.barrier()


def sum_over_ranks(t, world):
    """Sum a tensor over the ranks in place (the one exchange of a
    source-partitioned solve: each rank holds its sources' field)."""
    if world > 1:
        import torch
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.SUM)
    return t


def job_rate(units_per_rank, world, seconds):
    """Whole-job throughput: every rank processed units_per_rank in at most
    `seconds` (replicas, weak scaling)."""
    return world * float(units_per_rank) / float(seconds)


# ------------------------------------------------------------------ workload
# Expansion degree per workload: the headline runs the mixed-precision FMM at
# a degree whose sampled error stays below the metric's 1e-6 with margin, and
# the plain FP64 FMM beside it at the smallest degree that meets 1e-6.
DEFAULT_P = {"scale": 10, "volume": 12, "sum_an": 12, "topo_hex": 12, "points": 12}
FP64_P = {"scale": 10, "volume": 14}
SWEEP_P = (4, 6, 8)
REL_ERR_BAR = 1e-6


def make_workload(args):
    from paper_1107_5951_gb300 import workloads as wl
    if args.workload == "scale":
        return wl.layered_scale(n=args.side or 464, stations=args.stations or 1024)
    return wl.grf_volume(n=args.side or 128, stations=args.stations or 512)


def workload_p(args):
    return args.p if args.p else DEFAULT_P.get(args.workload, 12)


def workload_config(wk, world, parallel="replicas"):
    """The workload as both arms name it (identical dicts)."""
    par = "single" if world <= 1 else ("replicas" if parallel == "replicas" else "source_parts")
    return {"workload": wk.name, "N_sources": int(wk.n_sources), "M_observers": int(wk.n_obs),
            "rel_err_bar": REL_ERR_BAR, "parallelism": par,
            "l2_flush": "GPU arm: a 256 MiB buffer is written between timed steps; host arm: n/a"}


ORACLE_SAMPLE_PAIRS = 2.0e10     # bounds the oracle's sample to ~15 s on 16 cores


def oracle_sample(wk, args, seed=17):
    rng = np.random.default_rng(seed)
    cap = max(16, int(ORACLE_SAMPLE_PAIRS / wk.n_sources))
    idx = np.sort(rng.choice(wk.n_obs, size=min(args.sample_obs, cap, wk.n_obs), replace=False))
    return idx


def run_cpu_oracle(wk, idx):
    from oracle import direct
    t0 = time.perf_counter()
    rho = np.asarray(wk.rho, dtype=np.float64)
    g = direct.forward(wk.grid.n, wk.grid.origin, wk.grid.h, wk.xi, wk.w, rho, wk.obs[idx], wk.G)
    dt = time.perf_counter() - t0
    return g, dt, direct.max_threads()


def fp32_peak_tflops(peaks):
    return N_SM * FP32_LANES_PER_SM * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12


def sfu_peak_per_s(peaks):
    """Reciprocal square roots per second: 16 per SM per clock (SFU)."""
    return N_SM * SFU_RSQRT_PER_SM * peaks.get("sm_max_mhz", 2070.0) * 1e6


def level_boxes(info, l):
    n = 1
    for a in range(3):
        n *= int(info.src_hi[l][a]) - int(info.src_lo[l][a]) + 1
    return n


SPLIT_PRODUCTS = 3              # tensor-core products per algorithmic one (FP16 or TF32 high/low parts)
P2M_FLOPS_PER_HARMONIC = 10.0   # point P2M: one recursion step (6 flops) + the mass-weighted sum (4)


def fmm_roofline(stages, info, args, peaks, workload, nvox=None, rho_bytes=4, n_points=None):
    """Roofline of the kernel that dominates the forward: the near-field
    evaluation (ALU: 20 flops per pair, the paper's count; its SFU share
    beside it), the M2L (tensor: 2 K^2 flops per interaction-list box pair),
    or the HBM-bound P2M / M2M (densities read once and expansions written
    once; each child expansion read once and each parent written once)."""
    K = int(info.K)
    p = workload_p(args)
    tensor = (args.precision == "mixed" or args.m2l == "tensor") and p <= 15 and args.m2l != "simt"
    fbytes = 4 if args.precision == "mixed" else 8
    L = int(getattr(info, "L", 0))
    work = {"eval": ("alu", FLOPS_PER_PAIR * float(info.near_pairs),
                     "eval_kernel (near field) + eval_far_kernel (L2P, near + far, scatter)"),
            "m2l": ("tensor" if tensor else "alu", 2.0 * K * K * float(info.m2l_pairs),
                    "m2l_tc (tcgen05 FP16 parts, 3 products, all levels)" if tensor
                    else "m2l_simt (all levels)")}
    if nvox is not None and L >= 2:
        ns = {l: level_boxes(info, l) for l in range(2, L + 1)}
        # mixed precision on the tensor cores with L - 1 > 2: the P2M stage
        # makes level L-1 straight from the densities (its essential traffic:
        # the densities once, those expansions once) and the M2M stage starts
        # from level L-1
        up = tensor and L - 1 > 2
        top = L - 1 if up else L
        work["p2m"] = ("hbm", float(nvox * rho_bytes + ns[top] * K * fbytes),
                       "block_rows + m2l_tc P2M kinds (into level L-1 from the grid)" if up
                       else ("block_rows + m2l_tc P2M kind" if tensor else "p2m_fused"))
        work["m2m"] = ("hbm", float(sum(ns[l] * K * fbytes for l in range(3, top + 1))
                                    + sum(ns[l] * K * fbytes for l in range(2, top))),
                       "m2l_tc M2M kind + m2m_kernel (FP64 into level 2)" if tensor else "xlate_simt")
    if n_points is not None and L >= 2:
        # point sources: the P2M evaluates (p+1)(p+2)/2 complex harmonics per
        # point; the M2M reads each level's expansions once and writes the
        # parents' once
        ns = {l: level_boxes(info, l) for l in range(2, L + 1)}
        work["p2m"] = ("alu", P2M_FLOPS_PER_HARMONIC * (p + 1) * (p + 2) / 2 * float(n_points),
                       "point_p2m_f32 (packed pair recursion)" if args.precision == "mixed" else "point_p2m")
        work["m2m"] = ("hbm", float(sum(ns[l] * K * fbytes for l in range(3, L + 1))
                                    + sum(ns[l] * K * fbytes for l in range(2, L))),
                       "m2l_tc M2M kind + m2m_kernel (FP64 into level 2)" if tensor else "xlate_simt")
    dom = max(work, key=lambda k: stages.get(k, 0.0))
    bound, amount, kern = work[dom]
    extra = {}
    if bound == "tensor":
        peak, unit = peaks.get("bf16_tflops", 1870.7) * F16_PER_BF16, "TFLOP/s"
        note = ("FP16 dense = measured BF16 burst x nominal FP16/BF16 (1); the high/low split "
                "executes 3 MMAs per algorithmic flop")
        achieved = amount / (stages[dom] * 1e-3) / 1e12
        # three products per algorithmic one: the algorithmic fraction is at
        # most 1/3; pipe_frac is the tensor pipe's share of its peak
        extra = {"pipe_frac": SPLIT_PRODUCTS * achieved / peak,
                 "pipe_source": "algorithmic rate x 3 (high/low parts: hi*lo + lo*hi + hi*hi per product)"}
    elif bound == "hbm":
        peak, unit = peaks.get("hbm_gbs", 6774.6), "GB/s"
        note = "measured HBM copy bandwidth"
        achieved = amount / (stages[dom] * 1e-3) / 1e9
    elif args.precision == "mixed":
        peak, unit = fp32_peak_tflops(peaks), "TFLOP/s"
        note = "FP32 SIMT: 152 SM x 128 lanes x 2 x sm_max_mhz"
        achieved = amount / (stages[dom] * 1e-3) / 1e12
        if dom == "eval":
            rate = float(info.near_pairs) / (stages[dom] * 1e-3)
            extra = {"sfu_frac": rate / sfu_peak_per_s(peaks),
                     "sfu_frac_of_probe": rate / MUFU_RSQRT_PROBE,
                     "frac_of_fp32_probe": achieved / FP32_TFLOPS_PROBE,
                     "sfu_source": "one reciprocal square root per pair: 152 SM x 16 per clock x sm_max_mhz; "
                                   "probe = measured MUFU rsqrt throughput on this GPU (%.3g/s)"
                                   % MUFU_RSQRT_PROBE}
    else:
        peak, unit = FP64_TFLOPS_NOMINAL, "TFLOP/s"
        note = "FP64 nominal 1.25 TFLOP/s"
        achieved = amount / (stages[dom] * 1e-3) / 1e12
    traffic = ncu_traffic(dom, workload, p, args.precision, args.m2l)
    r = {"bound": bound, "kernel": kern, "stage": dom, "achieved": achieved, "peak": peak,
         "unit": unit, "frac": achieved / peak, "traffic": traffic, "peak_source": note,
         "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum, one capture "
                           "(profiles/), per launch set" if traffic else None,
         "algorithmic": "%.4g %s per launch set" % (amount, "bytes" if bound == "hbm" else "flops"),
         "stage_ms": stages[dom]}
    r.update(extra)
    return r


# ------------------------------------------------------------------ reference arm
def points_reference(args, world):
    """The host arm of the point-source workloads: the oracle's direct sum
    (node images and weights included for the hexahedra) on a bounded sample
    of stations per step."""
    from oracle import direct
    from paper_1107_5951_gb300 import workloads as wl
    hexes = args.workload == "topo_hex"
    if hexes:
        n = args.side or 256
        wk = wl.topo_workload(n, n, max(1, n // 4), args.stations or 512, 2)
        S = len(wk["rho"]) * len(wk["w"])
    else:
        wk = wl.points_cloud(args.points, args.stations or 512)
        S = len(wk["a"])
    M = len(wk["obs"])
    per_step = int(max(8, min(M, 3.0e9 / S)))
    rng = np.random.default_rng(31)
    times = []
    for s in range(args.warmup + args.steps):
        idx = np.sort(rng.choice(M, per_step, replace=False))
        t0 = time.perf_counter()
        if hexes:
            direct.forward_hex(wk["verts"], wk["xi"], wk["w"], wk["rho"], wk["obs"][idx], wk["G"])
        else:
            direct.forward_points(wk["x"], wk["a"], 1, wk["rho"], wk["obs"][idx], wk["G"])
        if s >= args.warmup:
            times.append(time.perf_counter() - t0)
    value = S * per_step * len(times) / sum(times)
    sample = "%d seeded stations per step of %d x all %d sources" % (per_step, M, S)
    line = {"impl": "reference",
            "metric": "effective interactions/s (%s)" % ("deformed hexahedra" if hexes else "scattered points"),
            "value": value, "unit": "interactions/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wk["name"], "N_sources": int(S), "M_observers": int(M),
                       "rel_err_bar": REL_ERR_BAR, "l2_flush": "host arm: n/a"},
            "method": {"impl": "FP64 direct sum on the host cores (the oracle)"},
            "cpu_baseline": {"value": value, "unit": "interactions/s", "cores": direct.max_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "interactions/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def bench_reference(args, rank, world):
    if rank != 0:
        return
    if args.workload in ("topo_hex", "points"):
        points_reference(args, world)
        return
    wk = make_workload(args)
    n_src = wk.n_sources
    idx_all = oracle_sample(wk, args)
    # each step evaluates a bounded sample of observers against every source
    # (about 2 s of host work per step)
    per_step = int(max(8, min(len(idx_all), 3.0e9 / n_src)))
    times = []
    for s in range(args.warmup + args.steps):
        idx = np.resize(np.roll(idx_all, -s * per_step), per_step)
        _, dt, cores = run_cpu_oracle(wk, idx)
        if s >= args.warmup:
            times.append((dt, len(idx)))
    tot_t = sum(t for t, _ in times)
    tot_pairs = sum(n * n_src for _, n in times)
    value = tot_pairs / tot_t
    sample = "%d observers per step (seeded subset of %d) x all %d sources" % (per_step, wk.n_obs, n_src)
    line = {"impl": "reference", "metric": "effective interactions/s", "value": value,
            "unit": "interactions/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot_t / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(wk, world, args.parallel),
            "method": {"impl": "FP64 direct sum on the host cores (the oracle)"},
            "cpu_baseline": {"value": value, "unit": "interactions/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "interactions/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm
def timed_forwards(plan, rho_d, g_d, stream, flush, reps):
    """Mean CUDA-event time of `reps` warm forwards on `stream`, L2 flushed
    before each."""
    import torch
    ev = []
    for k in range(reps):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        plan.forward(rho_d, g=g_d, stream=stream)
        b.record(stream)
        ev.append((a, b))
    torch.cuda.synchronize()
    return float(np.mean([a.elapsed_time(b) for a, b in ev]))


def bench_gf(args, rank, world):
    import torch

    import paper_1107_5951_gb300 as pkg

    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    peaks = load_peaks()
    wk = make_workload(args)
    N, M = wk.n_sources, wk.n_obs
    units = float(N) * float(M)
    p = workload_p(args)

    mode = args.mode
    if mode == "auto":
        mode = "fmm"
    stream = torch.cuda.Stream(device=dev)
    obs_d = torch.tensor(wk.obs, dtype=torch.float64, device=dev)
    rho_dtype = torch.float32 if args.precision == "mixed" else torch.float64
    rho_d = torch.tensor(wk.rho, dtype=rho_dtype, device=dev)
    g_d = torch.empty((M, 3), dtype=torch.float64, device=dev)

    parts = world > 1 and args.parallel == "sources"

    def make_plan(precision=args.precision, pp=p, obs=obs_d, m2l=args.m2l):
        pl = pkg.Plan(wk.grid.n, wk.grid.origin, wk.grid.h, wk.xi, wk.w, obs, mode=mode,
                      precision=precision, p=pp, leaf_vox=args.leaf_vox, G=wk.G,
                      stream=stream, m2l=m2l)
        if parts:
            pl.set_source_part(rank, world)
        return pl

    try:
        probe = make_plan()
    except pkg.GfError as e:
        if mode == "fmm" and args.mode == "auto" and e.status == 4:
            mode = "direct"
            probe = make_plan()
        else:
            raise
    plan_info = probe.info
    probe.close()

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        with torch.cuda.stream(stream):
            plan = make_plan()
            plan.forward(rho_d, g=g_d, stream=stream)
            if parts:
                sum_over_ranks(g_d, world)   # NCCL on the forward's stream
            plan.close()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(world)
    clocks = ClockSampler(local_rank, not args.no_clocks)
    launches0 = pkg.gf_launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.fill_(float(k))          # evict L2 between timed steps
        torch.cuda.synchronize()
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    launches = pkg.gf_launch_count() - launches0
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    torch.cuda.synchronize()
    tot_ms = max_over_ranks(float(sum(step_ms)), world, dev)
    # replicas: every rank solves the whole problem; source parts: the ranks
    # share one problem
    value = job_rate(units * args.steps, 1 if parts else world, tot_ms * 1e-3)

    # warm forward with the plan built; per-stage device times
    plan = make_plan()
    fwd_ms = timed_forwards(plan, rho_d, g_d, stream, flush, args.steps)
    if parts:
        with torch.cuda.stream(stream):
            sum_over_ranks(g_d, world)
        torch.cuda.synchronize()
    g_main = g_d.cpu().numpy()
    plan.set_timing(True)
    stage_runs = []
    for k in range(args.steps):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        plan.forward(rho_d, g=g_d, stream=stream)
        stage_runs.append(plan.stage_times())
    plan.set_timing(False)
    stages = {k: float(np.mean([r[k] for r in stage_runs])) for k in stage_runs[0]}
    info = plan.info
    plan.close()

    # the plain FP64 FMM on the same GPU, and the mixed form at lower degrees
    compare = {}
    sampled = {}
    if mode == "fmm" and not args.no_compare and not parts:
        rho64 = rho_d.double() if args.precision == "mixed" else rho_d
        pf = FP64_P.get(args.workload, 14)
        with make_plan("fp64", pf) as pl:
            pl.forward(rho64, g=g_d, stream=stream)
            ms = timed_forwards(pl, rho64, g_d, stream, flush, 2)
            sampled["fp64_fmm"] = g_d.cpu().numpy()
        compare["fp64_fmm"] = {"precision": "fp64", "p": pf, "ms_per_solve": ms,
                               "value": units / (ms * 1e-3), "unit": "interactions/s"}
        # the FP64 FMM with its M2L on the tensor cores (FP16 parts; the rest FP64)
        with make_plan("fp64", pf, m2l="tensor") as pl:
            pl.forward(rho64, g=g_d, stream=stream)
            ms = timed_forwards(pl, rho64, g_d, stream, flush, 2)
            sampled["fp64_tc_m2l"] = g_d.cpu().numpy()
            pl.set_timing(True)
            pl.forward(rho64, g=g_d, stream=stream)
            st64 = pl.stage_times()
            info64 = pl.info
        a64 = argparse.Namespace(precision="fp64", p=pf, m2l="tensor", workload=args.workload)
        compare["fp64_tc_m2l"] = {"precision": "fp64", "m2l": "tensor cores (FP16 parts)", "p": pf,
                                  "ms_per_solve": ms, "value": units / (ms * 1e-3), "unit": "interactions/s",
                                  "stages_ms": st64,
                                  "roofline": fmm_roofline(st64, info64, a64, peaks, wk.name + "_fp64")}
        del rho64
        if args.precision == "mixed":
            for ps in SWEEP_P:
                with make_plan("mixed", ps) as pl:
                    pl.forward(rho_d, g=g_d, stream=stream)
                    ms = timed_forwards(pl, rho_d, g_d, stream, flush, max(3, args.steps // 4))
                    sampled["p%d" % ps] = g_d.cpu().numpy()
                compare["mixed_p%d" % ps] = {"precision": "mixed", "p": ps, "ms_per_solve": ms,
                                             "value": units / (ms * 1e-3), "unit": "interactions/s"}
        compare["mixed_over_fp64"] = compare["fp64_fmm"]["ms_per_solve"] / fwd_ms

    # accuracy on the oracle's sample (rank 0 only)
    idx = oracle_sample(wk, args)
    cpu = None
    rel_err = None
    if rank == 0 and (world == 1 or parts) and not args.no_cpu_baseline:
        ref, dt, cores = run_cpu_oracle(wk, idx)
        nref = np.linalg.norm(ref)
        rel_err = float(np.linalg.norm(g_main[idx] - ref) / nref)
        for key, gs in sampled.items():
            ck = key if key.startswith("fp64") else "mixed_" + key
            compare[ck]["rel_err_vs_oracle_sample"] = float(np.linalg.norm(gs[idx] - ref) / nref)
        cpu = {"value": N * len(idx) / dt, "unit": "interactions/s", "cores": cores, "kind": "oracle",
               "sample": "%d seeded observers of %d x all %d sources (%.1f s)" % (len(idx), M, N, dt)}

    # roofline of the dominant kernel
    if mode == "direct":
        flops = FLOPS_PER_PAIR * units
        if args.precision == "mixed":
            peak = fp32_peak_tflops(peaks)
            peak_note = "FP32 SIMT: 152 SM x 128 lanes x 2 flop x sm_max_mhz (%s clocks)" % peaks["_source"]
        else:
            peak = FP64_TFLOPS_NOMINAL
            peak_note = "FP64 nominal 1.25 TFLOP/s"
        achieved = flops / (fwd_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "kernel": "direct_fwd_%s" % ("mixed" if args.precision == "mixed" else "f64"),
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "peak_source": peak_note,
                "algorithmic": "%.0f flops/pair x N*M pairs" % FLOPS_PER_PAIR}
    else:
        roof = fmm_roofline(stages, info, args, peaks, wk.name, nvox=wk.grid.nvox,
                            rho_bytes=4 if args.precision == "mixed" else 8)

    # end to end through the C ABI from pinned host buffers: the observers
    # are copied first (the plan build needs them), the densities on a second
    # stream while the plan is built, and the forward waits for them
    e2e = None
    if not args.no_e2e:
        obs_h = torch.tensor(wk.obs, dtype=torch.float64).pin_memory()
        rho_h = torch.tensor(wk.rho, dtype=rho_dtype).pin_memory()
        g_h = torch.empty((M, 3), dtype=torch.float64).pin_memory()
        obs_e = torch.empty_like(obs_d)
        rho_e = torch.empty_like(rho_d)
        copy_stream = torch.cuda.Stream(device=dev)
        e_ev = []
        for k in range(args.warmup + args.steps):   # warm-up passes first, as for the device leg
            flush.fill_(float(k))
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            with torch.cuda.stream(stream):
                obs_e.copy_(obs_h, non_blocking=True)
            copy_stream.wait_stream(stream)
            with torch.cuda.stream(copy_stream):
                rho_e.copy_(rho_h, non_blocking=True)
                rho_ready = torch.cuda.Event()
                rho_ready.record(copy_stream)
            with torch.cuda.stream(stream):
                pl = make_plan(obs=obs_e)
                stream.wait_event(rho_ready)
                pl.forward(rho_e, g=g_d, stream=stream)
                if parts:
                    sum_over_ranks(g_d, world)
                g_h.copy_(g_d, non_blocking=True)
                pl.close()
            b.record(stream)
            if k >= args.warmup:
                e_ev.append((a, b))
        torch.cuda.synchronize()
        e_ms = max_over_ranks(float(np.mean([a.elapsed_time(b) for a, b in e_ev])), world, dev)
        e2e = {"value": job_rate(units, 1 if parts else world, e_ms * 1e-3), "unit": "interactions/s",
               "h2d_bytes_per_step": int(obs_h.numel() * 8 + rho_h.numel() * rho_h.element_size()),
               "d2h_bytes_per_step": int(g_h.numel() * 8), "ms_per_step": e_ms}

    if rank != 0:
        return
    line = {"metric": "effective interactions/s", "value": value, "unit": "interactions/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
            "scaling": "strong" if parts else "weak",
            "vs_baseline": None, "dtype": "f32" if args.precision == "mixed" else "f64",
            "data": "synthetic",
            "config": workload_config(wk, world, args.parallel),
            "method": {"mode": mode, "precision": args.precision, "p": p if mode == "fmm" else None,
                       "m2l": args.m2l,
                       "leaf_vox": int(plan_info.leaf_vox) if mode == "fmm" else None,
                       "levels": int(plan_info.L) if mode == "fmm" else None,
                       "step": "plan build + forward + release"},
            "ms_per_solve": fwd_ms, "rel_err_vs_oracle_sample": rel_err,
            "meets_rel_err_bar": None if rel_err is None else bool(rel_err <= REL_ERR_BAR),
            "stages_ms": stages,
            "work": {"near_pairs": int(info.near_pairs), "m2l_box_pairs": int(info.m2l_pairs)},
            "compare": compare or None,
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
            "gpu_launches": int(launches)}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ adjoint
def bench_adjoint(args, rank, world):
    """Misfit gradient for a batch of 16 models (128^3 random fields, 256^2
    stations): one step = forward of the batch (g_z), residual against data
    synthesised from a hidden model, and the transposed FMM (gf_adjoint) of
    the residuals -> d misfit / d rho for all 16 models.  Unit of work: the
    N x M pairs of one model's forward plus its adjoint."""
    import torch

    import paper_1107_5951_gb300 as pkg
    from oracle import direct
    from paper_1107_5951_gb300 import workloads as wl

    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    B = 16
    wk = wl.adjoint_batch(n=args.side or 128, stations=args.stations or 256, batch=B)
    N, M = wk.n_sources, wk.n_obs
    stream = torch.cuda.Stream(device=dev)
    obs_d = torch.tensor(wk.obs, dtype=torch.float64, device=dev)
    rdt = torch.float32 if args.precision == "mixed" else torch.float64
    models = torch.tensor(wk.rho, dtype=rdt, device=dev)
    plan = pkg.Plan(wk.grid.n, wk.grid.origin, wk.grid.h, wk.xi, wk.w, obs_d, mode="fmm",
                    precision=args.precision, p=workload_p(args), max_batch=B, G=wk.G, stream=stream)
    hidden = torch.tensor(wk.extra["hidden"], dtype=rdt, device=dev)
    _, d = plan.forward(hidden, want_g=False, want_gz=True, stream=stream)
    gz = torch.empty((B, M), dtype=torch.float64, device=dev)
    grad = torch.empty((B,) + wk.grid.shape_zyx, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        with torch.cuda.stream(stream):
            plan.forward(models, gz=gz, want_g=False, want_gz=True, stream=stream)
            r = gz - d
            plan.adjoint(r, ncomp=1, grad=grad, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(world)
    clocks = ClockSampler(local_rank, not args.no_clocks)
    launches0 = pkg.gf_launch_count()
    ev = []
    for k in range(args.steps):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        ev.append((a, b))
    torch.cuda.synchronize()
    launches = pkg.gf_launch_count() - launches0
    clk = clocks.stop()
    ms = max_over_ranks(float(np.mean([a.elapsed_time(b) for a, b in ev])), world, dev)
    units = float(B) * N * M * 2
    # parity on sampled voxels of model 0 against the FP64 CPU transpose sum
    err, cpu = None, None
    if rank == 0 and not args.no_cpu_baseline:
        r0 = (gz[0] - d).cpu().numpy()
        rng = np.random.default_rng(23)
        vox = np.sort(rng.choice(wk.grid.nvox, 4096, replace=False))
        t1 = time.perf_counter()
        want = direct.adjoint_subset(wk.grid.n, wk.grid.origin, wk.grid.h, wk.xi, wk.w, wk.obs, r0, wk.G, vox)
        dt = time.perf_counter() - t1
        got = grad[0].reshape(-1).cpu().numpy()[vox]
        err = float(np.linalg.norm(got - want) / np.linalg.norm(want))
        cpu = {"value": len(vox) * M / dt, "unit": "interactions/s", "cores": direct.max_threads(),
               "kind": "oracle", "sample": "adjoint at 4096 seeded voxels of model 0 x all %d stations (%.1f s)"
               % (M, dt)}
    plan.close()
    if rank != 0:
        return
    line = {"metric": "misfit-gradient interactions/s (forward + adjoint, 16 models)",
            "value": job_rate(units, world, ms * 1e-3), "unit": "interactions/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == "mixed" else "f64",
            "data": "synthetic",
            "config": {"workload": wk.name, "precision": args.precision, "p": workload_p(args), "batch": B,
                       "N_sources": N, "M_observers": M,
                       "l2_flush": "256 MiB buffer written between timed steps",
                       "step": "forward of 16 models + residual + adjoint of 16 residuals"},
            "gradients_per_s": world * B / (ms * 1e-3), "rel_err_vs_oracle_sample": err,
            "roofline": None, "cpu_baseline": cpu, "clocks": clk, "gpu_launches": int(launches)}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ SUM-AN
def bench_sum_an(args, rank, world):
    """SUM-AN: every voxel integrated in closed form (Sec. 2.1).  FMM mode
    (default): the 128^3 random-field model of 250 m voxels at 512^2 surface
    stations, mixed precision, the voxels next to each station in closed
    form, the far field from exact voxel moments.  Direct mode (--mode
    direct): the 16^3 prism model (1 km voxels) at the 64^2 stations 100 m
    above it, every (voxel, station) pair in closed form, FP64.  One step =
    one forward.  Unit of work: a (voxel, observer) pair."""
    import torch

    import paper_1107_5951_gb300 as pkg
    from oracle import direct
    from paper_1107_5951_gb300 import workloads as wl

    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    fmm = args.mode != "direct"
    if fmm:
        wk = wl.grf_volume(n=args.side or 128, stations=args.stations or 512, volume_targets=False)
        precision, p = args.precision, workload_p(args)
    else:
        wk = wl.fp64_prism_noise(1)
        precision, p = "fp64", 8
    nvox, M = int(np.prod(wk.grid.n)), wk.n_obs
    stream = torch.cuda.Stream(device=dev)
    obs_d = torch.tensor(wk.obs, dtype=torch.float64, device=dev)
    rdt = torch.float32 if precision == "mixed" else torch.float64
    rho_d = torch.tensor(wk.rho, dtype=rdt, device=dev)
    g_d = torch.empty((M, 3), dtype=torch.float64, device=dev)
    plan = pkg.Plan(wk.grid.n, wk.grid.origin, wk.grid.h, wk.xi, wk.w, obs_d, mode="fmm" if fmm else "direct",
                    precision=precision, p=p, G=wk.G, stream=stream, voxels="closed_form")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        with torch.cuda.stream(stream):
            plan.forward(rho_d, g=g_d, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(world)
    clocks = ClockSampler(local_rank, not args.no_clocks)
    launches0 = pkg.gf_launch_count()
    ev = []
    for k in range(args.steps):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        ev.append((a, b))
    torch.cuda.synchronize()
    launches = pkg.gf_launch_count() - launches0
    clk = clocks.stop()
    ms = max_over_ranks(float(np.mean([a.elapsed_time(b) for a, b in ev])), world, dev)
    stages = None
    if fmm:
        plan.set_timing(True)
        plan.forward(rho_d, g=g_d, stream=stream)
        stages = plan.stage_times()
        plan.set_timing(False)
    units = float(nvox) * M
    err, cpu = None, None
    if rank == 0 and not args.no_cpu_baseline:
        rng = np.random.default_rng(29)
        idx = np.sort(rng.choice(M, 64 if fmm else 256, replace=False))
        rho64 = np.asarray(wk.rho, dtype=np.float32 if precision == "mixed" else np.float64).astype(np.float64)
        t1 = time.perf_counter()
        want = direct.forward_analytic(wk.grid.n, wk.grid.origin, wk.grid.h, rho64, wk.obs[idx], wk.G)
        dt = time.perf_counter() - t1
        got = g_d.cpu().numpy()[idx]
        err = float(np.linalg.norm(got - want) / np.linalg.norm(want))
        cpu = {"value": nvox * len(idx) / dt, "unit": "interactions/s", "cores": direct.max_threads(),
               "kind": "oracle", "sample": "%d seeded stations of %d x all %d voxels in closed form (%.1f s)"
               % (len(idx), M, nvox, dt)}
    plan.close()
    if rank != 0:
        return
    line = {"metric": "effective interactions/s (SUM-AN, closed-form voxels)",
            "value": job_rate(units, world, ms * 1e-3), "unit": "interactions/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if precision == "mixed" else "f64",
            "data": "synthetic",
            "config": {"workload": wk.name + "_sum_an", "voxels": nvox, "M_observers": M,
                       "l2_flush": "256 MiB buffer written between timed steps"},
            "method": {"mode": "fmm" if fmm else "direct", "precision": precision, "p": p if fmm else None,
                       "step": "forward (closed form next to each observer, exact voxel moments beyond)"
                       if fmm else "corner-lattice weights + closed-form sum over the corner lattice"},
            "stages_ms": stages, "rel_err_vs_oracle_sample": err, "roofline": None, "cpu_baseline": cpu,
            "clocks": clk, "gpu_launches": int(launches)}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ point sources
def bench_points(args, rank, world):
    """Weighted point sources.  topo_hex: a terrain-following hexahedral
    mesh (256 x 256 x 64 cells over 16 km x 16 km, 8 km deep, 800 m relief;
    the 2^3 Gauss rule per cell: 33.5M sources) at 512^2 stations draped
    50 m over the terrain; a step = gf_hex_sources (node images and |det J|
    weights) + plan build + forward + release.  points: 2^24 scattered
    points with volumes in a 16 km x 16 km x 4 km slab at 512^2 stations; a
    step = plan build + forward + release.  Unit of work: a (source,
    observer) pair."""
    import torch

    import paper_1107_5951_gb300 as pkg
    from oracle import direct
    from paper_1107_5951_gb300 import workloads as wl

    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    hexes = args.workload == "topo_hex"
    mode = "direct" if args.mode == "direct" else "fmm"
    precision = args.precision
    p = args.p if args.p else (DEFAULT_P[args.workload] if precision == "mixed" else 14)
    if hexes:
        n = args.side or 256
        wk = wl.topo_workload(n, n, max(1, n // 4), args.stations or 512, 2)
        per_cell = len(wk["w"])
        S = len(wk["rho"]) * per_cell
        verts_d = torch.tensor(wk["verts"], dtype=torch.float64, device=dev)
        name = wk["name"]
    else:
        wk = wl.points_cloud(args.points, args.stations or 512)
        per_cell, S = 1, len(wk["a"])
        x_d = torch.tensor(wk["x"], dtype=torch.float64, device=dev)
        a_d = torch.tensor(wk["a"], dtype=torch.float64, device=dev)
        name = wk["name"]
    M = len(wk["obs"])
    stream = torch.cuda.Stream(device=dev)
    obs_d = torch.tensor(wk["obs"], dtype=torch.float64, device=dev)
    rdt = torch.float32 if precision == "mixed" else torch.float64
    rho_d = torch.tensor(wk["rho"], dtype=rdt, device=dev)
    g_d = torch.empty((M, 3), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    kw = dict(per_cell=per_cell, mode=mode, precision=precision, p=p, G=wk["G"], stream=stream,
              m2l=args.m2l)

    def sources():
        if hexes:
            return pkg.hex_sources(verts_d, wk["xi"], wk["w"], precision=precision, stream=stream)
        return x_d, a_d

    def step():
        with torch.cuda.stream(stream):
            x, a = sources()
            plan = pkg.PointsPlan(x, a, obs_d, **kw)
            plan.forward(rho_d, g=g_d, stream=stream)
            plan.close()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(world)
    clocks = ClockSampler(local_rank, not args.no_clocks)
    launches0 = pkg.gf_launch_count()
    ev = []
    for k in range(args.steps):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        a0, b0 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        step()
        b0.record(stream)
        ev.append((a0, b0))
    torch.cuda.synchronize()
    launches = pkg.gf_launch_count() - launches0
    clk = clocks.stop()
    ms = max_over_ranks(float(np.mean([a.elapsed_time(b) for a, b in ev])), world, dev)
    # the forward alone, with the plan built; its stages
    with torch.cuda.stream(stream):
        x, a = sources()
        plan = pkg.PointsPlan(x, a, obs_d, **kw)
    torch.cuda.synchronize()
    ms_solve = timed_forwards(plan, rho_d, g_d, stream, flush, max(3, args.steps))
    stages = None
    roof = None
    info = plan.info
    if mode == "fmm":
        plan.set_timing(True)
        plan.forward(rho_d, g=g_d, stream=stream)
        stages = plan.stage_times()
        plan.set_timing(False)
        roof = fmm_roofline(stages, info, args, load_peaks(), name, n_points=S)
        if roof["stage"] == "eval":
            roof["kernel"] = "point_eval (near field over the neighbour leaves' points + L2P + combine)"
    torch.cuda.synchronize()
    g_host = g_d.cpu().numpy()
    work = {"near_pairs": int(info.near_pairs), "m2l_box_pairs": int(info.m2l_pairs), "levels": int(info.L),
            "leaf_side_m": float(info.leaf_side)}
    plan.close()
    err, cpu = None, None
    if rank == 0 and not args.no_cpu_baseline:
        rng = np.random.default_rng(31)
        idx = np.sort(rng.choice(M, min(M, 64), replace=False))
        rho64 = np.asarray(wk["rho"], dtype=np.float32 if precision == "mixed" else np.float64).astype(np.float64)
        t1 = time.perf_counter()
        if hexes:
            want = direct.forward_hex(wk["verts"], wk["xi"], wk["w"], rho64, wk["obs"][idx], wk["G"])
        else:
            want = direct.forward_points(wk["x"], wk["a"], 1, rho64, wk["obs"][idx], wk["G"])
        dt = time.perf_counter() - t1
        err = float(np.linalg.norm(g_host[idx] - want) / np.linalg.norm(want))
        cpu = {"value": S * len(idx) / dt, "unit": "interactions/s", "cores": direct.max_threads(),
               "kind": "oracle", "sample": "%d seeded stations of %d x all %d sources%s (%.1f s)"
               % (len(idx), M, S, ", node images and weights included" if hexes else "", dt)}
    if rank != 0:
        return
    line = {"metric": "effective interactions/s (%s)" % ("deformed hexahedra" if hexes else "scattered points"),
            "value": job_rate(float(S) * M, world, ms * 1e-3), "unit": "interactions/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if precision == "mixed" else "f64",
            "data": "synthetic",
            "config": {"workload": name, "N_sources": int(S), "M_observers": int(M), "rel_err_bar": REL_ERR_BAR,
                       "l2_flush": "256 MiB buffer written between timed steps"},
            "method": {"mode": mode, "precision": precision, "p": p if mode == "fmm" else None,
                       "step": ("gf_hex_sources + " if hexes else "") + "plan build + forward + release"},
            "ms_per_solve": ms_solve, "stages_ms": stages, "work": work, "rel_err_vs_oracle_sample": err,
            "meets_rel_err_bar": None if err is None else bool(err <= REL_ERR_BAR),
            "roofline": roof, "cpu_baseline": cpu, "e2e": None, "clocks": clk, "gpu_launches": int(launches)}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ serving
def bench_serving(args, rank, world):
    """Serving stream: `--requests` forward solves, grid side n log-uniform
    in [32, 256], 256^2 stations, random-field densities; geometry id = n.
    Warm-up passes submit the whole stream at once (plans are built and stay
    resident); timed passes do the same and give solves/s; a last pass
    submits at Poisson arrival times and gives p50/p99 of completion minus
    arrival.  Every request copies its densities from pinned host memory
    and its g_z back, inside the measured latency."""
    import torch

    import paper_1107_5951_gb300 as pkg
    from oracle import direct
    from paper_1107_5951_gb300 import workloads as wl

    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local_rank)
    reqs = wl.serving_stream(args.requests, stations=256)
    nmax = max(r["grid"].n[0] for r in reqs)
    field = wl.periodic_grf(256, reqs[0]["grid"].h[0], 2000.0, 150.0, 4, dtype=np.float32)
    sizes = [int(np.prod(r["grid"].n)) for r in reqs]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    rho_pool = torch.empty(int(offs[-1]), dtype=torch.float32, pin_memory=True)
    pool_np = rho_pool.numpy()
    for i, r in enumerate(reqs):
        pool_np[offs[i]:offs[i + 1]] = wl.serving_density(r, field).ravel()
    M = reqs[0]["obs"].shape[0]
    gz_pool = torch.empty((len(reqs), M), dtype=torch.float64, pin_memory=True)
    srv = pkg.Server(slots=args.slots, precision=args.precision, p=workload_p(args), use_graphs=True,
                     device=local_rank)
    xi, w = wl.gauss_rule(1)
    for r in reqs:
        g = r["grid"]
        srv.register(g.n[0], g.n, g.origin, g.h, xi, w, r["obs"])
    units = float(sum(sizes)) * M

    def rho_of(i):
        n = reqs[i]["grid"].n[0]
        return rho_pool[offs[i]:offs[i + 1]].view(n, n, n)

    def burst():
        t0 = time.perf_counter()
        tickets = [srv.submit(r["grid"].n[0], rho_of(i), gz=gz_pool[i]) for i, r in enumerate(reqs)]
        lat = [srv.wait(t)[2] for t in tickets]
        return time.perf_counter() - t0, lat

    cold_s, cold_lat = burst()          # first pass builds every plan
    st_cold = srv.stats()
    for _ in range(max(0, args.warmup - 1)):
        burst()
    barrier(world)
    clocks = ClockSampler(local_rank, not args.no_clocks)
    launches0 = pkg.gf_launch_count()
    pass_s = []
    for _ in range(args.steps):
        dt, _ = burst()
        pass_s.append(dt)
    launches = pkg.gf_launch_count() - launches0
    clk = clocks.stop()
    sat_s = max_over_ranks(sum(pass_s), world, torch.device("cuda", local_rank))
    sat_rate = len(reqs) * args.steps / sat_s
    # open loop at Poisson arrival times: half and 80% of the saturated rate,
    # and light load (the stream's own 100 requests/s, or a quarter of the
    # saturated rate if that is lower)
    def open_loop(rate):
        arr = np.array([r["arrival_s"] for r in reqs]) * (100.0 / rate)   # drawn at 100 requests/s
        t0 = time.perf_counter()
        tickets = []
        for i, r in enumerate(reqs):
            dt = arr[i] - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            tickets.append(srv.submit(r["grid"].n[0], rho_of(i), gz=gz_pool[i]))
        lat = np.array([srv.wait(t)[2] for t in tickets])
        return lat, time.perf_counter() - t0

    def lat_summary(rate, lat, secs):
        return {"rate_hz": rate, "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(lat.mean()), "max_ms": float(lat.max()), "achieved_hz": len(reqs) / secs}

    rate = args.rate if args.rate > 0 else 0.5 * sat_rate
    lat, open_s = open_loop(rate)
    lat_h, open_h = open_loop(0.8 * sat_rate)
    light = min(100.0, 0.25 * sat_rate)
    lat_l, open_l = open_loop(light)
    # the same stream one request at a time (submit, wait): the sum of these
    # solo times against a saturated pass shows how much the slots overlap
    solo_s = 0.0
    for i, r in enumerate(reqs):
        t1 = time.perf_counter()
        srv.wait(srv.submit(r["grid"].n[0], rho_of(i), gz=gz_pool[i]))
        solo_s += time.perf_counter() - t1
    st = srv.stats()
    srv.close()
    # accuracy of a few requests on a station sample, against the FP64 oracle
    errs = []
    if rank == 0 and not args.no_cpu_baseline:
        rng = np.random.default_rng(11)
        pick = sorted(rng.choice(len(reqs), 4, replace=False))
        t_cpu, pairs = 0.0, 0
        for i in pick:
            r = reqs[i]
            g = r["grid"]
            idx = np.sort(rng.choice(M, 64, replace=False))
            t1 = time.perf_counter()
            want = direct.forward(g.n, g.origin, g.h, xi, w, rho_of(i).numpy().astype(np.float64),
                                  r["obs"][idx], wl.G_PAPER)[:, 2]
            t_cpu += time.perf_counter() - t1
            pairs += sizes[i] * len(idx)
            got = gz_pool[i].numpy()[idx]
            errs.append(float(np.linalg.norm(got - want) / np.linalg.norm(want)))
        cpu = {"value": pairs / t_cpu, "unit": "interactions/s", "cores": direct.max_threads(),
               "kind": "oracle", "sample": "64 stations of 4 requests (sides %s), %.1f s"
               % ([reqs[i]["grid"].n[0] for i in pick], t_cpu)}
    else:
        cpu = None
    if rank != 0:
        return
    h2d = int(sum(sizes) * 4)
    d2h = int(len(reqs) * M * 8)
    line = {"metric": "serving solves/s (512-request stream, saturated)", "value": sat_rate * world,
            "unit": "solves/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(pass_s) / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.precision == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": "serving_stream_%d_req_n32-%d_256^2_stations" % (len(reqs), nmax),
                       "precision": args.precision, "p": workload_p(args), "slots": args.slots,
                       "step": "one pass of the whole stream, submitted at once",
                       "l2_flush": "inputs larger than L2 (%.1f GB of densities per pass)" % (h2d / 1e9)},
            "interactions_per_s": units * sat_rate * world / len(reqs),
            "latency_open_loop": lat_summary(rate, lat, open_s),
            "latency_open_loop_80pct": lat_summary(0.8 * sat_rate, lat_h, open_h),
            "latency_light_load": lat_summary(light, lat_l, open_l),
            "cold_pass": {"seconds": cold_s, "plans_created": int(st_cold["plans_created"]),
                          "solves_per_s": len(reqs) / cold_s},
            "overlap": {"solo_sum_ms": 1e3 * solo_s, "saturated_pass_ms": 1e3 * sum(pass_s) / args.steps,
                        "concurrency": solo_s / (sum(pass_s) / args.steps)},
            "server": {k: st[k] for k in ("completed", "failed", "plans_created", "plans_evicted",
                                          "graph_launches", "resident_bytes", "mem_budget")},
            "rel_err_vs_oracle_sample": errs, "roofline": None, "cpu_baseline": cpu,
            "e2e": {"value": sat_rate * world, "unit": "solves/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "clocks": clk, "gpu_launches": int(launches)}
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        bench_reference(args, rank, world)
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    try:
        if args.workload == "serving":
            bench_serving(args, rank, world)
        elif args.workload == "adjoint":
            bench_adjoint(args, rank, world)
        elif args.workload == "sum_an":
            bench_sum_an(args, rank, world)
        elif args.workload in ("topo_hex", "points"):
            bench_points(args, rank, world)
        else:
            bench_gf(args, rank, world)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
