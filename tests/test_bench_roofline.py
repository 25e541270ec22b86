"""The roofline object of bench.py's JSON line, on CPU: the dominant stage
picks the bound and the peak (FP16 dense = the measured BF16 burst for the
tensor-core M2L; 152 SMs x 128 lanes x 2 x clock for the FP32 evaluation;
FP64 nominal for the plain path), `achieved` is the algorithmic work over the
stage time, and the ncu traffic is reported only while the kernel's source
matches the captured one."""
import argparse
import os
import sys
from types import SimpleNamespace

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

INFO = SimpleNamespace(K=121, near_pairs=596922624, m2l_pairs=1125279)
PEAKS = {"bf16_tflops": 1870.7, "sm_max_mhz": 2070.0}
WORKLOAD = "layered_scale_464^3"


def args(precision="mixed", p=10, m2l="auto"):
    return argparse.Namespace(precision=precision, p=p, m2l=m2l)


def captured(stage):
    """The table's traffic while the kernel's source still has the captured
    SHA-1, else None."""
    nbytes, srcs, sha = bench.NCU_TRAFFIC[(stage, WORKLOAD, 10)]
    return nbytes if bench.sources_sha1(srcs) == sha else None


def test_evaluation_dominant():
    r = bench.fmm_roofline({"eval": 1.30, "m2l": 1.25}, INFO, args(), PEAKS, WORKLOAD)
    assert r["stage"] == "eval" and r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["peak"] == pytest.approx(152 * 128 * 2 * 2070e6 / 1e12)
    assert r["achieved"] == pytest.approx(20.0 * INFO.near_pairs / 1.30e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["traffic"] == captured("eval")


def test_tensor_core_m2l_dominant():
    r = bench.fmm_roofline({"eval": 1.0, "m2l": 1.25}, INFO, args(), PEAKS, WORKLOAD)
    assert r["stage"] == "m2l" and r["bound"] == "tensor"
    assert r["peak"] == pytest.approx(1870.7 * bench.F16_PER_BF16)
    assert r["achieved"] == pytest.approx(2.0 * INFO.K * INFO.K * INFO.m2l_pairs / 1.25e-3 / 1e12)
    assert r["traffic"] == captured("m2l")


def test_traffic_only_for_the_captured_configuration():
    assert bench.fmm_roofline({"eval": 1.3, "m2l": 1.0}, INFO, args(p=8), PEAKS, WORKLOAD)["traffic"] is None
    assert bench.fmm_roofline({"eval": 1.3, "m2l": 1.0}, INFO, args(m2l="simt"), PEAKS, WORKLOAD)["traffic"] is None
    assert bench.fmm_roofline({"eval": 1.3, "m2l": 1.0}, INFO, args(), PEAKS, "other")["traffic"] is None


def test_traffic_dropped_when_the_source_changes(monkeypatch):
    key = ("eval", WORKLOAD, 10)
    nbytes, src, _ = bench.NCU_TRAFFIC[key]
    monkeypatch.setitem(bench.NCU_TRAFFIC, key, (nbytes, src, "0" * 40))
    assert bench.fmm_roofline({"eval": 1.3, "m2l": 1.0}, INFO, args(), PEAKS, WORKLOAD)["traffic"] is None


def test_evaluation_reports_its_sfu_share():
    """One reciprocal square root per near pair: the SFU fraction against
    152 SMs x 16 per clock, and against the measured MUFU probe."""
    r = bench.fmm_roofline({"eval": 1.30, "m2l": 1.25}, INFO, args(), PEAKS, WORKLOAD)
    rate = INFO.near_pairs / 1.30e-3
    assert r["sfu_frac"] == pytest.approx(rate / (152 * 16 * 2070e6))
    assert r["sfu_frac_of_probe"] == pytest.approx(rate / bench.MUFU_RSQRT_PROBE)


def scale_info():
    """A 7-level tree over a 116^3 block of leaves (464^3 voxels, 4^3 per
    leaf): the source block of level l spans ceil(116 / 2^(7-l)) boxes."""
    L = 7
    lo = [[0, 0, 0] for _ in range(24)]
    hi = [[0, 0, 0] for _ in range(24)]
    for l in range(2, L + 1):
        n = -(-116 // (1 << (L - l)))
        hi[l] = [n - 1] * 3
    return SimpleNamespace(K=144, L=L, near_pairs=596922624, m2l_pairs=1125279, src_lo=lo, src_hi=hi)


def test_hbm_bound_upward_sweep_dominant():
    """When the P2M (or M2M) stage dominates, the roofline is HBM-bound:
    densities read once plus the level L-1 expansions (made straight from
    them) written once; children read once plus parents written once from
    level L-1 up; in GB/s against the measured copy rate."""
    info = scale_info()
    peaks = dict(PEAKS, hbm_gbs=6700.0)
    r = bench.fmm_roofline({"eval": 0.4, "m2l": 0.5, "p2m": 0.8, "m2m": 0.7}, info, args(p=11), peaks,
                           "layered_scale_464^3", nvox=464 ** 3, rho_bytes=4)
    assert r["stage"] == "p2m" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    want = 464 ** 3 * 4 + 58 ** 3 * 144 * 4      # densities once, level-6 expansions once
    assert r["achieved"] == pytest.approx(want / 0.8e-3 / 1e9)
    assert r["peak"] == 6700.0 and r["frac"] == pytest.approx(r["achieved"] / 6700.0)
    r = bench.fmm_roofline({"eval": 0.4, "m2l": 0.5, "p2m": 0.6, "m2m": 0.7}, info, args(p=11), peaks,
                           "layered_scale_464^3", nvox=464 ** 3, rho_bytes=4)
    ns = {l: (-(-116 // (1 << (7 - l)))) ** 3 for l in range(2, 8)}
    want = sum(ns[l] for l in range(3, 7)) * 144 * 4 + sum(ns[l] for l in range(2, 6)) * 144 * 4
    assert r["stage"] == "m2m" and r["achieved"] == pytest.approx(want / 0.7e-3 / 1e9)


def test_plain_fp64_path_against_the_fp64_rate():
    r = bench.fmm_roofline({"eval": 20.0, "m2l": 989.0}, INFO, args("fp64", 14, "auto"), PEAKS, WORKLOAD)
    assert r["stage"] == "m2l" and r["bound"] == "alu"
    assert r["peak"] == pytest.approx(bench.FP64_TFLOPS_NOMINAL)
    assert r["traffic"] is None


def test_point_p2m_dominant():
    """Point sources: the P2M is ALU-bound at 10 flops per complex harmonic,
    (p+1)(p+2)/2 harmonics per point, against the FP32 rate."""
    info = scale_info()
    r = bench.fmm_roofline({"eval": 0.3, "m2l": 0.8, "p2m": 3.0, "m2m": 0.6}, info, args(p=12), PEAKS,
                           "topo_hex_256x256x64", n_points=33554432)
    assert r["stage"] == "p2m" and r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(10.0 * 91 * 33554432 / 3.0e-3 / 1e12)
    assert r["peak"] == pytest.approx(152 * 128 * 2 * 2070e6 / 1e12)
    r = bench.fmm_roofline({"eval": 0.3, "m2l": 0.8, "p2m": 0.5, "m2m": 0.9}, info, args(p=12), PEAKS,
                           "topo_hex_256x256x64", n_points=33554432)
    assert r["stage"] == "m2m" and r["bound"] == "hbm"


def test_tensor_pipe_fraction_counts_the_three_products():
    """The M2L's algorithmic fraction is capped at 1/3 by the high/low split;
    pipe_frac reports the tensor pipe's share (three products each)."""
    r = bench.fmm_roofline({"eval": 0.3, "m2l": 1.25}, INFO, args(), PEAKS, WORKLOAD)
    assert r["stage"] == "m2l" and r["bound"] == "tensor"
    assert r["pipe_frac"] == pytest.approx(3 * r["frac"])
