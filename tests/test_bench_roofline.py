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

INFO = SimpleNamespace(K=169, near_pairs=3691610112, m2l_pairs=6039504)
PEAKS = {"bf16_tflops": 1870.7, "sm_max_mhz": 2070.0}
WORKLOAD = "grf_volume_128^3"


def args(precision="mixed", p=12, m2l="auto"):
    return argparse.Namespace(precision=precision, p=p, m2l=m2l)


def captured(stage):
    """The table's traffic while the kernel's source still has the captured
    SHA-1, else None."""
    import hashlib
    nbytes, src, sha = bench.NCU_TRAFFIC[(stage, WORKLOAD, 12)]
    with open(os.path.join(ROOT, src), "rb") as f:
        return nbytes if hashlib.sha1(f.read()).hexdigest() == sha else None


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
    assert r["achieved"] == pytest.approx(2.0 * 169 * 169 * INFO.m2l_pairs / 1.25e-3 / 1e12)
    assert r["traffic"] == captured("m2l")


def test_traffic_only_for_the_captured_configuration():
    assert bench.fmm_roofline({"eval": 1.3, "m2l": 1.0}, INFO, args(p=8), PEAKS, WORKLOAD)["traffic"] is None
    assert bench.fmm_roofline({"eval": 1.3, "m2l": 1.0}, INFO, args(m2l="simt"), PEAKS, WORKLOAD)["traffic"] is None
    assert bench.fmm_roofline({"eval": 1.3, "m2l": 1.0}, INFO, args(), PEAKS, "other")["traffic"] is None


def test_traffic_dropped_when_the_source_changes(monkeypatch):
    key = ("eval", WORKLOAD, 12)
    nbytes, src, _ = bench.NCU_TRAFFIC[key]
    monkeypatch.setitem(bench.NCU_TRAFFIC, key, (nbytes, src, "0" * 40))
    assert bench.fmm_roofline({"eval": 1.3, "m2l": 1.0}, INFO, args(), PEAKS, WORKLOAD)["traffic"] is None


def test_plain_fp64_path_against_the_fp64_rate():
    r = bench.fmm_roofline({"eval": 20.0, "m2l": 989.0}, INFO, args("fp64", 14, "auto"), PEAKS, WORKLOAD)
    assert r["stage"] == "m2l" and r["bound"] == "alu"
    assert r["peak"] == pytest.approx(bench.FP64_TFLOPS_NOMINAL)
    assert r["traffic"] is None
