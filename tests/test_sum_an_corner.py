"""The closed-form (SUM-AN) arithmetic of gf_sum_an.cuh, compiled for the host
by nvcc into tests/emu/sum_an_corner_host.cu, against the oracle:

* the corner function (an_corner, an_corner_z), summed with the corner signs
  over a prism's eight corners, gives the prism's closed-form field;
  observers inside and on faces, edges and corners agree to rounding,
  outside the eight-term sum cancels like (d / size)^3;
* the FMM form's near field (an_near_block: closed form on the voxels
  within Chebyshev distance 2 (FP32) or 3 (FP64) of the observer's voxel,
  midpoint plus a cube's l = 4 term beyond) over the 12^3 voxels of a
  leaf's 27 neighbours (leaves of 4^3 voxels) against the oracle's SUM-AN
  sum of the same voxels: the mixed-precision bar in FP32, the FP64 FMM
  bar in FP64."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import direct

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    d = tmp_path_factory.mktemp("corner")
    exe = str(d / "sum_an_corner_host")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17",
                    "-I" + os.path.join(ROOT, "include"), "-I" + os.path.join(ROOT, "paper_1107_5951_gb300", "csrc"),
                    "--expt-relaxed-constexpr", "-o", exe, os.path.join(ROOT, "tests", "emu", "sum_an_corner_host.cu")],
                   check=True)
    return exe, d


def test_corner_function_matches_the_oracle_prism_field(harness):
    exe, d = harness
    rng = np.random.default_rng(3)
    n = 400
    lo = rng.uniform(-3.0, 3.0, size=(n, 3))
    hi = lo + rng.uniform(0.3, 2.5, size=(n, 3))
    inside = rng.random(n) < 0.3
    r = np.where(inside[:, None], rng.uniform(lo, hi), rng.uniform(-6.0, 6.0, size=(n, 3)))
    r[0] = lo[0]                                                          # a corner
    r[1] = [lo[1, 0], 0.5 * (lo[1, 1] + hi[1, 1]), hi[1, 2]]               # an edge
    r[2] = [0.3 * lo[2, 0] + 0.7 * hi[2, 0], lo[2, 1], 0.5 * (lo[2, 2] + hi[2, 2])]   # a face
    inside[:3] = True
    np.concatenate([[n], np.concatenate([lo, hi, r], 1).ravel()]).tofile(str(d / "in.bin"))
    subprocess.run([exe, str(d / "in.bin"), str(d / "out.bin")], check=True)
    out = np.fromfile(str(d / "out.bin")).reshape(n, 4)
    ref = np.concatenate([direct.prism_g(lo[i], hi[i], 1.0, 1.0, r[i:i + 1]) for i in range(n)])
    scale = np.abs(ref).max(axis=1)
    err = np.abs(out[:, :3] - ref).max(axis=1) / scale
    dist = np.linalg.norm(r - 0.5 * (lo + hi), axis=1) / np.linalg.norm(hi - lo, axis=1)
    assert err[inside].max() <= 1e-14
    assert np.all(err[~inside] <= 1e-13 * np.maximum(dist[~inside], 1.0) ** 3)
    assert np.all(np.abs(out[:, 3] - ref[:, 2]) <= 1e-13 * np.maximum(dist, 1.0) ** 3 * scale)


@pytest.mark.parametrize("kind", ["positive", "zero_mean"])
def test_near_block_meets_the_mixed_bar(harness, kind):
    exe, d = harness
    nb = 12
    rng = np.random.default_rng(17 if kind == "positive" else 18)
    rho = rng.uniform(1.0, 3.0, size=(nb,) * 3) if kind == "positive" else rng.normal(size=(nb,) * 3)
    t = rng.uniform(4.0, 8.0, size=(64, 3))        # observers in the central leaf
    t[0] = [6.0, 6.0, 6.0]                          # a corner shared by eight voxels
    t[1] = [5.5, 6.0, 6.25]                         # on a face
    t[2] = [4.0, 7.999, 5.0]                        # on the leaf's boundary
    np.concatenate([[nb, len(t)], rho.ravel(), t.ravel()]).tofile(str(d / "near_in.bin"))
    subprocess.run([exe, str(d / "near_in.bin"), str(d / "near_out.bin"), "near"], check=True)
    out = np.fromfile(str(d / "near_out.bin")).reshape(-1, 6)
    ref = direct.forward_analytic((nb,) * 3, (0.0,) * 3, (1.0,) * 3, rho, t, 1.0)
    assert np.linalg.norm(out[:, :3] - ref) / np.linalg.norm(ref) <= 5e-6
    assert np.linalg.norm(out[:, 3:] - ref) / np.linalg.norm(ref) <= 5e-7
