"""Host model of a SUM-AN near field (tests/emu/sum_an_emu.cpp): constant-
density voxels integrated in closed form (Sec. 2.1) and regrouped onto the
voxel-corner lattice, one corner function per lattice point weighted by the
signed sum of the densities of the voxels sharing it.  Against the oracle's
per-voxel SUM-AN sum, shell by shell (Chebyshev distance in voxels from the
observer's voxel) over the 12^3 voxels of a leaf's 27 neighbour leaves
(leaves of 4^3 voxels), this pins the design a GPU kernel follows:

* the regrouping is exact (FP64: agreement to rounding);
* the closed form in FP32 stays within 1e-5 of the total field on the
  shells 0..2, its cancellation growing like (d/h)^3 beyond;
* Gauss rules fail near the observer (the integrand is singular in its own
  voxel) and reach the FP32 floor from shell 3 with 3^3 points;
* one point per voxel suffices from shell 3 once the l = 4 (hexadecapole)
  term of a uniform cube, -(7/192) G m h^4 (sum R_i^4 - 3/5 R^4) / R^9 in
  the potential, is added (a cube has no quadrupole), so the design --
  closed form on shells 0..2, corrected midpoint beyond -- stays within the
  mixed-precision bar of 1e-5.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import direct

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NB, SHELLS = 12, 6
LAT64, LAT32, G2, G3, G4, MIDHEX = range(6)


@pytest.fixture(scope="module")
def emu(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("sum_an")
    exe = str(d / "sum_an_emu")
    subprocess.run([gxx, "-O2", "-std=c++17", "-o", exe, os.path.join(ROOT, "tests", "emu", "sum_an_emu.cpp")],
                   check=True)
    return exe, d


def _run(emu, rho, obs):
    exe, d = emu
    inp, out = str(d / "in.bin"), str(d / "out.bin")
    np.concatenate([[NB, len(obs)], rho.ravel(), obs.ravel()]).astype(np.float64).tofile(inp)
    subprocess.run([exe, inp, out], check=True)
    return np.fromfile(out).reshape(6, SHELLS, len(obs), 3)


def _oracle_by_shell(rho, obs):
    kk, jj, ii = np.meshgrid(np.arange(NB), np.arange(NB), np.arange(NB), indexing="ij")
    ref = np.zeros((SHELLS, len(obs), 3))
    for j, o in enumerate(obs):
        v = np.floor(o).astype(int)
        d = np.minimum(np.maximum(np.maximum(abs(ii - v[0]), abs(jj - v[1])), abs(kk - v[2])), SHELLS - 1)
        for s in range(SHELLS):
            r = np.where(d == s, rho, 0.0)
            if np.any(r != 0):
                ref[s, j] = direct.forward_analytic((NB,) * 3, (0.0,) * 3, (1.0,) * 3, r, o[None], 1.0)[0]
    return ref


@pytest.mark.parametrize("kind", ["positive", "zero_mean"])
def test_corner_lattice_design(emu, kind):
    rng = np.random.default_rng(17 if kind == "positive" else 18)
    rho = rng.uniform(1.0, 3.0, size=(NB,) * 3) if kind == "positive" else rng.normal(size=(NB,) * 3)
    obs = rng.uniform(4.0, 8.0, size=(10, 3))       # inside the central leaf
    obs[0] = [6.0, 6.0, 6.0]                         # a corner shared by eight voxels
    obs[1] = [5.5, 6.0, 6.25]                        # on a face between two voxels
    g = _run(emu, rho, obs)
    ref = _oracle_by_shell(rho, obs)
    scale = np.linalg.norm(ref.sum(0), axis=1)
    err = (np.linalg.norm(g - ref[None], axis=3) / scale).max(axis=2)      # [method, shell]
    assert err[LAT64].max() <= 1e-12
    assert np.linalg.norm(g[LAT64].sum(0) - ref.sum(0), axis=1).max() <= 1e-12 * scale.min()
    assert err[LAT32, :3].max() <= 1e-5
    assert err[LAT32, 5] > err[LAT32, 0]              # cancellation grows with distance
    assert err[G2, 0] > 0.1 and err[G4, 1] > 1e-2     # quadrature fails next to the observer
    assert err[G3, 3:].max() <= 2e-6
    # the midpoint rule plus a cube's l = 4 term: error falls like (h/d)^6
    assert err[MIDHEX, 3:].max() <= 5e-6 and err[MIDHEX, 4:].max() <= 1e-6
    # the design: closed form on shells 0..2, corrected midpoint beyond
    design = g[LAT32, :3].sum(0) + g[MIDHEX, 3:].sum(0)
    assert (np.linalg.norm(design - ref.sum(0), axis=1) / scale).max() <= 1e-5
