"""The oracle's pins catch plausible mistakes.  Each case plants one mistake in
a copy of oracle/gf_oracle.c (a flipped sign, a dropped normalisation, a
transposed index, a wrong axis, a wrong corner sign, a wrong special axis;
for deformed cells and point sources a wrong reference-cube volume, a wrong
shape-function derivative, a wrong density index), builds the copy, and
checks that a pin which the real oracle passes fails on it: the
exact-arithmetic brute force, the closed-form prism field the quadrature
sums must converge to, Table 10's vertical formula, the axis relabelling of
that formula, the exact volume of trilinear cells, Gauss's law and the voxel
sum that undeformed cells must reproduce."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import direct
from paper_1107_5951_gb300 import workloads as wl
from test_oracle_pins import _exact_sum

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "gf_oracle.c")
_dp = ctypes.POINTER(ctypes.c_double)

MUTATIONS = {
    "separation_sign": ("const double d0 = r0 - x[0], d1 = r1 - x[1],", "const double d0 = x[0] - r0, d1 = r1 - x[1],"),
    "weight_not_normalised": ("                            const double wq = w[q] / wsum;",
                              "                            const double wq = w[q];"),
    "density_index_transposed": ("const long v = (k * ny + j) * nx + i;\n                        for (int q",
                                 "const long v = (k * ny + i) * nx + j;\n                        for (int q"),
    "node_offset_wrong_axis": ("x[0] = c0 + 0.5 * h[0] * xi_q[0];", "x[0] = c0 + 0.5 * h[1] * xi_q[0];"),
    "prism_corner_sign": ("const double s = ((a + b + c) & 1) ? 1.0 : -1.0;\n                acc += s * prism_corner(u, v, w);",
                          "const double s = ((a + b) & 1) ? 1.0 : -1.0;\n                acc += s * prism_corner(u, v, w);"),
    "gx_wrong_special_axis": ("ax += s * prism_corner(v, w, u);", "ax += s * prism_corner(u, w, v);"),
}

POINT_MUTATIONS = {
    "hex_reference_volume": ("a[s] = 8.0 * (w[q] / wsum) * fabs(det);", "a[s] = 4.0 * (w[q] / wsum) * fabs(det);"),
    "hex_shape_derivative": ("f0 * f1 * s2 / 8.0};", "f0 * f1 * s1 / 8.0};"),
    "points_density_index": ("const long c = s / per_cell;", "const long c = s % ncell;"),
}


def _build(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, name
    path = tmp_path / (name + ".c")
    path.write_text(src.replace(old, new))
    lib = tmp_path / (name + ".so")
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", str(path),
                    "-o", str(lib), "-lm"], check=True)
    L = ctypes.CDLL(str(lib))
    i64, i32, dbl = ctypes.c_long, ctypes.c_int, ctypes.c_double
    L.gfo_forward.argtypes = [i64, i64, i64, _dp, _dp, i32, _dp, _dp, _dp, i32, _dp, i64, dbl, _dp, i32]
    L.gfo_prism_gz_many.argtypes = [_dp, _dp, dbl, dbl, _dp, i64, _dp, i32]
    L.gfo_prism_g_many.argtypes = [_dp, _dp, dbl, dbl, _dp, i64, _dp, i32]
    L.gfo_hex_sources.argtypes = [i64, _dp, i32, _dp, _dp, _dp, _dp]
    L.gfo_forward_points.argtypes = [i64, _dp, _dp, i64, _dp, i32, _dp, i64, dbl, _dp, i32]
    return L


def _c(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a):
    return a.ctypes.data_as(_dp)


# nthreads = 0 everywhere: the copies share the process's OpenMP runtime, and
# setting a thread count there would also slow the real oracle in later tests
def _forward(L, shape, origin, h, xi, w, rho, obs):
    nx, ny, nz = shape
    rho, obs, xi, w = _c(rho), _c(obs).reshape(-1, 3), _c(xi).reshape(-1, 3), _c(w)
    out = np.zeros((1, obs.shape[0], 3))
    L.gfo_forward(nx, ny, nz, _p(_c(origin)), _p(_c(h)), xi.shape[0], _p(xi), _p(w), _p(rho), 1, _p(obs),
                  obs.shape[0], 1.0, _p(out), 0)
    return out[0]


def _pins_fail(L):
    """True when at least one pin rejects the library L."""
    # (1) a 2x2x2-Gauss sum over a refined uniform prism must approach the
    # closed form of the real oracle (fourth order): 8^3 cells, 1e-5
    lo, hi = np.array([0.0, 0.0, -1.0]), np.array([1.0, 1.0, 0.0])
    obs = np.array([[1.7, 1.3, 0.8], [-0.6, 0.4, 0.9]])
    xi, w = wl.gauss_rule(2)
    s = 8
    g = _forward(L, (s, s, s), lo, (1.0 / s,) * 3, xi, w, np.ones((s, s, s)), obs)
    exact = direct.prism_g(lo, hi, 1.0, 1.0, obs)
    if np.max(np.abs(g - exact)) > 1e-5 * np.max(np.abs(exact)):
        return True
    # (2) random densities on an anisotropic grid against the exact-arithmetic
    # brute force (to a few ulp of the sum of magnitudes)
    wk = wl.random_small(4, n=(2, 2, 2), npts=2, n_obs=6, h=(0.75, 1.25, 1.0), origin=(-1.0, 0.5, -2.0))
    g = _forward(L, wk.grid.n, wk.grid.origin, wk.grid.h, wk.xi, wk.w, wk.rho, wk.obs)
    exact, mag = _exact_sum(wk.grid.n, wk.grid.origin, wk.grid.h, wk.xi, wk.w, wk.rho, wk.obs)
    if np.any(np.abs(g - exact) > 4e-16 * mag + 1e-300):
        return True
    # (3) the closed-form prism field: its g_z against the Table-10-pinned
    # formula of the real oracle, g_x against g_z of the relabelled prism
    a, b = np.array([-0.5, 0.2, -1.0]), np.array([0.7, 1.1, 0.3])
    pts = np.array([[1.5, 0.4, 2.0], [-2.0, 1.0, -0.5], [0.1, 0.5, -0.2]])
    gz = np.zeros(3)
    L.gfo_prism_gz_many(_p(_c(a)), _p(_c(b)), 1.0, 1.0, _p(_c(pts)), 3, _p(gz), 0)
    if np.max(np.abs(gz - direct.prism_gz(a, b, 1.0, 1.0, pts))) > 1e-13:
        return True
    gv = np.zeros((3, 3))
    L.gfo_prism_g_many(_p(_c(a)), _p(_c(b)), 1.0, 1.0, _p(_c(pts)), 3, _p(gv), 0)
    perm = [1, 2, 0]
    gx_rot = direct.prism_gz(a[perm], b[perm], 1.0, 1.0, pts[:, perm])
    return np.max(np.abs(gv[:, 0] - gx_rot)) > 1e-13


@pytest.fixture(scope="module")
def gcc():
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")


def test_the_real_oracle_passes(gcc, tmp_path):
    same = MUTATIONS["separation_sign"][0]
    L = _build(tmp_path, "unchanged", same, same)
    assert not _pins_fail(L)


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_a_planted_mistake_fails_a_pin(gcc, tmp_path, name):
    old, new = MUTATIONS[name]
    assert _pins_fail(_build(tmp_path, name, old, new)), name


def _hex_sources(L, verts, xi, w):
    verts, xi, w = _c(verts), _c(xi).reshape(-1, 3), _c(w)
    n = verts.shape[0] * xi.shape[0]
    x, a = np.zeros((n, 3)), np.zeros(n)
    L.gfo_hex_sources(verts.shape[0], _p(verts), xi.shape[0], _p(xi), _p(w), _p(x), _p(a))
    return x, a


def _points(L, x, a, per_cell, rho, obs):
    x, a, rho, obs = _c(x), _c(a), _c(rho), _c(obs).reshape(-1, 3)
    out = np.zeros((1, obs.shape[0], 3))
    L.gfo_forward_points(x.shape[0], _p(x), _p(a), per_cell, _p(rho), 1, _p(obs), obs.shape[0], 1.0, _p(out), 0)
    return out[0]


def _point_pins_fail(L):
    """True when a pin of the deformed-cell / point-source sums rejects L."""
    xi, w = wl.gauss_rule(2)
    # (1) warped cells tiling a 3 x 2 x 1 brick hold its volume exactly
    _, a = _hex_sources(L, wl.hex_brick_mesh((3, 2, 2), (0.0, 0.0, 0.0), (3.0, 2.0, 1.0), warp=0.1), xi, w)
    if abs(a.sum() - 6.0) > 1e-12:
        return True
    # (2) undeformed cells reproduce the real oracle's voxel sum
    rng = np.random.default_rng(3)
    n, lo, h = (3, 2, 2), np.array([0.0, 0.0, 0.0]), np.array([1.0, 1.0, 1.0])
    rho = rng.normal(size=(2, 2, 3))
    obs = rng.uniform(-2, 4, size=(10, 3))
    x, a = _hex_sources(L, wl.hex_brick_mesh(n, lo, lo + np.array(n) * h), xi, w)
    got = _points(L, x, a, 8, rho.ravel(), obs)
    want = direct.forward(n, lo, h, xi, w, rho, obs, 1.0)
    return np.linalg.norm(got - want) > 1e-13 * np.linalg.norm(want)


def test_the_real_oracle_passes_the_point_pins(gcc, tmp_path):
    same = POINT_MUTATIONS["hex_reference_volume"][0]
    assert not _point_pins_fail(_build(tmp_path, "unchanged_points", same, same))


@pytest.mark.parametrize("name", sorted(POINT_MUTATIONS))
def test_a_planted_point_mistake_fails_a_pin(gcc, tmp_path, name):
    old, new = POINT_MUTATIONS[name]
    assert _point_pins_fail(_build(tmp_path, name, old, new)), name
