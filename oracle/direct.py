"""ctypes wrapper of the FP64 C oracle (``gf_oracle.c``).

TEST INFRASTRUCTURE ONLY (see the package docstring).  The shared object is
compiled with gcc from the single C file next to this module; ``build()`` is
idempotent and rebuilds when the source is newer than the library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gf_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libgf_oracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no FMA contraction)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, i32, dbl = ctypes.c_long, ctypes.c_int, ctypes.c_double
            lib.gfo_forward.argtypes = [i64, i64, i64, _dp, _dp, i32, _dp, _dp,
                                        _dp, i32, _dp, i64, dbl, _dp, i32]
            lib.gfo_forward.restype = i32
            lib.gfo_adjoint.argtypes = [i64, i64, i64, _dp, _dp, i32, _dp, _dp,
                                        _dp, i64, _dp, i32, i32, dbl, _dp, i32]
            lib.gfo_adjoint.restype = i32
            lib.gfo_adjoint_subset.argtypes = [i64, i64, i64, _dp, _dp, i32, _dp, _dp, _dp, i64, _dp, i32, i32,
                                               dbl, ctypes.POINTER(ctypes.c_long), i64, _dp, i32]
            lib.gfo_adjoint_subset.restype = i32
            lib.gfo_prism_gz.argtypes = [_dp, _dp, dbl, dbl, _dp]
            lib.gfo_prism_gz.restype = dbl
            lib.gfo_prism_gz_many.argtypes = [_dp, _dp, dbl, dbl, _dp, i64, _dp, i32]
            lib.gfo_prism_gz_many.restype = None
            lib.gfo_prism_norms.argtypes = [_dp, _dp, dbl, dbl, _dp, _dp, i64, i64,
                                            i32, _dp, _dp, _dp, i32]
            lib.gfo_prism_norms.restype = None
            lib.gfo_prism_g_many.argtypes = [_dp, _dp, dbl, dbl, _dp, i64, _dp, i32]
            lib.gfo_prism_g_many.restype = None
            lib.gfo_forward_analytic.argtypes = [i64, i64, i64, _dp, _dp, _dp, i32, _dp, i64, dbl, _dp, i32]
            lib.gfo_forward_analytic.restype = i32
            lib.gfo_adjoint_analytic.argtypes = [i64, i64, i64, _dp, _dp, _dp, i64, _dp, i32, i32, dbl, _dp, i32]
            lib.gfo_adjoint_analytic.restype = i32
            lib.gfo_max_threads.restype = i32
            lib.gfo_hex_sources.argtypes = [i64, _dp, i32, _dp, _dp, _dp, _dp]
            lib.gfo_hex_sources.restype = i32
            lib.gfo_forward_points.argtypes = [i64, _dp, _dp, i64, _dp, i32, _dp, i64, dbl, _dp, i32]
            lib.gfo_forward_points.restype = i32
            _lib = lib
    return _lib


def _c(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def max_threads() -> int:
    return int(_load().gfo_max_threads())


def forward(shape, origin, h, xi, w, rho, obs, G, nthreads: int = 0) -> np.ndarray:
    """Discretised Eq. 1 at the observers.

    shape  : (nx, ny, nz) voxel counts;  origin, h : (3,) lower corner, spacing
    xi, w  : (nq, 3) reference nodes in [-1, 1]^3 and (nq,) weights
    rho    : (nz, ny, nx) or (B, nz, ny, nx) densities
    obs    : (M, 3) observers
    returns g : (M, 3) or (B, M, 3)
    """
    nx, ny, nz = (int(s) for s in shape)
    rho = _c(rho)
    single = rho.ndim == 3
    rho = rho.reshape(-1, nz, ny, nx)
    B = rho.shape[0]
    obs = _c(obs).reshape(-1, 3)
    M = obs.shape[0]
    xi = _c(xi).reshape(-1, 3)
    w = _c(w).reshape(-1)
    out = np.zeros((B, M, 3), dtype=np.float64)
    rc = _load().gfo_forward(nx, ny, nz, _p(_c(origin)), _p(_c(h)), xi.shape[0],
                             _p(xi), _p(w), _p(rho), B, _p(obs), M, float(G),
                             _p(out), int(nthreads))
    if rc != 0:
        raise ValueError("gfo_forward: bad arguments")
    return out[0] if single else out


def adjoint(shape, origin, h, xi, w, obs, r, G, ncomp: int = 1,
            nthreads: int = 0) -> np.ndarray:
    """Transpose of :func:`forward`.

    r : weights on the outputs; ncomp = 1 weights g_z only and r is (M,) or
        (B, M); ncomp = 3 weights the full vector and r is (M, 3) or (B, M, 3).
    returns grad : (nz, ny, nx) or (B, nz, ny, nx)
    """
    nx, ny, nz = (int(s) for s in shape)
    obs = _c(obs).reshape(-1, 3)
    M = obs.shape[0]
    r = _c(r)
    if ncomp == 1:
        single = r.ndim == 1
        r = r.reshape(-1, M)
    elif ncomp == 3:
        single = r.ndim == 2
        r = r.reshape(-1, M, 3)
    else:
        raise ValueError("ncomp must be 1 or 3")
    B = r.shape[0]
    xi = _c(xi).reshape(-1, 3)
    w = _c(w).reshape(-1)
    out = np.zeros((B, nz, ny, nx), dtype=np.float64)
    rc = _load().gfo_adjoint(nx, ny, nz, _p(_c(origin)), _p(_c(h)), xi.shape[0],
                             _p(xi), _p(w), _p(obs), M, _p(_c(r)), ncomp, B,
                             float(G), _p(out), int(nthreads))
    if rc != 0:
        raise ValueError("gfo_adjoint: bad arguments")
    return out[0] if single else out


def adjoint_subset(shape, origin, h, xi, w, obs, r, G, vox, ncomp: int = 1,
                   nthreads: int = 0) -> np.ndarray:
    """:func:`adjoint` evaluated only at the voxels with linear indices
    `vox` (into [nz][ny][nx]); returns (B, len(vox)) or (len(vox),)."""
    nx, ny, nz = (int(s) for s in shape)
    obs = _c(obs).reshape(-1, 3)
    M = obs.shape[0]
    r = _c(r)
    if ncomp == 1:
        single = r.ndim == 1
        r = r.reshape(-1, M)
    else:
        single = r.ndim == 2
        r = r.reshape(-1, M, 3)
    B = r.shape[0]
    vox = np.ascontiguousarray(vox, dtype=np.int64)
    xi = _c(xi).reshape(-1, 3)
    w = _c(w).reshape(-1)
    out = np.zeros((B, vox.size), dtype=np.float64)
    rc = _load().gfo_adjoint_subset(nx, ny, nz, _p(_c(origin)), _p(_c(h)), xi.shape[0], _p(xi), _p(w),
                                    _p(obs), M, _p(_c(r)), ncomp, B, float(G),
                                    vox.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), vox.size,
                                    _p(out), int(nthreads))
    if rc != 0:
        raise ValueError("gfo_adjoint_subset: bad arguments")
    return out[0] if single else out


def prism_gz(lo, hi, rho, G, pts, nthreads: int = 0) -> np.ndarray:
    """Closed-form g_z of the prism [lo, hi] with density rho at pts (n, 3)."""
    pts = _c(pts).reshape(-1, 3)
    out = np.zeros(pts.shape[0], dtype=np.float64)
    _load().gfo_prism_gz_many(_p(_c(lo)), _p(_c(hi)), float(rho), float(G),
                              _p(pts), pts.shape[0], _p(out), int(nthreads))
    return out


def prism_g(lo, hi, rho, G, pts, nthreads: int = 0) -> np.ndarray:
    """Closed-form field g (all three components) of the prism [lo, hi]
    with density rho at pts (n, 3); returns (n, 3)."""
    pts = _c(pts).reshape(-1, 3)
    out = np.zeros((pts.shape[0], 3), dtype=np.float64)
    _load().gfo_prism_g_many(_p(_c(lo)), _p(_c(hi)), float(rho), float(G),
                             _p(pts), pts.shape[0], _p(out), int(nthreads))
    return out


def forward_analytic(shape, origin, h, rho, obs, G, nthreads: int = 0) -> np.ndarray:
    """SUM-AN: the exact field of the piecewise-constant density, each voxel
    integrated in closed form.  Same shapes as :func:`forward` (no
    quadrature rule)."""
    nx, ny, nz = (int(s) for s in shape)
    rho = _c(rho)
    single = rho.ndim == 3
    rho = rho.reshape(-1, nz, ny, nx)
    B = rho.shape[0]
    obs = _c(obs).reshape(-1, 3)
    M = obs.shape[0]
    out = np.zeros((B, M, 3), dtype=np.float64)
    rc = _load().gfo_forward_analytic(nx, ny, nz, _p(_c(origin)), _p(_c(h)), _p(rho), B,
                                      _p(obs), M, float(G), _p(out), int(nthreads))
    if rc != 0:
        raise ValueError("gfo_forward_analytic: bad arguments")
    return out[0] if single else out


def adjoint_analytic(shape, origin, h, obs, r, G, ncomp: int = 1, nthreads: int = 0) -> np.ndarray:
    """Transpose of :func:`forward_analytic`; same shapes as :func:`adjoint`."""
    nx, ny, nz = (int(s) for s in shape)
    obs = _c(obs).reshape(-1, 3)
    M = obs.shape[0]
    r = _c(r)
    if ncomp == 1:
        single = r.ndim == 1
        r = r.reshape(-1, M)
    elif ncomp == 3:
        single = r.ndim == 2
        r = r.reshape(-1, M, 3)
    else:
        raise ValueError("ncomp must be 1 or 3")
    B = r.shape[0]
    out = np.zeros((B, nz, ny, nx), dtype=np.float64)
    rc = _load().gfo_adjoint_analytic(nx, ny, nz, _p(_c(origin)), _p(_c(h)), _p(obs), M, _p(_c(r)), ncomp, B,
                                      float(G), _p(out), int(nthreads))
    if rc != 0:
        raise ValueError("gfo_adjoint_analytic: bad arguments")
    return out[0] if single else out


def prism_norms(plo, phi, rho, G, dlo, dhi, Mbar, m, ngauss=4, nthreads=0):
    """Appendix A: (||g_z||_1, ||g_z||_2, max|g_z|) of the analytic prism
    field over the domain [dlo, dhi], using an ngauss-point Gauss-Legendre
    rule per axis on m^3 sub-cells of each of the Mbar^3 cells."""
    gx, gw = np.polynomial.legendre.leggauss(int(ngauss))
    out = np.zeros(3, dtype=np.float64)
    _load().gfo_prism_norms(_p(_c(plo)), _p(_c(phi)), float(rho), float(G),
                            _p(_c(dlo)), _p(_c(dhi)), int(Mbar), int(m), int(ngauss),
                            _p(_c(gx)), _p(_c(gw)), _p(out), int(nthreads))
    return out


def hex_sources(verts, xi, w):
    """Quadrature points and volume weights of deformed hexahedral cells
    (trilinear maps of the reference cube, Sec. 2.1 general SUM-G1).

    verts : (ncell, 8, 3) corners, corner a = i + 2 j + 4 k at reference
            signs (2i - 1, 2j - 1, 2k - 1)
    xi, w : (nq, 3) reference nodes in [-1, 1]^3, (nq,) weights
    returns x : (ncell * nq, 3), a : (ncell * nq,)  (source s = c * nq + q)
    """
    verts = _c(verts).reshape(-1, 8, 3)
    xi = _c(xi).reshape(-1, 3)
    w = _c(w).reshape(-1)
    n = verts.shape[0] * xi.shape[0]
    x = np.zeros((n, 3), dtype=np.float64)
    a = np.zeros(n, dtype=np.float64)
    rc = _load().gfo_hex_sources(verts.shape[0], _p(verts), xi.shape[0], _p(xi), _p(w), _p(x), _p(a))
    if rc != 0:
        raise ValueError("gfo_hex_sources: bad arguments")
    return x, a


def forward_points(x, a, per_cell, rho, obs, G, nthreads: int = 0) -> np.ndarray:
    """Field of weighted point sources: g(r) = G sum_s rho_{s // per_cell}
    a_s (r - x_s) / |r - x_s|^3.

    x : (S, 3),  a : (S,),  rho : (ncell,) or (B, ncell) with ncell = S / per_cell
    returns g : (M, 3) or (B, M, 3)
    """
    x = _c(x).reshape(-1, 3)
    a = _c(a).reshape(-1)
    S = x.shape[0]
    ncell = S // int(per_cell)
    rho = _c(rho)
    single = rho.ndim == 1
    rho = rho.reshape(-1, ncell)
    B = rho.shape[0]
    obs = _c(obs).reshape(-1, 3)
    M = obs.shape[0]
    out = np.zeros((B, M, 3), dtype=np.float64)
    rc = _load().gfo_forward_points(S, _p(x), _p(a), int(per_cell), _p(rho), B, _p(obs), M, float(G), _p(out),
                                    int(nthreads))
    if rc != 0:
        raise ValueError("gfo_forward_points: bad arguments")
    return out[0] if single else out


def forward_hex(verts, xi, w, rho, obs, G, nthreads: int = 0) -> np.ndarray:
    """Discretised Eq. 1 over deformed hexahedral cells of constant density:
    :func:`hex_sources` then :func:`forward_points`."""
    x, a = hex_sources(verts, xi, w)
    return forward_points(x, a, np.asarray(xi).reshape(-1, 3).shape[0], rho, obs, G, nthreads)
