"""Thin Python binding of the C ABI in ``include/gf.h`` (ctypes).

Argument marshalling only: every step of the forward model runs in the CUDA
kernels of ``libgf.so``.  PyTorch supplies device memory and streams.  The
functions ``gf_plan_create``, ``gf_plan_create_points``, ``gf_hex_sources``,
``gf_forward``, ``gf_adjoint``, ``gf_plan_destroy``, ``gf_plan_check``,
``gf_plan_bytes``, ``gf_plan_get_info``, ``gf_plan_export_tree`` and ``gf_last_error`` mirror
the C entry points one to one; :class:`Plan` (voxel grids),
:class:`PointsPlan` (weighted point sources) and :func:`hex_sources` wrap
them for tensors.

There is no fallback: if ``libgf.so`` is missing or cannot be loaded, every
call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

GF_OK, GF_ERR_INVALID_ARG, GF_ERR_OOM, GF_ERR_CUDA = 0, 1, 2, 3
GF_ERR_UNSUPPORTED, GF_ERR_TIMEOUT, GF_ERR_DEVICE_CHECK, GF_ERR_BUSY = 4, 5, 6, 7
GF_MODE_DIRECT, GF_MODE_FMM = 0, 1
GF_PREC_FP64, GF_PREC_MIXED = 0, 1
GF_DTYPE_F64, GF_DTYPE_F32 = 0, 1

_STATUS_NAMES = {0: "GF_OK", 1: "GF_ERR_INVALID_ARG", 2: "GF_ERR_OOM", 3: "GF_ERR_CUDA",
                 4: "GF_ERR_UNSUPPORTED", 5: "GF_ERR_TIMEOUT", 6: "GF_ERR_DEVICE_CHECK",
                 7: "GF_ERR_BUSY"}


class GfError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (_STATUS_NAMES.get(status, str(status)), msg))
        self.status = status


class gf_grid(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64 * 3), ("origin", ctypes.c_double * 3),
                ("h", ctypes.c_double * 3)]


class gf_quad(ctypes.Structure):
    _fields_ = [("nq", ctypes.c_int32), ("xi", ctypes.POINTER(ctypes.c_double)),
                ("w", ctypes.POINTER(ctypes.c_double))]


class gf_options(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("precision", ctypes.c_int32), ("p", ctypes.c_int32),
                ("leaf_vox", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("reserved0", ctypes.c_int32), ("G", ctypes.c_double)]


class gf_plan_info(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("precision", ctypes.c_int32), ("p", ctypes.c_int32),
                ("K", ctypes.c_int32), ("L", ctypes.c_int32), ("leaf_vox", ctypes.c_int32),
                ("voxel_offset", ctypes.c_int64 * 3), ("lo", ctypes.c_double * 3),
                ("leaf_side", ctypes.c_double), ("inv_leaf_side", ctypes.c_double),
                ("n_target_boxes", ctypes.c_int64 * 24), ("src_lo", (ctypes.c_int64 * 3) * 24),
                ("src_hi", (ctypes.c_int64 * 3) * 24), ("M", ctypes.c_int64),
                ("n_sources", ctypes.c_int64), ("near_pairs", ctypes.c_int64),
                ("m2l_pairs", ctypes.c_int64), ("device_bytes", ctypes.c_size_t)]


class gf_server_options(ctypes.Structure):
    _fields_ = [("max_slots", ctypes.c_int32), ("precision", ctypes.c_int32), ("p", ctypes.c_int32),
                ("leaf_vox", ctypes.c_int32), ("use_graphs", ctypes.c_int32), ("device", ctypes.c_int32),
                ("mem_budget", ctypes.c_size_t), ("G", ctypes.c_double)]


class gf_request(ctypes.Structure):
    _fields_ = [("grid", gf_grid), ("quad", gf_quad), ("obs_host", ctypes.c_void_p), ("M", ctypes.c_int64),
                ("geometry_id", ctypes.c_uint64), ("rho_host", ctypes.c_void_p), ("rho_dtype", ctypes.c_int32),
                ("on_device", ctypes.c_int32), ("gz_host", ctypes.c_void_p), ("g_host", ctypes.c_void_p)]


class gf_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("plans_created", ctypes.c_int64), ("plans_evicted", ctypes.c_int64),
                ("graph_launches", ctypes.c_int64), ("resident_bytes", ctypes.c_size_t),
                ("mem_budget", ctypes.c_size_t), ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("mean_ms", ctypes.c_double), ("busy_s", ctypes.c_double)]


GF_NUM_STAGES = 8
STAGE_NAMES = ("densities", "p2m", "m2m", "m2l_split", "m2l", "l2l", "eval", "forward")


_lib = None
_lock = threading.Lock()
_vp = ctypes.c_void_p


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libgf.so (building it with nvcc first if it is missing or
    stale).  Raises if it cannot be built or loaded."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing and _build.is_stale():
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError("libgf.so is not built (run __graft_entry__.build())")
        lib = ctypes.CDLL(_build.LIB)
        i32, i64 = ctypes.c_int32, ctypes.c_int64
        P = ctypes.POINTER
        lib.gf_plan_create.argtypes = [P(gf_grid), P(gf_quad), _vp, i64, P(gf_options), _vp, P(_vp)]
        lib.gf_forward.argtypes = [_vp, _vp, i32, i32, _vp, _vp, _vp]
        lib.gf_adjoint.argtypes = [_vp, _vp, i32, i32, _vp, _vp]
        lib.gf_plan_destroy.argtypes = [_vp]
        lib.gf_plan_check.argtypes = [_vp, _vp]
        lib.gf_plan_bytes.argtypes = [P(gf_grid), P(gf_quad), i64, P(gf_options), P(ctypes.c_size_t)]
        lib.gf_plan_get_info.argtypes = [_vp, P(gf_plan_info)]
        lib.gf_plan_export_tree.argtypes = [_vp, i32, _vp, _vp, _vp, _vp, _vp]
        lib.gf_direct_forward_static.argtypes = [P(gf_grid), P(gf_quad), _vp, i64, _vp, i32, i32,
                                                 ctypes.c_double, _vp, _vp, _vp]
        lib.gf_direct_forward_static.restype = ctypes.c_int
        lib.gf_hex_sources.argtypes = [_vp, i64, P(gf_quad), i32, _vp, _vp, _vp]
        lib.gf_plan_create_points.argtypes = [_vp, _vp, i64, i32, _vp, i64, P(gf_options), _vp, P(_vp)]
        lib.gf_plan_set_timing.argtypes = [_vp, i32]
        lib.gf_plan_set_source_part.argtypes = [_vp, i32, i32, P(i32), P(i32)]
        lib.gf_plan_stage_times.argtypes = [_vp, P(ctypes.c_double)]
        lib.gf_server_create.argtypes = [P(gf_server_options), P(_vp)]
        lib.gf_server_submit.argtypes = [_vp, P(gf_request), P(i64)]
        lib.gf_server_wait.argtypes = [_vp, i64, ctypes.c_double, P(ctypes.c_double)]
        lib.gf_server_stats_get.argtypes = [_vp, P(gf_server_stats)]
        lib.gf_server_destroy.argtypes = [_vp]
        for name in ("gf_plan_create", "gf_hex_sources", "gf_plan_create_points", "gf_forward", "gf_adjoint", "gf_plan_destroy", "gf_plan_check",
                     "gf_plan_bytes", "gf_plan_get_info", "gf_plan_export_tree", "gf_plan_set_timing",
                     "gf_plan_stage_times", "gf_plan_set_source_part", "gf_server_create", "gf_server_submit", "gf_server_wait",
                     "gf_server_stats_get", "gf_server_destroy"):
            getattr(lib, name).restype = ctypes.c_int
        lib.gf_last_error.argtypes = []
        lib.gf_last_error.restype = ctypes.c_char_p
        lib.gf_version.restype = ctypes.c_int32
        lib.gf_launch_count.restype = ctypes.c_int64
        _lib = lib
        return lib


def gf_last_error() -> str:
    return load().gf_last_error().decode(errors="replace")


def _check(status: int):
    if status != GF_OK:
        raise GfError(status, gf_last_error())


# ------------------------------------------------------------ raw entry points
def gf_plan_create(grid: gf_grid, quad: gf_quad, obs_ptr: int, M: int, opt: gf_options,
                   stream: int = 0) -> int:
    plan = _vp()
    _check(load().gf_plan_create(ctypes.byref(grid), ctypes.byref(quad), _vp(obs_ptr), M,
                                 ctypes.byref(opt), _vp(stream), ctypes.byref(plan)))
    return plan.value


def gf_hex_sources(verts_ptr: int, ncell: int, quad: gf_quad, precision: int, x_ptr: int, a_ptr: int,
                   stream: int = 0):
    _check(load().gf_hex_sources(_vp(verts_ptr), ncell, ctypes.byref(quad), precision, _vp(x_ptr), _vp(a_ptr),
                                 _vp(stream)))


def gf_plan_create_points(src_ptr: int, wt_ptr: int, S: int, per_cell: int, obs_ptr: int, M: int,
                          opt: gf_options, stream: int = 0) -> int:
    plan = _vp()
    _check(load().gf_plan_create_points(_vp(src_ptr), _vp(wt_ptr), S, per_cell, _vp(obs_ptr), M,
                                        ctypes.byref(opt), _vp(stream), ctypes.byref(plan)))
    return plan.value


def gf_forward(plan: int, rho_ptr: int, rho_dtype: int, B: int, g_ptr: int, gz_ptr: int,
               stream: int = 0):
    _check(load().gf_forward(_vp(plan), _vp(rho_ptr), rho_dtype, B, _vp(g_ptr or None),
                             _vp(gz_ptr or None), _vp(stream)))


def gf_adjoint(plan: int, r_ptr: int, ncomp: int, B: int, grad_ptr: int, stream: int = 0):
    _check(load().gf_adjoint(_vp(plan), _vp(r_ptr or None), ncomp, B, _vp(grad_ptr), _vp(stream)))


def gf_direct_forward_static(grid: gf_grid, quad: gf_quad, obs_ptr: int, M: int, rho_ptr: int,
                             rho_dtype: int, B: int, G: float, g_ptr: int, gz_ptr: int, stream: int = 0):
    """Allocation-free direct forward (mixed precision, M <= 65536): for
    callers that cannot allocate device memory at solve time.  Calls whose
    device work overlaps share one scratch array and race."""
    _check(load().gf_direct_forward_static(ctypes.byref(grid), ctypes.byref(quad), _vp(obs_ptr), int(M),
                                           _vp(rho_ptr), rho_dtype, B, float(G), _vp(g_ptr or None),
                                           _vp(gz_ptr or None), _vp(stream)))


def gf_plan_destroy(plan: int):
    _check(load().gf_plan_destroy(_vp(plan)))


def gf_plan_check(plan: int, stream: int = 0):
    _check(load().gf_plan_check(_vp(plan), _vp(stream)))


def gf_plan_bytes(grid: gf_grid, quad: gf_quad, M: int, opt: gf_options) -> int:
    out = ctypes.c_size_t()
    _check(load().gf_plan_bytes(ctypes.byref(grid), ctypes.byref(quad), M, ctypes.byref(opt),
                                ctypes.byref(out)))
    return int(out.value)


def gf_plan_get_info(plan: int) -> gf_plan_info:
    info = gf_plan_info()
    _check(load().gf_plan_get_info(_vp(plan), ctypes.byref(info)))
    return info


def gf_plan_export_tree(plan: int, level: int, perm_ptr=None, keys_ptr=None, box_keys_ptr=None,
                        ilist_ptr=None, near_ptr=None):
    _check(load().gf_plan_export_tree(_vp(plan), level, _vp(perm_ptr), _vp(keys_ptr),
                                      _vp(box_keys_ptr), _vp(ilist_ptr), _vp(near_ptr)))


def gf_plan_set_source_part(plan: int, part: int, nparts: int):
    """Restrict a FMM plan's forward to source part `part` of `nparts`;
    returns the part's range [lo, hi) of level-2 Morton codes."""
    lo, hi = ctypes.c_int32(0), ctypes.c_int32(0)
    _check(load().gf_plan_set_source_part(_vp(plan), int(part), int(nparts), ctypes.byref(lo), ctypes.byref(hi)))
    return int(lo.value), int(hi.value)


def gf_plan_set_timing(plan: int, enable: bool):
    _check(load().gf_plan_set_timing(_vp(plan), 1 if enable else 0))


def gf_plan_stage_times(plan: int) -> dict:
    ms = (ctypes.c_double * GF_NUM_STAGES)()
    _check(load().gf_plan_stage_times(_vp(plan), ms))
    return {STAGE_NAMES[i]: float(ms[i]) for i in range(GF_NUM_STAGES)}


def gf_version() -> int:
    return int(load().gf_version())


def gf_launch_count() -> int:
    return int(load().gf_launch_count())


def gf_server_create(opt: gf_server_options) -> int:
    h = _vp()
    _check(load().gf_server_create(ctypes.byref(opt), ctypes.byref(h)))
    return h.value


def gf_server_submit(server: int, req: gf_request) -> int:
    t = ctypes.c_int64()
    _check(load().gf_server_submit(server, ctypes.byref(req), ctypes.byref(t)))
    return t.value


def gf_server_wait(server: int, ticket: int, timeout_ms: float = -1.0) -> float:
    lat = ctypes.c_double()
    _check(load().gf_server_wait(server, int(ticket), float(timeout_ms), ctypes.byref(lat)))
    return lat.value


def gf_server_stats_get(server: int) -> gf_server_stats:
    st = gf_server_stats()
    _check(load().gf_server_stats_get(server, ctypes.byref(st)))
    return st


def gf_server_destroy(server: int):
    _check(load().gf_server_destroy(server))


# ------------------------------------------------------------ marshalling
def make_grid(shape, origin, h) -> gf_grid:
    g = gf_grid()
    for a in range(3):
        g.n[a] = int(shape[a])
        g.origin[a] = float(origin[a])
        g.h[a] = float(h[a])
    return g


class _Quad:
    """Keeps the host arrays of a gf_quad alive."""

    def __init__(self, xi, w):
        self.xi = np.ascontiguousarray(xi, dtype=np.float64).reshape(-1, 3)
        self.w = np.ascontiguousarray(w, dtype=np.float64).reshape(-1)
        self.c = gf_quad()
        self.c.nq = int(self.w.shape[0])
        self.c.xi = self.xi.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        self.c.w = self.w.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


GF_FLAG_M2L_SIMT = 1
GF_FLAG_SUM_AN = 2
GF_FLAG_TEST_WAIT_TIMEOUT = 4
GF_FLAG_M2L_TENSOR = 8


def make_options(mode="fmm", precision="fp64", p=8, leaf_vox=0, max_batch=1, G=0.0, flags=0) -> gf_options:
    o = gf_options()
    o.reserved0 = int(flags)
    o.mode = {"direct": GF_MODE_DIRECT, "fmm": GF_MODE_FMM}[mode] if isinstance(mode, str) else int(mode)
    o.precision = ({"fp64": GF_PREC_FP64, "mixed": GF_PREC_MIXED}[precision]
                   if isinstance(precision, str) else int(precision))
    o.p = int(p)
    o.leaf_vox = int(leaf_vox)
    o.max_batch = int(max_batch)
    o.G = float(G)
    return o


def _stream_handle(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _check_tensor(t, name, numel, device=None, dtypes=None):
    """Reject a tensor the kernels would read or write out of bounds: it must
    be contiguous, hold `numel` elements of one of `dtypes` (default float64)
    and live on `device` (a CUDA device; None means host memory)."""
    import torch
    dtypes = dtypes or (torch.float64,)
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch tensor" % name)
    if device is None:
        if t.is_cuda:
            raise TypeError("%s must be in host memory" % name)
    elif not (t.is_cuda and t.device == device):
        raise TypeError("%s must be a CUDA tensor on %s (got %s)" % (name, device, t.device))
    if t.dtype not in dtypes:
        raise TypeError("%s must have dtype %s (got %s)" % (name, " or ".join(map(str, dtypes)), t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if t.numel() != numel:
        raise ValueError("%s must hold %d elements (got %d)" % (name, numel, t.numel()))


def _check_array(a, name, numel):
    """Host output arrays of a serving request: C-contiguous float64 with
    `numel` elements."""
    if not isinstance(a, np.ndarray):
        raise TypeError("%s must be a numpy array" % name)
    if a.dtype != np.float64 or not a.flags.c_contiguous or not a.flags.writeable:
        raise TypeError("%s must be a writeable C-contiguous float64 array" % name)
    if a.size != numel:
        raise ValueError("%s must hold %d elements (got %d)" % (name, numel, a.size))


class Plan:
    """A forward-model plan for one voxel grid, quadrature rule and
    observer set (see ``gf_plan_create``).

    obs must be a CUDA float64 tensor of shape (M, 3).  m2l="simt" runs the
    mixed-precision M2L on the SIMT cores; m2l="tensor" runs an FP64 plan's
    M2L on the tensor cores (FP16 parts, the rest FP64); voxels="closed_form" integrates
    every voxel exactly (SUM-AN; direct mode, FP64) instead of sampling it
    with the rule (xi, w).  flags: further GF_FLAG_* bits (testing aids)."""

    def __init__(self, shape, origin, h, xi, w, obs, mode="fmm", precision="fp64", p=8,
                 leaf_vox=0, max_batch=1, G=0.0, stream=None, m2l="auto", voxels="quadrature",
                 flags=0):
        import torch
        if not (isinstance(obs, torch.Tensor) and obs.is_cuda):
            raise TypeError("obs must be a CUDA tensor")
        obs = obs.to(torch.float64).contiguous().reshape(-1, 3)
        self.shape = tuple(int(s) for s in shape)
        self.M = int(obs.shape[0])
        self.max_batch = int(max_batch)
        self.device = obs.device
        self._grid = make_grid(shape, origin, h)
        self._quad = _Quad(xi, w)
        if m2l not in ("auto", "simt", "tensor") or voxels not in ("quadrature", "closed_form"):
            raise ValueError("m2l must be 'auto', 'simt' or 'tensor', voxels 'quadrature' or 'closed_form'")
        self._opt = make_options(mode, precision, p, leaf_vox, max_batch, G,
                                 (GF_FLAG_M2L_SIMT if m2l == "simt" else 0)
                                 | (GF_FLAG_M2L_TENSOR if m2l == "tensor" else 0)
                                 | (GF_FLAG_SUM_AN if voxels == "closed_form" else 0) | int(flags))
        self.handle = None
        with torch.cuda.device(self.device):
            self.handle = gf_plan_create(self._grid, self._quad.c, obs.data_ptr(), self.M, self._opt,
                                         _stream_handle(stream))

    @property
    def info(self) -> gf_plan_info:
        return gf_plan_get_info(self.handle)

    def forward(self, rho, g=None, gz=None, want_g=True, want_gz=False, stream=None):
        """rho: CUDA tensor (nz, ny, nx) or (B, nz, ny, nx), float32/float64,
        on the plan's device.  Returns (g, gz) with g (B?, M, 3) and gz
        (B?, M) float64 (None for an output not requested).  Outputs passed
        in must be contiguous float64 CUDA tensors of B*M*3 (g) or B*M (gz)
        elements on the same device; they are filled and returned as given."""
        import torch
        nx, ny, nz = self.shape
        if not isinstance(rho, torch.Tensor) or rho.dim() not in (3, 4) or tuple(rho.shape[-3:]) != (nz, ny, nx):
            raise ValueError("rho must be a tensor of shape (nz, ny, nx) or (B, nz, ny, nx) = (B?, %d, %d, %d)"
                             % (nz, ny, nx))
        single = rho.dim() == 3
        rho = rho.contiguous().reshape(-1, nz, ny, nx)
        B = int(rho.shape[0])
        _check_tensor(rho, "rho", B * nz * ny * nx, self.device, (torch.float32, torch.float64))
        dt = GF_DTYPE_F64 if rho.dtype == torch.float64 else GF_DTYPE_F32
        own_g, own_gz = g is None, gz is None
        if want_g and g is None:
            g = torch.empty((B, self.M, 3), dtype=torch.float64, device=rho.device)
        if want_gz and gz is None:
            gz = torch.empty((B, self.M), dtype=torch.float64, device=rho.device)
        if g is not None:
            _check_tensor(g, "g", B * self.M * 3, self.device)
        if gz is not None:
            _check_tensor(gz, "gz", B * self.M, self.device)
        with torch.cuda.device(self.device):
            gf_forward(self.handle, rho.data_ptr(), dt, B, g.data_ptr() if g is not None else 0,
                       gz.data_ptr() if gz is not None else 0, _stream_handle(stream))
        if single:
            g = g[0] if (g is not None and own_g) else g
            gz = gz[0] if (gz is not None and own_gz) else gz
        return g, gz

    def adjoint(self, r, ncomp=1, grad=None, stream=None):
        """r: CUDA float64 (B?, M) for ncomp = 1 or (B?, M, 3) for ncomp = 3.
        Returns grad (B?, nz, ny, nx) float64."""
        import torch
        nx, ny, nz = self.shape
        if ncomp not in (1, 3):
            raise ValueError("ncomp must be 1 (weights on g_z) or 3 (weights on g)")
        if not (isinstance(r, torch.Tensor) and r.is_cuda and r.device == self.device):
            raise TypeError("r must be a CUDA tensor on %s" % self.device)
        single = r.dim() == (1 if ncomp == 1 else 2)
        r = r.to(torch.float64).contiguous()
        if self.M == 0:
            B = 1 if single else int(r.shape[0])
        elif r.numel() % (self.M * ncomp) == 0 and r.numel() > 0:
            B = r.numel() // (self.M * ncomp)
        else:
            raise ValueError("r must have shape (B?, M) for ncomp = 1 or (B?, M, 3) for ncomp = 3")
        own = grad is None
        if grad is None:
            grad = torch.empty((B, nz, ny, nx), dtype=torch.float64, device=r.device)
        _check_tensor(grad, "grad", B * nz * ny * nx, self.device)
        with torch.cuda.device(self.device):
            gf_adjoint(self.handle, r.data_ptr(), ncomp, B, grad.data_ptr(), _stream_handle(stream))
        return grad[0] if (single and own) else grad

    def set_timing(self, enable=True):
        gf_plan_set_timing(self.handle, enable)

    def stage_times(self) -> dict:
        """Device milliseconds per stage of the last timed forward."""
        return gf_plan_stage_times(self.handle)

    def check(self, stream=None):
        gf_plan_check(self.handle, _stream_handle(stream))

    def set_source_part(self, part, nparts):
        """Restrict the forward to source part `part` of `nparts` (one
        device's share of a source-partitioned solve); the sum of the parts'
        fields is the whole field.  Returns the level-2 Morton range."""
        return gf_plan_set_source_part(self.handle, part, nparts)

    def export_tree(self, level):
        """Host copies of the observer order, leaf keys, occupied boxes of
        `level`, their interaction lists and (level == L) near lists."""
        info = self.info
        nb = int(info.n_target_boxes[level])
        perm = np.zeros(self.M, dtype=np.int32)
        keys = np.zeros(self.M, dtype=np.uint64)
        boxes = np.zeros(nb, dtype=np.uint64)
        il = np.zeros((nb, 316), dtype=np.int64)
        near = np.zeros((nb, 27), dtype=np.int64) if level == info.L else None
        gf_plan_export_tree(self.handle, level, perm.ctypes.data, keys.ctypes.data, boxes.ctypes.data,
                            il.ctypes.data, near.ctypes.data if near is not None else None)
        return perm, keys, boxes, il, near

    def close(self):
        if self.handle:
            gf_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def hex_sources(verts, xi, w, precision="fp64", stream=None):
    """Quadrature points and volume weights of deformed hexahedral cells
    (``gf_hex_sources``).  verts: CUDA float64 tensor (ncell, 8, 3), corner
    a = i + 2 j + 4 k at reference signs (2i - 1, 2j - 1, 2k - 1); (xi, w):
    the rule on [-1, 1]^3; precision "fp64" or "mixed" (FP32 relative to
    each cell's first corner, for mixed-precision plans).  Returns x
    (ncell * nq, 3) and a (ncell * nq,), source c * nq + q being node q of
    cell c."""
    import torch
    if not (isinstance(verts, torch.Tensor) and verts.is_cuda):
        raise TypeError("verts must be a CUDA tensor")
    verts = verts.to(torch.float64).contiguous()
    if verts.numel() % 24 != 0:
        raise ValueError("verts must have shape (ncell, 8, 3)")
    ncell = verts.numel() // 24
    q = _Quad(xi, w)
    nq = int(q.c.nq)
    x = torch.empty((ncell * nq, 3), dtype=torch.float64, device=verts.device)
    a = torch.empty((ncell * nq,), dtype=torch.float64, device=verts.device)
    with torch.cuda.device(verts.device):
        prec = {"fp64": GF_PREC_FP64, "mixed": GF_PREC_MIXED}[precision] if isinstance(precision, str) \
            else int(precision)
        gf_hex_sources(verts.data_ptr(), ncell, q.c, prec, x.data_ptr(), a.data_ptr(), _stream_handle(stream))
    return x, a


class PointsPlan(Plan):
    """A forward-model plan over weighted point sources
    (``gf_plan_create_points``): source s at src[s] with volume weight
    wt[s] samples density s // per_cell.  src (S, 3), wt (S,) and obs (M, 3)
    are CUDA float64 tensors; forward takes rho of shape (ncell,) or
    (B, ncell), ncell = S // per_cell."""

    def __init__(self, src, wt, obs, per_cell=1, mode="fmm", precision="fp64", p=8, max_batch=1, G=0.0,
                 stream=None, m2l="auto", flags=0):
        import torch
        for t, n in ((src, "src"), (wt, "wt"), (obs, "obs")):
            if not (isinstance(t, torch.Tensor) and t.is_cuda):
                raise TypeError("%s must be a CUDA tensor" % n)
        src = src.to(torch.float64).contiguous().reshape(-1, 3)
        wt = wt.to(torch.float64).contiguous().reshape(-1)
        obs = obs.to(torch.float64).contiguous().reshape(-1, 3)
        if wt.shape[0] != src.shape[0]:
            raise ValueError("wt must hold one weight per source")
        self.S = int(src.shape[0])
        self.per_cell = int(per_cell)
        self.ncell = self.S // max(self.per_cell, 1)
        self.shape = (self.ncell,)
        self.M = int(obs.shape[0])
        self.max_batch = int(max_batch)
        self.device = obs.device
        if m2l not in ("auto", "simt"):
            raise ValueError("m2l must be 'auto' or 'simt'")
        self._opt = make_options(mode, precision, p, 0, max_batch, G,
                                 (GF_FLAG_M2L_SIMT if m2l == "simt" else 0) | int(flags))
        self.handle = None
        with torch.cuda.device(self.device):
            self.handle = gf_plan_create_points(src.data_ptr(), wt.data_ptr(), self.S, self.per_cell,
                                                obs.data_ptr(), self.M, self._opt, _stream_handle(stream))

    def forward(self, rho, g=None, gz=None, want_g=True, want_gz=False, stream=None):
        """rho: CUDA tensor (ncell,) or (B, ncell), float32/float64.  Returns
        (g, gz) as :meth:`Plan.forward` does."""
        import torch
        if not isinstance(rho, torch.Tensor) or rho.dim() not in (1, 2) or rho.shape[-1] != self.ncell:
            raise ValueError("rho must be a tensor of shape (ncell,) or (B, ncell), ncell = %d" % self.ncell)
        single = rho.dim() == 1
        B = 1 if single else int(rho.shape[0])
        rho = rho.contiguous().reshape(B, self.ncell)
        _check_tensor(rho, "rho", B * self.ncell, self.device, (torch.float32, torch.float64))
        dt = GF_DTYPE_F64 if rho.dtype == torch.float64 else GF_DTYPE_F32
        own_g, own_gz = g is None, gz is None
        if want_g and g is None:
            g = torch.empty((B, self.M, 3), dtype=torch.float64, device=rho.device)
        if want_gz and gz is None:
            gz = torch.empty((B, self.M), dtype=torch.float64, device=rho.device)
        if g is not None:
            _check_tensor(g, "g", B * self.M * 3, self.device)
        if gz is not None:
            _check_tensor(gz, "gz", B * self.M, self.device)
        with torch.cuda.device(self.device):
            gf_forward(self.handle, rho.data_ptr(), dt, B, g.data_ptr() if g is not None else 0,
                       gz.data_ptr() if gz is not None else 0, _stream_handle(stream))
        if single:
            g = g[0] if (g is not None and own_g) else g
            gz = gz[0] if (gz is not None and own_gz) else gz
        return g, gz

    def adjoint(self, r, ncomp=1, grad=None, stream=None):
        """Not implemented for point sources: the library answers
        GF_ERR_UNSUPPORTED, raised here as GfError."""
        import torch
        if grad is None:
            grad = torch.empty((1, self.ncell), dtype=torch.float64, device=self.device)
        with torch.cuda.device(self.device):
            gf_adjoint(self.handle, r.data_ptr(), ncomp, 1, grad.data_ptr(), _stream_handle(stream))
        return grad


def plan_bytes(shape, origin, h, xi, w, M, **opts) -> int:
    q = _Quad(xi, w)
    return gf_plan_bytes(make_grid(shape, origin, h), q.c, int(M), make_options(**opts))


class Server:
    """Continuous-batching forward server (``gf_server_*``): requests for
    any registered geometry are queued and run concurrently on ``slots``
    CUDA streams, each geometry's plan kept resident (and its forward
    replayed as a CUDA graph) until evicted under ``mem_budget``."""

    def __init__(self, slots=4, precision="mixed", p=12, leaf_vox=0, use_graphs=True, device=0,
                 mem_budget=0, G=0.0):
        o = gf_server_options()
        o.max_slots = int(slots)
        o.precision = {"fp64": GF_PREC_FP64, "mixed": GF_PREC_MIXED}[precision]
        o.p = int(p)
        o.leaf_vox = int(leaf_vox)
        o.use_graphs = 1 if use_graphs else 0
        o.device = int(device)
        o.mem_budget = int(mem_budget)
        o.G = float(G)
        self._geoms = {}
        self._pending = {}
        self._device_index = int(device)
        self.handle = None
        self.handle = gf_server_create(o)

    def register(self, gid, shape, origin, h, xi, w, obs):
        """Declare geometry `gid`: grid, quadrature rule, observers (M, 3)."""
        obs = np.ascontiguousarray(obs, dtype=np.float64).reshape(-1, 3)
        self._geoms[int(gid)] = (make_grid(shape, origin, h), _Quad(xi, w), obs,
                                 tuple(int(v) for v in shape))

    def submit(self, gid, rho, gz=None, g=None, want_gz=True, want_g=False) -> int:
        """Queue a forward of densities `rho` (nz, ny, nx) on geometry `gid`.
        rho and the outputs are host arrays (numpy, or CPU tensors; pinned
        ones make the copies asynchronous) or all CUDA tensors on the
        server's device; outputs passed in are contiguous float64 with M
        (gz) or 3M (g) elements.  Returns a ticket for :meth:`wait`."""
        import torch
        grid, quad, obs, shape = self._geoms[int(gid)]
        M = obs.shape[0]
        if not isinstance(rho, torch.Tensor):
            rho = np.ascontiguousarray(rho)
        if tuple(rho.shape) != (shape[2], shape[1], shape[0]):
            raise ValueError("rho must have shape (nz, ny, nx) = %r" % ((shape[2], shape[1], shape[0]),))
        if isinstance(rho, torch.Tensor):
            on_device = rho.is_cuda
            dev = torch.device("cuda", self._device_index) if on_device else None
            pin = (not on_device) and rho.is_pinned()
            rho = rho.contiguous()
            _check_tensor(rho, "rho", rho.numel(), dev, (torch.float32, torch.float64))
            rdt = GF_DTYPE_F64 if rho.dtype == torch.float64 else GF_DTYPE_F32
            if want_gz and gz is None:
                gz = torch.empty(M, dtype=torch.float64, device=rho.device, pin_memory=pin)
            if want_g and g is None:
                g = torch.empty((M, 3), dtype=torch.float64, device=rho.device, pin_memory=pin)
            if gz is not None:
                _check_tensor(gz, "gz", M, dev)
            if g is not None:
                _check_tensor(g, "g", 3 * M, dev)
            ptr = lambda a: a.data_ptr()  # noqa: E731
        else:
            on_device = False
            if rho.dtype not in (np.dtype(np.float64), np.dtype(np.float32)):
                raise TypeError("rho must be float32 or float64")
            rdt = GF_DTYPE_F64 if rho.dtype == np.float64 else GF_DTYPE_F32
            if want_gz and gz is None:
                gz = np.empty(M, dtype=np.float64)
            if want_g and g is None:
                g = np.empty((M, 3), dtype=np.float64)
            if gz is not None:
                _check_array(gz, "gz", M)
            if g is not None:
                _check_array(g, "g", 3 * M)
            ptr = lambda a: a.ctypes.data  # noqa: E731
        r = gf_request()
        r.grid = grid
        r.quad = quad.c
        r.obs_host = obs.ctypes.data
        r.M = M
        r.geometry_id = int(gid)
        r.rho_host = ptr(rho)
        r.rho_dtype = rdt
        r.on_device = 1 if on_device else 0
        r.gz_host = ptr(gz) if gz is not None else None
        r.g_host = ptr(g) if g is not None else None
        t = gf_server_submit(self.handle, r)
        self._pending[t] = (gz, g, rho)
        return t

    def wait(self, ticket, timeout_ms=-1.0):
        """Wait for a request; returns (gz, g, latency_ms).  Each ticket is
        waited for once."""
        lat = gf_server_wait(self.handle, ticket, timeout_ms)
        gz, g, _ = self._pending.pop(ticket)
        return gz, g, lat

    def stats(self) -> dict:
        st = gf_server_stats_get(self.handle)
        return {k: getattr(st, k) for k, _ in gf_server_stats._fields_}

    def close(self):
        if self.handle:
            gf_server_destroy(self.handle)
            self.handle = None
            self._pending.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
