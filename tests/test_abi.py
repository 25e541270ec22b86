"""The C-ABI library builds for sm_103a, loads without a GPU, exports every
entry point include/gf.h declares, and rejects bad arguments on the host
before touching the device."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import paper_1107_5951_gb300 as pkg
from paper_1107_5951_gb300 import gf, workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\s*(?:[\w\s\*]+?)\b(gf_\w+)\s*\(", src, flags=re.M))
    return sorted(names)


def test_every_declared_symbol_is_exported():
    lib = pkg.load()
    declared = _declared()
    assert "gf_forward" in declared and "gf_plan_create" in declared
    for name in declared:
        assert hasattr(lib, name), name


def test_struct_layouts_match_the_header(tmp_path):
    """ctypes mirrors of the public structs have the C sizes and offsets."""
    prog = tmp_path / "sz.c"
    prog.write_text('#include "gf.h"\n#include <stdio.h>\n#include <stddef.h>\nint main(void){'
                    'printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(gf_grid), sizeof(gf_quad),'
                    ' sizeof(gf_options), sizeof(gf_plan_info), offsetof(gf_plan_info, M),'
                    ' offsetof(gf_options, G)); return 0;}')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    out = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert out == [ctypes.sizeof(gf.gf_grid), ctypes.sizeof(gf.gf_quad), ctypes.sizeof(gf.gf_options),
                   ctypes.sizeof(gf.gf_plan_info), gf.gf_plan_info.M.offset, gf.gf_options.G.offset]


def _args(**kw):
    grid = gf.make_grid((4, 4, 4), (0, 0, 0), (1, 1, 1))
    q = gf._Quad(*wl.gauss_rule(1))
    opt = gf.make_options(**kw)
    return grid, q, opt


@pytest.mark.parametrize("bad", [
    dict(mode="direct", max_batch=0),
    dict(mode=7),
    dict(mode="fmm", p=0),
    dict(mode="fmm", p=99),
    dict(mode="direct", precision=5),
    dict(mode="direct", G=-1.0),
])
def test_invalid_options_rejected_on_host(bad):
    grid, q, opt = _args(**bad)
    with pytest.raises(gf.GfError) as e:
        gf.gf_plan_bytes(grid, q.c, 10, opt)
    assert e.value.status == gf.GF_ERR_INVALID_ARG


def test_invalid_grid_and_quadrature_rejected():
    grid, q, opt = _args(mode="direct")
    grid.n[1] = 0
    with pytest.raises(gf.GfError) as e:
        gf.gf_plan_bytes(grid, q.c, 10, opt)
    assert e.value.status == gf.GF_ERR_INVALID_ARG
    grid, q, opt = _args(mode="direct")
    q.w[0] = -1.0
    with pytest.raises(gf.GfError):
        gf.gf_plan_bytes(grid, q.c, 10, opt)
    grid, q, opt = _args(mode="fmm", p=6)
    grid.h[2] = 2.0
    with pytest.raises(gf.GfError) as e:
        gf.gf_plan_bytes(grid, q.c, 10, opt)
    assert e.value.status == gf.GF_ERR_UNSUPPORTED


@pytest.mark.parametrize("n,ok", [((1 << 22,) * 3, False), ((1 << 14,) * 3, False),
                                  ((1 << 13,) * 3, True), ((1 << 22, 1 << 18, 1), True)])
def test_total_voxel_count_is_bounded(n, ok):
    """Grids above 2^40 voxels are rejected before any index product could
    overflow; each axis may still reach 2^22."""
    grid, q, opt = _args(mode="direct")
    for a in range(3):
        grid.n[a] = n[a]
    if ok:
        assert gf.gf_plan_bytes(grid, q.c, 10, opt) > 0
    else:
        with pytest.raises(gf.GfError) as e:
            gf.gf_plan_bytes(grid, q.c, 10, opt)
        assert e.value.status == gf.GF_ERR_INVALID_ARG
        assert "2^40" in gf.gf_last_error()


def test_closed_form_voxels_modes():
    """GF_FLAG_SUM_AN is accepted in direct mode in FP64 (the plan then holds
    the corner-lattice weights) and in FMM mode with 4^3-voxel leaves in
    either precision, and refused in mixed direct mode and with other leaf
    sizes; unknown flag bits are invalid arguments."""
    grid, q, opt = _args(mode="direct")
    plain = gf.gf_plan_bytes(grid, q.c, 10, opt)
    opt.reserved0 = gf.GF_FLAG_SUM_AN
    assert gf.gf_plan_bytes(grid, q.c, 10, opt) >= plain + 5 ** 3 * 8
    for ok in (dict(mode="fmm", p=6), dict(mode="fmm", p=6, precision="mixed", leaf_vox=4)):
        grid, q, opt = _args(flags=gf.GF_FLAG_SUM_AN, **ok)
        assert gf.gf_plan_bytes(grid, q.c, 10, opt) > 0
    for bad in (dict(mode="fmm", p=6, leaf_vox=2), dict(mode="direct", precision="mixed")):
        grid, q, opt = _args(flags=gf.GF_FLAG_SUM_AN, **bad)
        with pytest.raises(gf.GfError) as e:
            gf.gf_plan_bytes(grid, q.c, 10, opt)
        assert e.value.status == gf.GF_ERR_UNSUPPORTED
    grid, q, opt = _args(mode="direct", flags=16)
    with pytest.raises(gf.GfError) as e:
        gf.gf_plan_bytes(grid, q.c, 10, opt)
    assert e.value.status == gf.GF_ERR_INVALID_ARG


def test_null_plan_and_null_outputs_rejected():
    lib = pkg.load()
    assert lib.gf_forward(None, None, 0, 1, None, None, None) == gf.GF_ERR_INVALID_ARG
    assert "plan is NULL" in gf.gf_last_error()
    assert lib.gf_plan_destroy(None) == gf.GF_OK


def test_plan_bytes_grows_with_problem():
    grid, q, opt = _args(mode="direct", precision="mixed")
    small = gf.gf_plan_bytes(grid, q.c, 1000, opt)
    big = gf.gf_plan_bytes(grid, q.c, 100000, opt)
    assert big > small > 0


def test_server_struct_layouts_match_the_header(tmp_path):
    """ctypes mirrors of the serving structs have the C sizes and offsets."""
    prog = tmp_path / "ss.c"
    prog.write_text('#include "gf.h"\n#include <stdio.h>\n#include <stddef.h>\nint main(void){'
                    'printf("%zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(gf_server_options), sizeof(gf_request),'
                    ' sizeof(gf_server_stats), offsetof(gf_server_options, mem_budget), offsetof(gf_request, rho_host),'
                    ' offsetof(gf_request, g_host), offsetof(gf_server_stats, p99_ms), offsetof(gf_server_stats, busy_s));'
                    ' return 0;}')
    exe = tmp_path / "ss"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    out = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert out == [ctypes.sizeof(gf.gf_server_options), ctypes.sizeof(gf.gf_request),
                   ctypes.sizeof(gf.gf_server_stats), gf.gf_server_options.mem_budget.offset,
                   gf.gf_request.rho_host.offset, gf.gf_request.g_host.offset, gf.gf_server_stats.p99_ms.offset,
                   gf.gf_server_stats.busy_s.offset]


def test_server_arguments_rejected_on_host():
    """Bad server options and requests fail with GF_ERR_INVALID_ARG before any
    device call (this also holds on a machine without a GPU)."""
    lib = pkg.load()
    o = gf.gf_server_options()
    o.max_slots = 0
    o.precision = gf.GF_PREC_MIXED
    o.p = 12
    h = ctypes.c_void_p()
    assert lib.gf_server_create(ctypes.byref(o), ctypes.byref(h)) == gf.GF_ERR_INVALID_ARG
    o.max_slots = 4
    o.p = 99
    assert lib.gf_server_create(ctypes.byref(o), ctypes.byref(h)) == gf.GF_ERR_INVALID_ARG
    t = ctypes.c_int64()
    assert lib.gf_server_submit(None, None, ctypes.byref(t)) == gf.GF_ERR_INVALID_ARG
    assert lib.gf_server_wait(None, 1, 0.0, None) == gf.GF_ERR_INVALID_ARG
    assert lib.gf_server_destroy(None) == gf.GF_OK


def test_no_gpu_means_an_error_not_a_fallback():
    """Without a usable GPU, creating a plan or a server reports a CUDA error;
    nothing silently computes on the CPU."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lib = pkg.load()
    o = gf.gf_server_options()
    o.max_slots = 2
    o.precision = gf.GF_PREC_MIXED
    o.p = 8
    h = ctypes.c_void_p()
    rc = lib.gf_server_create(ctypes.byref(o), ctypes.byref(h))
    assert rc == gf.GF_ERR_CUDA and not h.value
    grid, q, opt = _args(mode="direct")
    obs = np.zeros((3, 3))
    plan = ctypes.c_void_p()
    rc = lib.gf_plan_create(ctypes.byref(grid), ctypes.byref(q.c), obs.ctypes.data, 1, ctypes.byref(opt), None,
                            ctypes.byref(plan))
    assert rc != gf.GF_OK and not plan.value


def test_point_source_arguments_rejected_on_host():
    """gf_plan_create_points and gf_hex_sources reject bad sizes, a per_cell
    that does not divide S, missing pointers and the closed-form flag before
    any device call; gf_hex_sources with no cells enqueues nothing."""
    lib = pkg.load()
    plan = ctypes.c_void_p()
    buf = np.zeros(64)
    p = buf.ctypes.data

    def create(S, per_cell, src=p, wt=p, obs=p, M=2, **kw):
        opt = gf.make_options(**kw)
        return lib.gf_plan_create_points(src, wt, S, per_cell, obs, M, ctypes.byref(opt), None,
                                         ctypes.byref(plan))

    assert create(10, 3, mode="direct") == gf.GF_ERR_INVALID_ARG
    assert "divide" in gf.gf_last_error()
    assert create(10, 0, mode="direct") == gf.GF_ERR_INVALID_ARG
    assert create(-1, 1, mode="direct") == gf.GF_ERR_INVALID_ARG
    assert create(1 << 31, 1, mode="direct") == gf.GF_ERR_INVALID_ARG
    assert create(4, 1, src=None, mode="direct") == gf.GF_ERR_INVALID_ARG
    assert create(4, 1, obs=None, mode="fmm", p=6) == gf.GF_ERR_INVALID_ARG
    assert create(4, 1, mode="fmm", p=0) == gf.GF_ERR_INVALID_ARG
    assert create(4, 1, mode="fmm", p=6, flags=gf.GF_FLAG_SUM_AN) == gf.GF_ERR_UNSUPPORTED
    assert not plan.value
    q = gf._Quad(*wl.gauss_rule(2))
    for prec in (gf.GF_PREC_FP64, gf.GF_PREC_MIXED):
        assert lib.gf_hex_sources(None, 0, ctypes.byref(q.c), prec, None, None, None) == gf.GF_OK
        assert lib.gf_hex_sources(None, 3, ctypes.byref(q.c), prec, None, None, None) == gf.GF_ERR_INVALID_ARG
        assert lib.gf_hex_sources(p, -1, ctypes.byref(q.c), prec, p, p, None) == gf.GF_ERR_INVALID_ARG
    assert lib.gf_hex_sources(p, 1, ctypes.byref(q.c), 7, p, p, None) == gf.GF_ERR_INVALID_ARG
    q.w[0] = 0.0
    assert lib.gf_hex_sources(p, 1, ctypes.byref(q.c), gf.GF_PREC_FP64, p, p, None) == gf.GF_ERR_INVALID_ARG


def test_tensor_m2l_flag_only_for_fp64_fmm():
    """GF_FLAG_M2L_TENSOR is accepted for FP64 FMM plans and refused in mixed
    precision, in direct mode and together with GF_FLAG_M2L_SIMT."""
    grid, q, opt = _args(mode="fmm", precision="fp64", p=8, flags=gf.GF_FLAG_M2L_TENSOR)
    assert gf.gf_plan_bytes(grid, q.c, 10, opt) > 0
    for bad in (dict(mode="fmm", precision="mixed", p=8), dict(mode="direct", precision="fp64"),
                dict(mode="fmm", precision="fp64", p=8, flags_extra=gf.GF_FLAG_M2L_SIMT)):
        extra = bad.pop("flags_extra", 0)
        grid, q, opt = _args(flags=gf.GF_FLAG_M2L_TENSOR | extra, **bad)
        with pytest.raises(gf.GfError) as e:
            gf.gf_plan_bytes(grid, q.c, 10, opt)
        assert e.value.status == gf.GF_ERR_UNSUPPORTED
