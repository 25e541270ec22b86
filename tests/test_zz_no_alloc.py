"""The allocation-free direct forward (gf_direct_forward_static), called
through the C ABI, against the plan-based mixed-precision direct forward.

This entry point serves callers that cannot allocate device memory at solve
time (allocator callbacks that must not re-enter the allocator, memory held
by a foreign caching pool, fixed-footprint services).  Its scratch is one
shared static device array, so two calls in a row must not see each other's
leftovers.  The file is named to be collected last."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1107_5951_gb300 as pkg  # noqa: E402
from paper_1107_5951_gb300 import gf, workloads as wl  # noqa: E402

DEV = "cuda:0"
TOL = 1e-5   # the mixed-precision bar used by the direct-mode tests


def _plan_result(wk, rho):
    obs = torch.tensor(wk.obs, dtype=torch.float64, device=DEV)
    with pkg.Plan(wk.grid.n, wk.grid.origin, wk.grid.h, wk.xi, wk.w, obs, mode="direct",
                  precision="mixed", max_batch=rho.shape[0], G=wk.G) as plan:
        g, gz = plan.forward(rho, want_gz=True)
        torch.cuda.synchronize()
        return g.cpu().numpy(), gz.cpu().numpy()


def _static_result(wk, rho):
    obs = torch.tensor(wk.obs, dtype=torch.float64, device=DEV)
    B, M = rho.shape[0], wk.n_obs
    g = torch.full((B, M, 3), float("nan"), dtype=torch.float64, device=DEV)
    gz = torch.full((B, M), float("nan"), dtype=torch.float64, device=DEV)
    quad = gf._Quad(wk.xi, wk.w)
    dtype = gf.GF_DTYPE_F32 if rho.dtype == torch.float32 else gf.GF_DTYPE_F64
    stream = torch.cuda.current_stream().cuda_stream
    gf.gf_direct_forward_static(gf.make_grid(wk.grid.n, wk.grid.origin, wk.grid.h), quad.c, obs.data_ptr(),
                                M, rho.data_ptr(), dtype, B, wk.G, g.data_ptr(), gz.data_ptr(), stream)
    torch.cuda.synchronize()
    return g.cpu().numpy(), gz.cpu().numpy()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_static_forward_matches_plan_on_two_calls_in_a_row():
    # first call: 2x2x2 Gauss, float64 densities, a batch of two
    wk1 = wl.random_small(71, n=(9, 7, 6), npts=2, n_obs=3000, B=2)
    rho1 = torch.tensor(wk1.rho, dtype=torch.float64, device=DEV)
    # second call: another grid, rule, observer count and dtype
    wk2 = wl.random_small(72, n=(13, 5, 8), npts=1, n_obs=777, h=(2.0, 1.5, 1.0))
    rho2 = torch.tensor(wk2.rho[None], dtype=torch.float32, device=DEV)
    s1, z1 = _static_result(wk1, rho1)
    s2, z2 = _static_result(wk2, rho2)
    p1, q1 = _plan_result(wk1, rho1)
    p2, q2 = _plan_result(wk2, rho2)
    for s, z, p, q in ((s1, z1, p1, q1), (s2, z2, p2, q2)):
        assert np.all(np.isfinite(s)) and np.all(np.isfinite(z))
        assert _rel(s, p) <= TOL
        assert _rel(z, q) <= TOL


def test_static_forward_allocates_no_device_memory():
    """What the entry point exists for: once the library's module is loaded
    (a first call), a call changes neither the device's free memory nor
    torch's reserved memory."""
    wk = wl.random_small(74, n=(11, 9, 7), npts=2, n_obs=5000, B=1)
    rho = torch.tensor(wk.rho[None], dtype=torch.float32, device=DEV)
    _static_result(wk, rho)          # loads the kernels (and the static array) if not yet loaded
    obs = torch.tensor(wk.obs, dtype=torch.float64, device=DEV)
    g = torch.empty((1, wk.n_obs, 3), dtype=torch.float64, device=DEV)
    quad = gf._Quad(wk.xi, wk.w)
    grid = gf.make_grid(wk.grid.n, wk.grid.origin, wk.grid.h)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    reserved0 = torch.cuda.memory_reserved()
    for _ in range(3):
        gf.gf_direct_forward_static(grid, quad.c, obs.data_ptr(), wk.n_obs, rho.data_ptr(), gf.GF_DTYPE_F32, 1,
                                    wk.G, g.data_ptr(), 0, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_reserved() == reserved0


def test_static_forward_rejects_too_many_observers():
    wk = wl.random_small(73, n=(2, 2, 2), npts=1, n_obs=4)
    obs = torch.zeros((65537, 3), dtype=torch.float64, device=DEV)
    rho = torch.tensor(wk.rho, dtype=torch.float64, device=DEV)
    out = torch.empty((65537, 3), dtype=torch.float64, device=DEV)
    quad = gf._Quad(wk.xi, wk.w)
    with pytest.raises(gf.GfError) as e:
        gf.gf_direct_forward_static(gf.make_grid(wk.grid.n, wk.grid.origin, wk.grid.h), quad.c,
                                    obs.data_ptr(), 65537, rho.data_ptr(), gf.GF_DTYPE_F64, 1, 1.0,
                                    out.data_ptr(), 0, 0)
    assert e.value.status == gf.GF_ERR_INVALID_ARG
    assert "65536" in str(e.value)
