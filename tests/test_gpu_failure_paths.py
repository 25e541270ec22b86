"""Failure paths that the device reports instead of faulting (Sec. 2.1
densities must be finite; the FMM's bounded waits must end): a non-finite
density in any mode sets the plan's device status word and the next
gf_plan_check returns GF_ERR_DEVICE_CHECK; a tensor-core M2L whose barrier
wait runs out (GF_FLAG_TEST_WAIT_TIMEOUT makes the MMA issuer wait on a
barrier that nothing completes, with a short bound) stops, drains its copies,
frees its tensor memory and reports the timed-out wait the same way, and the
device stays usable.  No test here traps or faults the GPU."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1107_5951_gb300 as pkg  # noqa: E402
from oracle import direct  # noqa: E402
from paper_1107_5951_gb300 import gf, workloads as wl  # noqa: E402

DEV = "cuda:0"


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def layered(n=48, stations=24):
    """Leaf-aligned grid (every axis a multiple of the 4-voxel leaf) with
    stations on the top face: the parent-level expansions then come straight
    from the density grid, and only the top slabs are copied leaf by leaf."""
    h = 100.0
    grid = wl.Grid((n, n, n), (0.0, 0.0, -n * h), (h, h, h))
    rng = np.random.default_rng(5)
    rho = (2700.0 + 50.0 * rng.standard_normal(grid.shape_zyx)).astype(np.float32)
    xi, w = wl.gauss_rule(1)
    obs = wl.station_plane(0.0, n * h, 0.0, n * h, stations, stations, grid.top)
    return wl.Workload("layered_small", grid, rho, xi, w, obs)


def plan_for(wk, **kw):
    obs = torch.tensor(wk.obs, dtype=torch.float64, device=DEV)
    return pkg.Plan(wk.grid.n, wk.grid.origin, wk.grid.h, wk.xi, wk.w, obs, G=wk.G, **kw)


def expect_device_check(plan, rho, text):
    plan.forward(rho)
    torch.cuda.synchronize()
    with pytest.raises(gf.GfError) as e:
        plan.check()
    assert e.value.status == gf.GF_ERR_DEVICE_CHECK
    assert text in str(e.value)
    plan.check()   # the status word is cleared by the report


@pytest.mark.parametrize("where", ["top", "deep"])
@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_nan_density_reported_in_fmm_mode(where, precision):
    """A NaN next to the stations (read by the near field) and one at the
    bottom of the grid (read only by the upward sweep) are both reported."""
    wk = layered()
    rho = np.array(wk.rho, dtype=np.float32 if precision == "mixed" else np.float64)
    k = wk.grid.n[2] - 1 if where == "top" else 0
    rho[k, 17, 29] = np.nan
    with plan_for(wk, mode="fmm", precision=precision, p=12) as plan:
        assert plan.info.L >= 4
        expect_device_check(plan, torch.tensor(rho, device=DEV), "non-finite density 1")
        # a finite density afterwards is clean again and meets the oracle
        good = np.array(wk.rho, dtype=rho.dtype)
        g, _ = plan.forward(torch.tensor(good, device=DEV))
        torch.cuda.synchronize()
        plan.check()
        ref = direct.forward(wk.grid.n, wk.grid.origin, wk.grid.h, wk.xi, wk.w, good.astype(np.float64),
                             wk.obs, wk.G)
        assert rel_l2(g.cpu().numpy(), ref) <= 1e-5


@pytest.mark.parametrize("precision,voxels", [("fp64", "quadrature"), ("mixed", "quadrature"),
                                              ("fp64", "closed_form")])
def test_nan_density_reported_in_direct_mode(precision, voxels):
    wk = wl.random_small(81, n=(7, 6, 5), npts=1, n_obs=50)
    rho = np.array(wk.rho, dtype=np.float64)
    rho[3, 2, 4] = np.inf
    with plan_for(wk, mode="direct", precision=precision, voxels=voxels) as plan:
        expect_device_check(plan, torch.tensor(rho, device=DEV), "non-finite density 1")


def test_m2l_bounded_wait_runs_out_and_reports():
    """The tensor-core M2L's issuer waits on a barrier that nothing
    completes; the wait ends at its bound, the kernel drains and returns, the
    plan reports the timed-out wait, and the next plan on the same device
    computes the right field."""
    wk = wl.random_small(82, n=(28, 25, 23), npts=1, n_obs=400, h=(1.0, 1.0, 1.0),
                         origin=(-5.0, 3.0, -20.0), obs_pad=3.0)
    rho = torch.tensor(wk.rho, dtype=torch.float32, device=DEV)
    with plan_for(wk, mode="fmm", precision="mixed", p=8, flags=gf.GF_FLAG_TEST_WAIT_TIMEOUT) as plan:
        assert plan.info.L >= 3
        expect_device_check(plan, rho, "bounded wait 1")
    ref = direct.forward(wk.grid.n, wk.grid.origin, wk.grid.h, wk.xi, wk.w, wk.rho, wk.obs, wk.G)
    with plan_for(wk, mode="fmm", precision="mixed", p=12) as plan:
        g, _ = plan.forward(rho)
        torch.cuda.synchronize()
        plan.check()
        assert rel_l2(g.cpu().numpy(), ref) <= 1e-5
