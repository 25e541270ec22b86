"""The workloads of the paper's scale at full size against the FP64 CPU
direct-sum oracle (discretised Eq. 1) on seeded observer samples.

* 464^3 layered model (99,897,344 voxels of 100 m, FP32 densities, 1024^2
  stations on the top face): the mixed-precision FMM at the benchmark's
  degree p = 10 and at p = 11 within the metric's 1e-6, at p = 8 within the
  mixed bar 1e-5, and the plain FP64 FMM at p = 10 within 1e-6.
* 128^3 random-field volume workload (2,097,152 sources, 2,359,296
  observers): the plain FP64 FMM at p = 14 within 1e-6.

The oracle sums every source for each sampled observer, so the samples are
kept to a few hundred observers."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1107_5951_gb300 as pkg  # noqa: E402
from oracle import direct  # noqa: E402
from paper_1107_5951_gb300 import workloads as wl  # noqa: E402

DEV = "cuda:0"


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def scale():
    wk = wl.layered_scale()
    rng = np.random.default_rng(1234)
    idx = np.sort(rng.choice(wk.n_obs, 160, replace=False))
    ref = direct.forward(wk.grid.n, wk.grid.origin, wk.grid.h, wk.xi, wk.w,
                         np.asarray(wk.rho, dtype=np.float64), wk.obs[idx], wk.G)
    obs = torch.tensor(wk.obs, dtype=torch.float64, device=DEV)
    rho = torch.tensor(wk.rho, dtype=torch.float32, device=DEV)
    return wk, idx, ref, obs, rho


def scale_run(scale, precision, p):
    wk, idx, ref, obs, rho = scale
    r = rho if precision == "mixed" else rho.double()
    with pkg.Plan(wk.grid.n, wk.grid.origin, wk.grid.h, wk.xi, wk.w, obs, mode="fmm", precision=precision,
                  p=p, G=wk.G) as plan:
        assert plan.info.L == 7
        g, gz = plan.forward(r, want_gz=True)
        torch.cuda.synchronize()
        plan.check()
        g = g.cpu().numpy()
        assert np.all(np.isfinite(g))
        assert np.array_equal(gz.cpu().numpy(), g[:, 2])
        return g[idx]


@pytest.mark.parametrize("precision,p,tol", [("mixed", 10, 1e-6), ("mixed", 11, 1e-6), ("mixed", 8, 1e-5),
                                              ("fp64", 10, 1e-6)])
def test_layered_scale_464_full_size(scale, precision, p, tol):
    g = scale_run(scale, precision, p)
    err = rel_l2(g, scale[2])
    print("layered_scale 464^3 %s p=%d sampled rel L2 %.3e" % (precision, p, err))
    assert err <= tol


def test_grf_volume_full_size_fp64_p14():
    wk = wl.grf_volume()
    rng = np.random.default_rng(98)
    idx = np.sort(rng.choice(wk.n_obs, 256, replace=False))
    ref = direct.forward(wk.grid.n, wk.grid.origin, wk.grid.h, wk.xi, wk.w, wk.rho, wk.obs[idx], wk.G)
    obs = torch.tensor(wk.obs, dtype=torch.float64, device=DEV)
    with pkg.Plan(wk.grid.n, wk.grid.origin, wk.grid.h, wk.xi, wk.w, obs, mode="fmm", precision="fp64", p=14,
                  G=wk.G) as plan:
        g, _ = plan.forward(torch.tensor(wk.rho, dtype=torch.float64, device=DEV))
        torch.cuda.synchronize()
        plan.check()
        err = rel_l2(g.cpu().numpy()[idx], ref)
    print("grf_volume 128^3 fp64 p=14 sampled rel L2 %.3e" % err)
    assert err <= 1e-6
