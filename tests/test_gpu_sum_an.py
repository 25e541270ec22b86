"""SUM-AN on the GPU (direct mode, FP64, every voxel integrated in closed
form, Sec. 2.1) against the FP64 CPU oracle's per-voxel closed-form sum and
its transpose, element by element, and against the prism formula that
Table 10 pins.  The kernels regroup the voxels' corners onto the corner
lattice, so agreement is to rounding, not bit for bit: bar 1e-12 (the
direct-mode FP64 bar; measured 1e-15 to 9e-14)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1107_5951_gb300 as pkg  # noqa: E402
from oracle import direct  # noqa: E402
from paper_1107_5951_gb300 import workloads as wl  # noqa: E402

DEV = "cuda:0"
TOL = 1e-12


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def _case(seed, n, n_obs, B=1, h=(0.5, 0.75, 1.0), origin=(-1.0, 0.5, -2.0)):
    rng = np.random.default_rng(seed)
    rho = rng.normal(size=(B, n[2], n[1], n[0]))
    lo, hi = np.array(origin), np.array(origin) + np.array(n) * np.array(h)
    obs = np.concatenate([rng.uniform(lo - 2.0, hi + 2.0, size=(n_obs, 3)), rng.uniform(lo, hi, size=(4, 3))])
    obs[-1] = lo + np.array([1, 2, 1]) * np.array(h)             # a lattice corner inside the grid
    obs[-2] = lo + np.array([0.5, 1, 0.25]) * np.array(h)        # on a face between voxels
    return rho, obs, tuple(lo), tuple(h)


def _plan(n, origin, h, obs, B):
    xi, w = wl.gauss_rule(1)
    return pkg.Plan(n, origin, h, xi, w, torch.tensor(obs, dtype=torch.float64, device=DEV), mode="direct",
                    precision="fp64", max_batch=B, G=0.3, voxels="closed_form")


@pytest.mark.parametrize("n,n_obs,B", [((5, 4, 3), 20, 2), ((11, 7, 9), 300, 1), ((1, 1, 1), 3, 1)])
def test_sum_an_forward_matches_oracle(n, n_obs, B):
    """Several 128-corner tiles with a ragged tail, a batch, the one-voxel grid."""
    rho, obs, origin, h = _case(1 + n[0], n, n_obs, B)
    ref = direct.forward_analytic(n, origin, h, rho, obs, 0.3)
    with _plan(n, origin, h, obs, B) as plan:
        g, gz = plan.forward(torch.tensor(rho, device=DEV), want_gz=True)
        torch.cuda.synchronize()
        plan.check()
        g, gz = g.cpu().numpy(), gz.cpu().numpy()
    print("SUM-AN forward %s rel L2 %.3e" % (n, rel_l2(g, ref)))
    assert rel_l2(g, ref) <= TOL
    assert np.array_equal(gz, g[..., 2])


@pytest.mark.parametrize("ncomp", [1, 3])
def test_sum_an_adjoint_matches_oracle(ncomp):
    n = (6, 5, 4)
    rho, obs, origin, h = _case(7, n, 40, 2)
    rng = np.random.default_rng(8)
    r = rng.normal(size=(2, len(obs)) if ncomp == 1 else (2, len(obs), 3))
    ref = direct.adjoint_analytic(n, origin, h, obs, r, 0.3, ncomp=ncomp)
    with _plan(n, origin, h, obs, 2) as plan:
        grad = plan.adjoint(torch.tensor(r, device=DEV), ncomp=ncomp).cpu().numpy()
    print("SUM-AN transpose ncomp=%d rel L2 %.3e" % (ncomp, rel_l2(grad, ref)))
    assert rel_l2(grad, ref) <= TOL


def test_sum_an_prism_model_is_the_closed_form():
    """The 16^3 model of 1 km voxels with a constant-density prism on voxels
    [4, 12) x [4, 12) x [6, 10) and 64 x 64 stations 100 m above: integrated
    voxel by voxel in closed form it is the field of the whole prism (the
    integral is additive), which the Table 10 formula gives."""
    n, h = (16, 16, 16), (1000.0, 1000.0, 1000.0)
    origin = (0.0, 0.0, -16000.0)
    rho = np.zeros((16, 16, 16))
    rho[6:10, 4:12, 4:12] = 300.0
    obs = wl.station_plane(0.0, 16000.0, 0.0, 16000.0, 64, 64, 100.0)
    lo = (4000.0, 4000.0, -10000.0)
    hi = (12000.0, 12000.0, -6000.0)
    ref = direct.prism_gz(lo, hi, 300.0, 0.3, obs)
    with _plan(n, origin, h, obs, 1) as plan:
        _, gz = plan.forward(torch.tensor(rho, device=DEV), want_g=False, want_gz=True)
        gz = gz.cpu().numpy()
    print("SUM-AN prism model rel L2 %.3e" % rel_l2(gz, ref))
    assert rel_l2(gz, ref) <= 1e-12
