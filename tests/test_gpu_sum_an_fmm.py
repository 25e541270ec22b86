"""SUM-AN in FMM mode (Sec. 2.1 closed-form voxels, Sec. 2.3 FMM): the
voxels next to each observer integrated in closed form, the rest of the near
field by the midpoint rule with a uniform cube's l = 4 term, the far field
from multipole expansions of the exact voxel integrals.  Checked element by
element against the FP64 oracle's closed-form sum (every voxel integrated
exactly): mixed precision <= 1e-5, FP64 <= 1e-6 (relative L2), observers
inside the grid (voxel centres, corners and faces included) and outside it,
and on the 16^3 prism model against the Table-10-pinned prism formula."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1107_5951_gb300 as pkg  # noqa: E402
from oracle import direct  # noqa: E402
from paper_1107_5951_gb300 import gf, workloads as wl  # noqa: E402

DEV = "cuda:0"
BARS = {"mixed": 1e-5, "fp64": 1e-6}


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def run(grid, rho, obs, precision, p, B=1):
    xi, w = wl.gauss_rule(1)
    o = torch.tensor(obs, dtype=torch.float64, device=DEV)
    with pkg.Plan(grid.n, grid.origin, grid.h, xi, w, o, mode="fmm", precision=precision, p=p, max_batch=B,
                  G=0.5, voxels="closed_form") as plan:
        assert plan.info.leaf_vox == 4 and plan.info.L >= 3
        g, gz = plan.forward(torch.tensor(rho, dtype=torch.float32 if precision == "mixed" else torch.float64,
                                          device=DEV), want_gz=True)
        torch.cuda.synchronize()
        plan.check()
        return g.cpu().numpy(), gz.cpu().numpy()


def random_case(seed, n=(28, 24, 21), h=2.0, n_obs=500):
    rng = np.random.default_rng(seed)
    grid = wl.Grid(n, (-7.0, 3.0, -40.0), (h, h, h))
    rho = rng.normal(1.0, 1.0, size=grid.shape_zyx)
    lo = np.array(grid.origin)
    hi = lo + np.array(n) * h
    obs = [rng.uniform(lo - 6.0, hi + 6.0, size=(n_obs, 3)),   # inside and around the grid
           wl.voxel_centres(grid)[rng.choice(grid.nvox, 100, replace=False)],
           lo + h * rng.integers(0, np.array(n) + 1, size=(40, 3)),                  # lattice corners
           lo + h * (rng.integers(0, np.array(n), size=(40, 3)) + np.array([0.5, 0.5, 0.0]))]   # faces
    return grid, rho, np.concatenate(obs)


@pytest.mark.parametrize("precision,p", [("mixed", 12), ("fp64", 14)])
@pytest.mark.parametrize("seed", [1, 2])
def test_sum_an_fmm_matches_the_closed_form_oracle(precision, p, seed):
    grid, rho, obs = random_case(seed)
    if precision == "mixed":
        rho = rho.astype(np.float32).astype(np.float64)   # the densities the GPU reads
    ref = direct.forward_analytic(grid.n, grid.origin, grid.h, rho, obs, 0.5)
    g, gz = run(grid, rho, obs, precision, p)
    assert np.all(np.isfinite(g))
    assert np.array_equal(gz, g[:, 2])
    err = rel_l2(g, ref)
    print("SUM-AN FMM %s p=%d seed %d rel L2 %.3e" % (precision, p, seed, err))
    assert err <= BARS[precision]


def test_sum_an_fmm_batch_equals_single():
    grid, rho, obs = random_case(3, n=(16, 16, 16), n_obs=200)
    rng = np.random.default_rng(4)
    rhos = np.stack([rho, rng.normal(size=rho.shape)])
    g2, _ = run(grid, rhos, obs, "fp64", 10, B=2)
    for bb in range(2):
        g1, _ = run(grid, rhos[bb], obs, "fp64", 10)
        assert np.array_equal(g1, g2[bb])


@pytest.mark.parametrize("precision,p", [("mixed", 12), ("fp64", 14)])
def test_sum_an_fmm_prism_model(precision, p):
    """16^3 voxels of 1 km, a constant +300 kg/m^3 prism on voxels
    [4,12) x [4,12) x [6,10) and 64 x 64 stations 100 m above: integrated
    voxel by voxel in closed form it is the field of the whole prism, which
    the Table 10 formula gives."""
    grid = wl.Grid((16, 16, 16), (0.0, 0.0, -16000.0), (1000.0, 1000.0, 1000.0))
    rho = np.zeros(grid.shape_zyx)
    rho[6:10, 4:12, 4:12] = 300.0
    obs = wl.station_plane(0.0, 16000.0, 0.0, 16000.0, 64, 64, 100.0)
    ref = direct.prism_gz((4000.0, 4000.0, -10000.0), (12000.0, 12000.0, -6000.0), 300.0, 0.5, obs)
    _, gz = run(grid, rho, obs, precision, p)
    err = rel_l2(gz, ref)
    print("SUM-AN FMM prism model %s rel L2 %.3e" % (precision, err))
    assert err <= BARS[precision]


def test_sum_an_fmm_has_no_adjoint():
    grid, rho, obs = random_case(5, n=(8, 8, 8), n_obs=20)
    xi, w = wl.gauss_rule(1)
    o = torch.tensor(obs, dtype=torch.float64, device=DEV)
    with pkg.Plan(grid.n, grid.origin, grid.h, xi, w, o, mode="fmm", precision="fp64", p=8,
                  voxels="closed_form") as plan:
        with pytest.raises(gf.GfError) as e:
            plan.adjoint(torch.zeros(len(obs), dtype=torch.float64, device=DEV))
        assert e.value.status == gf.GF_ERR_UNSUPPORTED
