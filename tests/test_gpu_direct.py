"""Direct mode (Sec. 2.1 summation, every pair) on the GPU against the FP64
CPU oracle, element by element.  Bar: relative L2 <= 1e-12 in FP64, 1e-5 in
mixed precision."""
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


def run(wk, precision, rho=None, gz=True, B=None):
    rho = wk.rho if rho is None else rho
    obs = torch.tensor(wk.obs, dtype=torch.float64, device=DEV)
    r = torch.tensor(rho, device=DEV)
    nb = 1 if r.dim() == 3 else r.shape[0]
    with pkg.Plan(wk.grid.n, wk.grid.origin, wk.grid.h, wk.xi, wk.w, obs, mode="direct",
                  precision=precision, max_batch=nb, G=wk.G) as plan:
        g, z = plan.forward(r, want_gz=gz)
        torch.cuda.synchronize()
        return g.cpu().numpy(), (z.cpu().numpy() if z is not None else None)


CASES = [
    dict(seed=1, n=(5, 4, 3), npts=1, n_obs=17),
    dict(seed=2, n=(7, 3, 6), npts=2, n_obs=300),     # 1008 sources: several 256-tiles + ragged
    dict(seed=3, n=(1, 1, 1), npts=1, n_obs=1),       # smallest problem
    dict(seed=4, n=(9, 8, 7), npts=3, n_obs=1000),    # 27-point rule, ragged tiles
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "n%dx%dx%d_q%d_m%d" % (c["n"] + (c["npts"], c["n_obs"])))
def test_direct_fp64_matches_oracle(case):
    wk = wl.random_small(case["seed"], n=case["n"], npts=case["npts"], n_obs=case["n_obs"])
    ref = direct.forward(wk.grid.n, wk.grid.origin, wk.grid.h, wk.xi, wk.w, wk.rho, wk.obs, wk.G)
    g, gz = run(wk, "fp64")
    assert rel_l2(g, ref) <= 1e-12
    assert np.array_equal(gz, g[:, 2])


@pytest.mark.parametrize("case", CASES[:2] + CASES[3:], ids=lambda c: "seed%d" % c["seed"])
def test_direct_mixed_matches_oracle(case):
    wk = wl.random_small(case["seed"], n=case["n"], npts=case["npts"], n_obs=case["n_obs"])
    ref = direct.forward(wk.grid.n, wk.grid.origin, wk.grid.h, wk.xi, wk.w, wk.rho, wk.obs, wk.G)
    g, _ = run(wk, "mixed")
    assert rel_l2(g, ref) <= 1e-5


def test_direct_coincident_observers_skip_self_pair():
    """Observers exactly at voxel centres with the midpoint rule: the
    coincident source contributes nothing (no inf/NaN), as in the oracle."""
    wk = wl.random_small(9, n=(6, 5, 4), npts=1, n_obs=1, h=(1.0, 1.0, 1.0), origin=(0.0, 0.0, -4.0))
    wk.obs = wl.voxel_centres(wk.grid)
    ref = direct.forward(wk.grid.n, wk.grid.origin, wk.grid.h, wk.xi, wk.w, wk.rho, wk.obs, wk.G)
    for prec, tol in (("fp64", 1e-12), ("mixed", 1e-5)):
        g, _ = run(wk, prec)
        assert np.all(np.isfinite(g))
        assert rel_l2(g, ref) <= tol


def test_direct_batch_and_float32_density():
    wk = wl.random_small(12, n=(6, 5, 4), npts=2, n_obs=77, B=3)
    ref = direct.forward(wk.grid.n, wk.grid.origin, wk.grid.h, wk.xi, wk.w, wk.rho, wk.obs, wk.G)
    g, _ = run(wk, "fp64")
    for b in range(3):
        assert rel_l2(g[b], ref[b]) <= 1e-12
    rho32 = wk.rho.astype(np.float32)
    ref32 = direct.forward(wk.grid.n, wk.grid.origin, wk.grid.h, wk.xi, wk.w, rho32.astype(np.float64),
                           wk.obs, wk.G)
    g32, _ = run(wk, "fp64", rho=rho32)
    assert rel_l2(g32, ref32) <= 1e-12


def test_direct_fp64_prism_noise_16cubed():
    """The 16^3 x 1 km prism-plus-noise workload (2x2x2 Gauss, 32768
    sources, 64x64 stations 100 m above the top), in full."""
    wk = wl.fp64_prism_noise()
    ref = direct.forward(wk.grid.n, wk.grid.origin, wk.grid.h, wk.xi, wk.w, wk.rho, wk.obs, wk.G)
    g, gz = run(wk, "fp64")
    assert rel_l2(g, ref) <= 1e-12
    assert rel_l2(gz, ref[:, 2]) <= 1e-12
    gm, _ = run(wk, "mixed")
    assert rel_l2(gm, ref) <= 1e-5


@pytest.mark.parametrize("ncomp", [1, 3])
def test_direct_adjoint_matches_oracle(ncomp):
    wk = wl.random_small(13, n=(6, 5, 4), npts=2, n_obs=300)
    rng = np.random.default_rng(3)
    r = rng.normal(size=(2, wk.n_obs) if ncomp == 1 else (2, wk.n_obs, 3))
    ref = direct.adjoint(wk.grid.n, wk.grid.origin, wk.grid.h, wk.xi, wk.w, wk.obs, r, wk.G, ncomp=ncomp)
    obs = torch.tensor(wk.obs, dtype=torch.float64, device=DEV)
    with pkg.Plan(wk.grid.n, wk.grid.origin, wk.grid.h, wk.xi, wk.w, obs, mode="direct",
                  precision="fp64", max_batch=2, G=wk.G) as plan:
        grad = plan.adjoint(torch.tensor(r, device=DEV), ncomp=ncomp).cpu().numpy()
    assert rel_l2(grad, ref) <= 1e-12


def test_invalid_forward_arguments_on_gpu():
    wk = wl.random_small(1)
    obs = torch.tensor(wk.obs, dtype=torch.float64, device=DEV)
    with pkg.Plan(wk.grid.n, wk.grid.origin, wk.grid.h, wk.xi, wk.w, obs, mode="direct") as plan:
        with pytest.raises(pkg.GfError):
            plan.forward(torch.zeros((2,) + wk.grid.shape_zyx, dtype=torch.float64, device=DEV))  # B > max_batch
        with pytest.raises(TypeError):
            plan.forward(torch.zeros(wk.grid.shape_zyx, dtype=torch.int32, device=DEV))
