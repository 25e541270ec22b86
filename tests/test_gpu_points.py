"""Weighted point sources on the GPU (gf_hex_sources, gf_plan_create_points):
the quadrature points of deformed hexahedral cells (the general summation of
Sec. 2.1: trilinear maps, the Jacobian of each cell at the rule's nodes) and
scattered density points carrying the volumes of their Voronoi cells
(Sec. 4), compared element by element with the FP64 oracle's direct sums
(oracle.direct.hex_sources, forward_points, forward_hex).  Bars as for voxel
grids: relative L2 <= 1e-12 (FP64 direct), <= 1e-5 (mixed), <= 1e-6 (FP64
FMM, p = 14)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1107_5951_gb300 as pkg  # noqa: E402
from oracle import direct  # noqa: E402
from paper_1107_5951_gb300 import gf, workloads as wl  # noqa: E402

DEV = "cuda:0"
BARS = {("direct", "fp64"): 1e-12, ("direct", "mixed"): 1e-5, ("fmm", "fp64"): 1e-6, ("fmm", "mixed"): 1e-5}
P = {"fp64": 14, "mixed": 12}


def t(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def points_case(seed, n=3000):
    """Scattered points in a 2 km x 1.5 km x 1 km box with Voronoi volumes,
    densities N(2500, 300); observers inside, around and above the box."""
    lo, hi = np.array([-1000.0, 200.0, -1200.0]), np.array([1000.0, 1700.0, -200.0])
    x = wl.scattered_points(n, lo, hi, seed)
    a = wl.voronoi_volumes(x, lo, hi)
    rng = np.random.default_rng(seed + 100)
    rho = rng.normal(2500.0, 300.0, size=n)
    obs = np.concatenate([rng.uniform(lo - 300.0, hi + 300.0, size=(300, 3)),
                          np.column_stack([rng.uniform(lo[0], hi[0], 64), rng.uniform(lo[1], hi[1], 64),
                                           np.full(64, 50.0)])])
    return x, a, 1, rho, obs


def hex_case(nx=10, ny=10, nz=5, stations=8, npts=2):
    wk = wl.topo_workload(nx, ny, nz, stations, npts)
    x, a = direct.hex_sources(wk["verts"], wk["xi"], wk["w"])
    return wk, x, a


def run(x, a, per_cell, rho, obs, mode, precision, B=1, G=wl.G_PAPER):
    dt = torch.float32 if precision == "mixed" else torch.float64
    with pkg.PointsPlan(t(x), t(a), t(obs), per_cell=per_cell, mode=mode, precision=precision, p=P[precision],
                        max_batch=B, G=G) as plan:
        assert plan.info.n_sources == len(a)
        g, gz = plan.forward(torch.tensor(rho, dtype=dt, device=DEV), want_gz=True)
        torch.cuda.synchronize()
        plan.check()
        return g.cpu().numpy(), gz.cpu().numpy(), plan.info


def test_hex_sources_match_the_oracle():
    """Node images and |det J| weights of warped brick cells and of a
    terrain-following mesh, 1, 8 and 27 nodes per cell."""
    meshes = [wl.hex_brick_mesh((7, 5, 4), (-100.0, 20.0, -300.0), (150.0, 140.0, -20.0), warp=0.15),
              wl.topo_mesh(6, 5, 4)[0]]
    for verts in meshes:
        ext = float(np.ptp(verts.reshape(-1, 3), axis=0).max())
        for npts in (1, 2, 3):
            xi, w = wl.gauss_rule(npts)
            x, a = pkg.hex_sources(t(verts), xi, w)
            torch.cuda.synchronize()
            xr, ar = direct.hex_sources(verts, xi, w)
            assert np.abs(x.cpu().numpy() - xr).max() <= 1e-14 * ext
            assert np.abs(a.cpu().numpy() - ar).max() <= 1e-13 * ar.max()
    # a brick that is not warped: every cell's weights sum to its volume
    verts = wl.hex_brick_mesh((3, 2, 2), (0.0, 0.0, 0.0), (3.0, 4.0, 2.0))
    _, a = pkg.hex_sources(t(verts), *wl.gauss_rule(2))
    assert np.allclose(a.cpu().numpy().reshape(-1, 8).sum(axis=1), 2.0, rtol=1e-14, atol=0)


def test_hex_sources_mixed_within_their_bound():
    """The FP32 form (fixed-point corners, image relative to the first
    corner): positions within 1e-6 of the cell extent, weights within 1e-6
    relative, on warped bricks far from the origin and on the terrain mesh."""
    meshes = [wl.hex_brick_mesh((7, 5, 4), (4.0e5, 6.2e6, -3000.0), (4.3e5, 6.23e6, 200.0), warp=0.2),
              wl.topo_mesh(12, 10, 6)[0]]
    for verts in meshes:
        cell = float(np.ptp(verts, axis=1).max())
        for npts in (1, 2, 3):
            xi, w = wl.gauss_rule(npts)
            x, a = pkg.hex_sources(t(verts), xi, w, precision="mixed")
            torch.cuda.synchronize()
            xr, ar = direct.hex_sources(verts, xi, w)
            assert np.abs(x.cpu().numpy() - xr).max() <= 1e-6 * cell
            assert np.abs(a.cpu().numpy() / ar - 1.0).max() <= 1e-6


@pytest.mark.parametrize("mode,precision", [("direct", "fp64"), ("direct", "mixed"), ("fmm", "fp64"),
                                            ("fmm", "mixed")])
@pytest.mark.parametrize("seed", [1, 2])
def test_scattered_points_match_the_oracle(mode, precision, seed):
    x, a, per_cell, rho, obs = points_case(seed)
    if precision == "mixed":
        rho = rho.astype(np.float32).astype(np.float64)   # the densities the GPU reads
    ref = direct.forward_points(x, a, per_cell, rho, obs, wl.G_PAPER)
    g, gz, info = run(x, a, per_cell, rho, obs, mode, precision)
    err = rel_l2(g, ref)
    print("points seed %d %s %s: rel L2 %.3e" % (seed, mode, precision, err))
    assert err <= BARS[(mode, precision)]
    assert rel_l2(gz, ref[:, 2]) <= 2 * BARS[(mode, precision)]
    if mode == "fmm":
        assert 0 < info.near_pairs < len(obs) * len(a)


@pytest.mark.parametrize("mode,precision", [("direct", "fp64"), ("direct", "mixed"), ("fmm", "fp64"),
                                            ("fmm", "mixed")])
def test_deformed_hexahedra_match_the_oracle(mode, precision):
    """Terrain-following cells, 8 Gauss nodes per cell, stations draped
    over the topography: the GPU's own gf_hex_sources feeds the plan."""
    wk, _, _ = hex_case()
    rho = wk["rho"].astype(np.float32).astype(np.float64) if precision == "mixed" else wk["rho"]
    ref = direct.forward_hex(wk["verts"], wk["xi"], wk["w"], rho, wk["obs"], wk["G"])
    x, a = pkg.hex_sources(t(wk["verts"]), wk["xi"], wk["w"], precision=precision)
    dt = torch.float32 if precision == "mixed" else torch.float64
    with pkg.PointsPlan(x, a, t(wk["obs"]), per_cell=len(wk["w"]), mode=mode, precision=precision,
                        p=P[precision], G=wk["G"]) as plan:
        g, _ = plan.forward(torch.tensor(rho, dtype=dt, device=DEV))
        torch.cuda.synchronize()
        plan.check()
    err = rel_l2(g.cpu().numpy(), ref)
    print("hex %s %s: rel L2 %.3e" % (mode, precision, err))
    assert err <= BARS[(mode, precision)]


@pytest.mark.parametrize("mode", ["direct", "fmm"])
def test_batched_densities_and_float32_input(mode):
    """B density vectors in one call equal B single calls; per_cell > 1
    maps source s to density s // per_cell."""
    x, a, _, _, obs = points_case(3, n=2400)
    rng = np.random.default_rng(5)
    rho = rng.normal(1.0, 1.0, size=(3, 600))
    ref = direct.forward_points(x, a, 4, rho, obs, 1.0)
    with pkg.PointsPlan(t(x), t(a), t(obs), per_cell=4, mode=mode, precision="fp64", p=14, max_batch=3,
                        G=1.0) as plan:
        g, _ = plan.forward(t(rho))
        g1, _ = plan.forward(t(rho[1]))
        g32, _ = plan.forward(torch.tensor(rho, dtype=torch.float32, device=DEV))
        torch.cuda.synchronize()
        plan.check()
    bar = BARS[(mode, "fp64")]
    for b in range(3):
        assert rel_l2(g[b].cpu().numpy(), ref[b]) <= bar
    assert np.array_equal(g1.cpu().numpy(), g[1].cpu().numpy())
    ref32 = direct.forward_points(x, a, 4, rho.astype(np.float32).astype(np.float64), obs, 1.0)
    assert rel_l2(g32.cpu().numpy(), ref32) <= bar


@pytest.mark.parametrize("mode,precision", [("direct", "fp64"), ("direct", "mixed"), ("fmm", "fp64"),
                                            ("fmm", "mixed")])
def test_degenerate_layouts(mode, precision):
    """No sources (zero field), no observers, one source, coincident
    observer and source (the pair contributes nothing), every source on one
    plane (a flat layer), and observers far above a small cloud."""
    rng = np.random.default_rng(11)
    bar = BARS[(mode, precision)]
    dt = torch.float32 if precision == "mixed" else torch.float64
    # no sources
    obs = rng.uniform(-1.0, 1.0, size=(40, 3))
    with pkg.PointsPlan(t(np.zeros((0, 3))), t(np.zeros(0)), t(obs), mode=mode, precision=precision,
                        p=P[precision], G=1.0) as plan:
        g, _ = plan.forward(torch.zeros(0, dtype=dt, device=DEV))
        torch.cuda.synchronize()
        assert np.all(g.cpu().numpy() == 0.0)
    cases = []
    # one source, observers around it (one of them on it)
    x1 = np.array([[0.3, -0.2, 0.1]])
    cases.append((x1, np.array([2.0]), np.concatenate([rng.uniform(-2, 2, size=(30, 3)), x1])))
    # sources on the plane z = 0 (a flat layer), observers above and within it
    xf = np.column_stack([rng.uniform(0, 100, 1500), rng.uniform(0, 60, 1500), np.zeros(1500)])
    cases.append((xf, np.full(1500, 4.0), np.column_stack([rng.uniform(-10, 110, 200), rng.uniform(-10, 70, 200),
                                                           rng.choice([0.0, 0.5, 5.0, 30.0], 200)])))
    # a small cloud and observers 50 cloud diameters away (a deep tree)
    xc = rng.uniform(0.0, 1.0, size=(500, 3))
    cases.append((xc, np.full(500, 2e-3), np.concatenate([rng.uniform(0.0, 1.0, size=(20, 3)),
                                                          rng.uniform(-50.0, 50.0, size=(40, 3)) + [0, 0, 50.0]])))
    # observers placed exactly on sources
    xs = rng.uniform(-5, 5, size=(800, 3))
    cases.append((xs, np.full(800, 0.1), np.concatenate([xs[::40], rng.uniform(-6, 6, size=(50, 3))])))
    for x, a, o in cases:
        rho = rng.normal(1.0, 0.3, size=len(a))
        if precision == "mixed":
            rho = rho.astype(np.float32).astype(np.float64)
        ref = direct.forward_points(x, a, 1, rho, o, 1.0)
        g, _, _ = run(x, a, 1, rho, o, mode, precision, G=1.0)
        assert np.all(np.isfinite(g))
        assert rel_l2(g, ref) <= bar, (len(a), rel_l2(g, ref))
    # no observers
    with pkg.PointsPlan(t(xs), t(np.ones(800)), t(np.zeros((0, 3))), mode=mode, precision=precision,
                        p=P[precision]) as plan:
        g, _ = plan.forward(torch.ones(800, dtype=dt, device=DEV))
        torch.cuda.synchronize()
        assert g.shape == (0, 3)


def test_point_plans_refuse_adjoint_and_source_parts():
    x, a, _, rho, obs = points_case(1, n=500)
    with pkg.PointsPlan(t(x), t(a), t(obs), mode="fmm", precision="mixed", p=8) as plan:
        with pytest.raises(gf.GfError) as e:
            plan.adjoint(t(np.ones(len(obs))))
        assert e.value.status == gf.GF_ERR_UNSUPPORTED
        with pytest.raises(gf.GfError) as e:
            plan.set_source_part(0, 2)
        assert e.value.status == gf.GF_ERR_UNSUPPORTED


def test_nonfinite_density_is_reported():
    x, a, _, rho, obs = points_case(2, n=500)
    rho = rho.copy()
    rho[17] = np.nan
    for mode in ("direct", "fmm"):
        with pkg.PointsPlan(t(x), t(a), t(obs), mode=mode, precision="mixed", p=8) as plan:
            plan.forward(torch.tensor(rho, dtype=torch.float32, device=DEV))
            with pytest.raises(gf.GfError) as e:
                plan.check()
            assert e.value.status == gf.GF_ERR_DEVICE_CHECK


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_large_scattered_cloud_sampled(precision):
    """Two million scattered points (unit volumes), FMM: 256 observers
    sampled out of 65536 checked against the oracle's direct sum over every
    source."""
    n = 1 << 21
    lo, hi = np.zeros(3), np.array([4000.0, 3000.0, 1000.0])
    x = wl.scattered_points(n, lo, hi, seed=21)
    a = np.full(n, np.prod(hi - lo) / n)
    rng = np.random.default_rng(22)
    rho = rng.normal(2600.0, 200.0, size=n)
    if precision == "mixed":
        rho = rho.astype(np.float32).astype(np.float64)
    obs = np.column_stack([rng.uniform(0, 4000, 65536), rng.uniform(0, 3000, 65536), rng.uniform(-200, 1200, 65536)])
    g, _, info = run(x, a, 1, rho, obs, "fmm", precision)
    pick = rng.choice(len(obs), 256, replace=False)
    ref = direct.forward_points(x, a, 1, rho, obs[pick], wl.G_PAPER)
    err = rel_l2(g[pick], ref)
    print("2M points %s: rel L2 %.3e, L = %d" % (precision, err, info.L))
    assert err <= BARS[("fmm", precision)]
