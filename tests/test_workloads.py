"""The seeded synthetic inputs (paper_1107_5951_gb300/workloads.py) follow
the recipes they state: quadrature rules, cell-centred stations and voxel
centres, exponential-covariance random fields (standard deviation and
correlation length), the layered model, the serving stream's sizes and
arrivals, and determinism under the seeds."""
import numpy as np
import pytest

from paper_1107_5951_gb300 import workloads as wl


def test_gauss_rules():
    xi, w = wl.gauss_rule(1)
    assert xi.shape == (1, 3) and np.all(xi == 0.0) and w.sum() == pytest.approx(8.0)
    xi, w = wl.gauss_rule(2)
    assert xi.shape == (8, 3) and w.sum() == pytest.approx(8.0)
    assert np.allclose(np.abs(xi), 1.0 / np.sqrt(3.0))
    assert np.all(np.diff(xi[:2, 0]) > 0) and xi[0, 1] == xi[1, 1]   # x fastest


def test_stations_and_voxel_centres():
    st = wl.station_plane(0.0, 100.0, 0.0, 50.0, 4, 2, 7.0)
    assert st.shape == (8, 3) and np.all(st[:, 2] == 7.0)
    assert st[0, 0] == pytest.approx(12.5) and st[1, 0] == pytest.approx(37.5) and st[4, 1] == pytest.approx(37.5)
    g = wl.Grid((3, 2, 2), (1.0, 2.0, -4.0), (2.0, 1.0, 2.0))
    vc = wl.voxel_centres(g)
    assert vc.shape == (12, 3)
    assert np.allclose(vc[0], (2.0, 2.5, -3.0)) and np.allclose(vc[1], (4.0, 2.5, -3.0))


def _lag_corr(f, lag, axis):
    a = np.moveaxis(f, axis, 0)
    x, y = a[:-lag].ravel(), a[lag:].ravel()
    x = x - x.mean()
    y = y - y.mean()
    return float((x * y).mean() / np.sqrt((x * x).mean() * (y * y).mean()))


def test_exponential_covariance_field():
    n, h, ell, sigma = 32, 250.0, 2000.0, 150.0
    fields = [wl.exp_cov_grf(n, h, ell, sigma, seed) for seed in range(4)]
    assert np.array_equal(fields[0], wl.exp_cov_grf(n, h, ell, sigma, 0))
    assert not np.array_equal(fields[0], fields[1])
    sd = np.mean([f.std() for f in fields])
    assert sd == pytest.approx(sigma, rel=0.25)
    for lag, tol in ((1, 0.05), (4, 0.12)):
        c = np.mean([_lag_corr(f, lag, ax) for f in fields for ax in range(3)])
        assert c == pytest.approx(np.exp(-lag * h / ell), abs=tol)


def test_periodic_field_has_the_requested_sigma():
    f = wl.periodic_grf(24, 250.0, 2000.0, 150.0, seed=9)
    assert f.dtype == np.float32 and f.shape == (24, 24, 24)
    assert float(f.std()) == pytest.approx(150.0, rel=1e-4)
    assert _lag_corr(f.astype(np.float64), 1, 0) > 0.6


def test_layered_model():
    wk = wl.layered_scale(n=30, h=1000.0, seed=3, stations=4)
    rho = wk.rho
    base = {2600.0, 2700.0, 2900.0}
    bg = np.isin(rho, list(base))
    assert bg.mean() > 0.5                     # ellipsoids cover a minority of the box
    assert np.all(np.isin(np.unique(rho), [b + k * 400.0 for b in base for k in (-1, 0, 1, 2)]))
    assert rho[0, 0, 0] in (2900.0, 3300.0, 2500.0) and rho[-1, 0, 0] in (2600.0, 3000.0, 2200.0)
    assert wk.obs.shape == (16, 3) and np.all(wk.obs[:, 2] == wk.grid.top)


def test_prism_noise_anomaly():
    wk = wl.fp64_prism_noise(seed=1)
    assert wk.rho.shape == (16, 16, 16)
    assert wk.rho[6:10, 4:12, 4:12].mean() == pytest.approx(300.0, abs=3.0)
    outside = np.ones_like(wk.rho, dtype=bool)
    outside[6:10, 4:12, 4:12] = False
    assert abs(wk.rho[outside].mean()) < 1.0 and wk.rho[outside].std() == pytest.approx(10.0, rel=0.05)
    assert wk.obs.shape == (4096, 3) and np.all(wk.obs[:, 2] == 100.0)


def test_serving_stream_sizes_and_arrivals():
    reqs = wl.serving_stream(n_requests=400, seed=4)
    sides = np.array([r["grid"].n[0] for r in reqs])
    assert sides.min() >= 32 and sides.max() <= 256
    assert np.mean(np.log(sides)) == pytest.approx(0.5 * (np.log(32) + np.log(256)), abs=0.12)
    t = np.array([r["arrival_s"] for r in reqs])
    assert t[0] == 0.0 and np.all(np.diff(t) >= 0.0)
    assert np.mean(np.diff(t)) == pytest.approx(0.01, rel=0.2)     # 100 Hz Poisson arrivals
    assert reqs[3]["obs"].shape == (256 * 256, 3)


def test_serving_density_window_wraps_the_shared_field():
    field = wl.periodic_grf(16, 250.0, 2000.0, 150.0, seed=1)
    req = {"grid": wl.Grid((8, 8, 8), (0.0, 0.0, -2000.0), (250.0,) * 3), "seed": 77}
    w = wl.serving_density(req, field)
    off = np.random.Generator(np.random.PCG64(77)).integers(0, 16, size=3)
    idx = [(o + np.arange(8)) % 16 for o in off]
    assert np.array_equal(w, field[np.ix_(idx[0], idx[1], idx[2])])


def test_adjoint_batch():
    wk = wl.adjoint_batch(n=12, stations=8, batch=3)
    assert wk.rho.shape == (3, 12, 12, 12) and wk.extra["hidden"].shape == (12, 12, 12)
    assert not np.array_equal(wk.rho[0], wk.rho[1])
    assert np.array_equal(wk.rho[1], wl.exp_cov_grf(12, 250.0, 2000.0, 150.0, 7))


def test_voronoi_volumes_tile_the_box():
    """The scattered-point volumes (Sec. 4) partition the box: all positive,
    summing to its volume."""
    pytest.importorskip("scipy")
    lo, hi = (0.0, 0.0, -2.0), (3.0, 2.0, 0.0)
    pts = wl.scattered_points(400, lo, hi, seed=3)
    vol = wl.voronoi_volumes(pts, lo, hi)
    assert np.all(vol > 0)
    assert vol.sum() == pytest.approx(12.0, rel=1e-10)


def test_topography_workload_recipe():
    """Terrain-following cells: columns from the flat bottom to the seeded
    surface; stations 50 m above that surface."""
    d = wl.topo_workload(nx=8, ny=6, nz=4, stations=5)
    assert d["verts"].shape == (8 * 6 * 4, 8, 3)
    assert np.allclose(d["verts"][:, :, 2].min(), -8000.0)
    surf = wl.topo_surface(d["obs"][:, 0], d["obs"][:, 1], 16000.0, 16000.0, 800.0, 6)
    assert np.allclose(d["obs"][:, 2] - surf, 50.0)
    assert d["rho"].shape == (8 * 6 * 4,) and np.all(np.abs(d["rho"] - 2670.0) <= 300.0)
