"""Serving form: continuous batching of forward solves on several CUDA
streams (gf_server_*).  A request's result must be bit-identical alone, in
any mix of concurrent requests, after its plan was evicted and rebuilt, and
to the plain plan API; and it must meet the precision's error bar against
the FP64 CPU direct-sum oracle (discretised Eq. 1)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1107_5951_gb300 as pkg  # noqa: E402
from oracle import direct  # noqa: E402
from paper_1107_5951_gb300 import workloads as wl  # noqa: E402

H = 250.0
SIDES = (12, 17, 24, 31, 40)


def geometry(n, stations=20):
    grid = wl.Grid((n, n, n), (0.0, 0.0, -n * H), (H, H, H))
    obs = wl.station_plane(0.0, n * H, 0.0, n * H, stations, stations, grid.top)
    xi, w = wl.gauss_rule(1)
    return grid, xi, w, obs


def register_all(srv):
    geo = {}
    for gid, n in enumerate(SIDES):
        grid, xi, w, obs = geometry(n)
        srv.register(gid, grid.n, grid.origin, grid.h, xi, w, obs)
        geo[gid] = (grid, xi, w, obs)
    return geo


def densities(gid, k, dtype=np.float32):
    return wl.periodic_grf(SIDES[gid], H, 2000.0, 150.0, 1000 * gid + k, dtype=dtype)


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("precision,tol", [("mixed", 1e-5), ("fp64", 1e-6)])
def test_alone_equals_in_the_mix_and_meets_oracle(precision, tol):
    p = 12 if precision == "mixed" else 14
    jobs = [(gid, k) for k in range(3) for gid in range(len(SIDES))]
    rhos = {j: densities(*j, dtype=np.float32 if precision == "mixed" else np.float64) for j in jobs}
    # alone: one slot, each request waited for before the next
    alone = {}
    with pkg.Server(slots=1, precision=precision, p=p) as srv:
        register_all(srv)
        for j in jobs:
            gz, _, _ = srv.wait(srv.submit(j[0], rhos[j]))
            alone[j] = gz
    # in the mix: four slots, everything queued at once, geometries interleaved
    with pkg.Server(slots=4, precision=precision, p=p) as srv:
        geo = register_all(srv)
        tickets = {j: srv.submit(j[0], rhos[j]) for j in jobs}
        mixed = {j: srv.wait(t)[0] for j, t in tickets.items()}
        st = srv.stats()
    assert st["completed"] == len(jobs) and st["failed"] == 0
    assert st["graph_launches"] == len(jobs)
    assert 0 < st["p50_ms"] <= st["p99_ms"]
    for j in jobs:
        assert np.array_equal(alone[j], mixed[j]), j
    # the plain plan API gives the same bits
    gid = 3
    grid, xi, w, obs = geo[gid]
    with pkg.Plan(grid.n, grid.origin, grid.h, xi, w, torch.tensor(obs, device="cuda:0"), mode="fmm",
                  precision=precision, p=p) as plan:
        _, gz = plan.forward(torch.tensor(rhos[(gid, 1)], device="cuda:0"), want_g=False, want_gz=True)
        assert np.array_equal(gz.cpu().numpy(), mixed[(gid, 1)])
    # accuracy against the FP64 direct sum
    for gid in (1, 4):
        grid, xi, w, obs = geo[gid]
        want = direct.forward(grid.n, grid.origin, grid.h, xi, w, rhos[(gid, 0)].astype(np.float64), obs,
                              wl.G_PAPER)[:, 2]
        assert rel_l2(mixed[(gid, 0)], want) <= tol


def test_eviction_under_memory_budget_keeps_results():
    """With room for about two plans, cycling through five geometries evicts
    plans least-recently-used first; rebuilt plans give the same bits."""
    grid, xi, w, obs = geometry(SIDES[-1])
    big = pkg.plan_bytes(grid.n, grid.origin, grid.h, xi, w, obs.shape[0], mode="fmm", precision="mixed",
                         p=8) + 4 * SIDES[-1] ** 3 + 32 * obs.shape[0]
    budget = int(2.2 * big)
    jobs = [(gid, 0) for gid in range(len(SIDES))] * 2
    rhos = {j: densities(*j) for j in set(jobs)}
    ref = {}
    with pkg.Server(slots=1, precision="mixed", p=8) as srv:
        register_all(srv)
        for j in set(jobs):
            ref[j] = srv.wait(srv.submit(j[0], rhos[j]))[0]
    with pkg.Server(slots=2, precision="mixed", p=8, mem_budget=budget) as srv:
        register_all(srv)
        tickets = [(j, srv.submit(j[0], rhos[j])) for j in jobs]
        for j, t in tickets:
            gz, _, _ = srv.wait(t)
            assert np.array_equal(gz, ref[j]), j
        st = srv.stats()
    assert st["plans_evicted"] > 0
    assert st["plans_created"] > len(SIDES)
    assert st["resident_bytes"] <= budget


def test_oversize_request_is_refused_and_timeout_reported():
    with pkg.Server(slots=1, precision="mixed", p=8, mem_budget=1 << 20) as srv:
        register_all(srv)
        with pytest.raises(pkg.GfError) as e:
            srv.submit(4, densities(4, 0))
        assert e.value.status == 7   # GF_ERR_BUSY
    with pkg.Server(slots=1, precision="mixed", p=8) as srv:
        register_all(srv)
        t = srv.submit(4, densities(4, 0))
        with pytest.raises(pkg.GfError) as e:
            srv.wait(t, timeout_ms=0.0)   # the plan is still being built
        assert e.value.status == 5   # GF_ERR_TIMEOUT
        gz, _, lat = srv.wait(t)
        assert lat > 0 and np.all(np.isfinite(gz))


def test_device_and_pinned_buffers_give_the_same_bits():
    with pkg.Server(slots=2, precision="mixed", p=10) as srv:
        register_all(srv)
        rho = densities(2, 5)
        gz_host, g_host, _ = srv.wait(srv.submit(2, rho, want_g=True))
        pinned = torch.from_numpy(rho).pin_memory()
        gz_pin, g_pin, _ = srv.wait(srv.submit(2, pinned, want_g=True))
        dev = torch.from_numpy(rho).to("cuda:0")
        gz_dev, g_dev, _ = srv.wait(srv.submit(2, dev, want_g=True))
        torch.cuda.synchronize()
    assert np.array_equal(gz_host, gz_pin.numpy()) and np.array_equal(gz_host, gz_dev.cpu().numpy())
    assert np.array_equal(g_host, g_pin.numpy()) and np.array_equal(g_host, g_dev.cpu().numpy())
    assert np.array_equal(g_host[:, 2], gz_host)


@pytest.mark.parametrize("precision,tol", [("mixed", 1e-5), ("fp64", 1e-6)])
def test_serving_sides_up_to_256(precision, tol):
    """Requests of the serving workload's full size range (32^3 to 256^3
    voxels of 250 m, 256^2 stations), queued together on four slots: each
    meets the oracle on sampled stations and equals the plain plan API bit
    for bit."""
    p = 12 if precision == "mixed" else 14
    sides = (32, 91, 160, 256)
    dtype = np.float32 if precision == "mixed" else np.float64
    geo, rhos = {}, {}
    with pkg.Server(slots=4, precision=precision, p=p) as srv:
        for gid, n in enumerate(sides):
            grid, xi, w, obs = geometry(n, stations=256)
            srv.register(100 + gid, grid.n, grid.origin, grid.h, xi, w, obs)
            geo[gid] = (grid, xi, w, obs)
            rhos[gid] = wl.periodic_grf(n, H, 2000.0, 150.0, 77 + gid, dtype=dtype)
        tickets = {gid: srv.submit(100 + gid, rhos[gid]) for gid in geo}
        got = {gid: srv.wait(t)[0] for gid, t in tickets.items()}
    rng = np.random.default_rng(19)
    for gid, (grid, xi, w, obs) in geo.items():
        idx = np.sort(rng.choice(len(obs), 48, replace=False))
        ref = direct.forward(grid.n, grid.origin, grid.h, xi, w, rhos[gid].astype(np.float64), obs[idx],
                             wl.G_PAPER)[:, 2]
        assert rel_l2(got[gid][idx], ref) <= tol, sides[gid]
        with pkg.Plan(grid.n, grid.origin, grid.h, xi, w, torch.tensor(obs, dtype=torch.float64, device="cuda:0"),
                      mode="fmm", precision=precision, p=p, G=wl.G_PAPER) as plan:
            _, gz = plan.forward(torch.tensor(rhos[gid], device="cuda:0"), want_g=False, want_gz=True)
            torch.cuda.synchronize()
            assert np.array_equal(gz.cpu().numpy(), got[gid]), sides[gid]
