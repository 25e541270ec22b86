"""Seeded synthetic inputs shaped like the paper's workloads.

This module generates INPUTS only -- voxel grids, densities, quadrature rules
and observer sets -- and holds none of the forward model's arithmetic.  It is
the one module that both the CUDA library's tests/benchmarks and the CPU
oracle's tests draw their inputs from.

Workloads (all coordinates in metres, z up, densities in kg/m^3):

* ``prism_model``  -- the synthetic model of Sec. 3: domain [0,600]^2 x
  [-450,150], a centred 100 m cube of density 2000, void elsewhere.
* ``fp64_prism_noise`` -- 16^3 voxels of 1 km, a +300 prism on voxels
  [4,12)x[4,12)x[6,10) plus N(0, 10^2) noise, 2x2x2 Gauss, 64x64 stations
  100 m above the top face.
* ``grf_volume``  -- 128^3 voxels of 250 m, exponential-covariance Gaussian
  random field (correlation length 2 km, sigma 150), midpoint rule, 512^2
  surface stations plus every voxel centre.
* ``layered_scale`` -- 464^3 voxels of 100 m, layered 2600/2700/2900
  background with three seeded +-400 ellipsoids, 1024^2 surface stations.
* ``serving_stream`` -- request sizes n^3 with n log-uniform in [32, 256],
  random-field densities, 256^2 surface stations, Poisson arrival times.
* ``adjoint_batch`` -- a hidden 128^3 random field, its 256^2 stations, and
  16 candidate models.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# Gravitational constant used by the paper: the Appendix A table of norms is
# reproduced exactly with the CODATA-2006 value.
G_PAPER = 6.67428e-11


@dataclass
class Grid:
    """Brick of nx*ny*nz voxels (Sec. 2.1); voxel (i,j,k) spans
    origin + [i, i+1) * h along each axis.  Arrays are [nz][ny][nx]."""
    n: tuple          # (nx, ny, nz)
    origin: tuple     # lower corner (m)
    h: tuple          # voxel size (m)

    @property
    def shape_zyx(self):
        return (self.n[2], self.n[1], self.n[0])

    @property
    def nvox(self) -> int:
        return int(self.n[0]) * int(self.n[1]) * int(self.n[2])

    @property
    def top(self) -> float:
        return float(self.origin[2] + self.n[2] * self.h[2])


@dataclass
class Workload:
    name: str
    grid: Grid
    rho: np.ndarray            # [B?][nz][ny][nx]
    xi: np.ndarray             # [nq][3] reference nodes in [-1,1]^3
    w: np.ndarray              # [nq] weights
    obs: np.ndarray            # [M][3]
    G: float = G_PAPER
    extra: dict = field(default_factory=dict)

    @property
    def n_sources(self) -> int:
        return self.grid.nvox * int(self.xi.shape[0])

    @property
    def n_obs(self) -> int:
        return int(self.obs.shape[0])


def gauss_rule(npts: int):
    """Tensor Gauss-Legendre rule with npts nodes per axis on [-1,1]^3
    (npts = 1: the cell centroid, SUM-G1; npts = 2: 2x2x2 Gauss, SUM-G2).
    Node order: x fastest.  Returns (xi [nq,3], w [nq])."""
    x, wt = np.polynomial.legendre.leggauss(int(npts))
    zz, yy, xx = np.meshgrid(x, x, x, indexing="ij")
    wz, wy, wx = np.meshgrid(wt, wt, wt, indexing="ij")
    xi = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1)
    return np.ascontiguousarray(xi), np.ascontiguousarray((wx * wy * wz).ravel())


def station_plane(x0, x1, y0, y1, nx, ny, z) -> np.ndarray:
    """nx*ny stations, cell-centred over [x0,x1]x[y0,y1] at height z
    (x fastest)."""
    xs = x0 + (np.arange(nx) + 0.5) * ((x1 - x0) / nx)
    ys = y0 + (np.arange(ny) + 0.5) * ((y1 - y0) / ny)
    yy, xx = np.meshgrid(ys, xs, indexing="ij")
    return np.ascontiguousarray(
        np.stack([xx.ravel(), yy.ravel(), np.full(xx.size, float(z))], axis=1))


def voxel_centres(grid: Grid) -> np.ndarray:
    """Centres of all voxels in grid order (x fastest):
    origin + (i + 0.5) * h."""
    nx, ny, nz = grid.n
    cx = (np.arange(nx) + 0.5) * grid.h[0] + grid.origin[0]
    cy = (np.arange(ny) + 0.5) * grid.h[1] + grid.origin[1]
    cz = (np.arange(nz) + 0.5) * grid.h[2] + grid.origin[2]
    zz, yy, xx = np.meshgrid(cz, cy, cx, indexing="ij")
    return np.ascontiguousarray(np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1))


def exp_cov_grf(n: int, h: float, corr_len: float, sigma: float, seed: int,
                dtype=np.float64) -> np.ndarray:
    """Stationary Gaussian random field with covariance
    sigma^2 exp(-r / corr_len) on an n^3 grid of spacing h, by circulant
    embedding on the (2n)^3 torus (negative eigenvalues clipped to 0).
    Returns [n][n][n] (z, y, x)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    m = 2 * n
    d = np.minimum(np.arange(m), m - np.arange(m)) * h
    r = np.sqrt(d[:, None, None] ** 2 + d[None, :, None] ** 2 + d[None, None, :] ** 2)
    c = sigma * sigma * np.exp(-r / corr_len)
    lam = np.fft.rfftn(c).real
    np.maximum(lam, 0.0, out=lam)
    white = rng.standard_normal((m, m, m))
    f = np.fft.irfftn(np.sqrt(lam) * np.fft.rfftn(white), s=(m, m, m), axes=(0, 1, 2))
    return np.ascontiguousarray(f[:n, :n, :n], dtype=dtype)


def periodic_grf(n: int, h: float, corr_len: float, sigma: float, seed: int,
                 dtype=np.float32) -> np.ndarray:
    """Cheaper random field for large request streams: the same exponential
    covariance wrapped on the n^3 torus (spectral synthesis without padding),
    rescaled to standard deviation sigma.  Returns [n][n][n]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    d = np.minimum(np.arange(n), n - np.arange(n)) * h
    r = np.sqrt(d[:, None, None] ** 2 + d[None, :, None] ** 2 + d[None, None, :] ** 2)
    lam = np.fft.rfftn(np.exp(-r / corr_len)).real
    np.maximum(lam, 0.0, out=lam)
    white = rng.standard_normal((n, n, n))
    f = np.fft.irfftn(np.sqrt(lam) * np.fft.rfftn(white), s=(n, n, n), axes=(0, 1, 2))
    f *= sigma / max(float(f.std()), 1e-30)
    return np.ascontiguousarray(f, dtype=dtype)


# ---------------------------------------------------------------- workloads
def prism_model(Mbar: int, npts: int = 1, rho: float = 2000.0) -> Workload:
    """Sec. 3 synthetic model discretised by Mbar^3 cells of h = 600/Mbar;
    only the anomaly cells carry density, so the grid returned covers just
    the 100 m cube [250,350]^2 x [-200,-100] and the observers are the
    centroids of all Mbar^3 cells of the domain (the error norms of
    Eqs. 11-13 are taken over the whole domain)."""
    h = 600.0 / Mbar
    nc = int(round(100.0 / h))
    grid = Grid((nc, nc, nc), (250.0, 250.0, -200.0), (h, h, h))
    dom = Grid((Mbar, Mbar, Mbar), (0.0, 0.0, -450.0), (h, h, h))
    xi, w = gauss_rule(npts)
    return Workload(f"prism_model_{Mbar}", grid, np.full(grid.shape_zyx, rho), xi, w,
                    voxel_centres(dom), extra={"domain": dom, "prism_lo": (250.0, 250.0, -200.0),
                                               "prism_hi": (350.0, 350.0, -100.0), "rho": rho})


def fp64_prism_noise(seed: int = 1) -> Workload:
    """16^3 x 1 km voxels, origin (0,0,-16 km) so the top face is z = 0;
    +300 kg/m^3 on voxels [4,12)x[4,12)x[6,10) (x, y, z indices, z counted
    from the bottom) plus N(0, 10^2) noise; 2x2x2 Gauss (32768 sources);
    64 x 64 stations 100 m above the top face."""
    n, h = 16, 1000.0
    grid = Grid((n, n, n), (0.0, 0.0, -n * h), (h, h, h))
    rng = np.random.Generator(np.random.PCG64(seed))
    rho = rng.normal(0.0, 10.0, size=grid.shape_zyx)
    rho[6:10, 4:12, 4:12] += 300.0
    xi, w = gauss_rule(2)
    obs = station_plane(0.0, n * h, 0.0, n * h, 64, 64, grid.top + 100.0)
    return Workload("fp64_prism_noise_16^3", grid, rho, xi, w, obs)


def grf_volume(n: int = 128, h: float = 250.0, seed: int = 2, stations: int = 512,
               volume_targets: bool = True) -> Workload:
    """n^3 voxels of h, exponential-covariance random field (2 km, sigma
    150), midpoint rule; stations^2 surface stations at the top face plus,
    when volume_targets, every voxel centre."""
    grid = Grid((n, n, n), (0.0, 0.0, -n * h), (h, h, h))
    rho = exp_cov_grf(n, h, 2000.0, 150.0, seed)
    xi, w = gauss_rule(1)
    obs = station_plane(0.0, n * h, 0.0, n * h, stations, stations, grid.top)
    if volume_targets:
        obs = np.concatenate([obs, voxel_centres(grid)], axis=0)
    return Workload(f"grf_volume_{n}^3", grid, rho, xi, w, obs)


def layered_scale(n: int = 464, h: float = 100.0, seed: int = 3, stations: int = 1024,
                  dtype=np.float32) -> Workload:
    """n^3 voxels of h: 2600/2700/2900 kg/m^3 in equal thirds (top to
    bottom) plus three axis-aligned ellipsoids (centres uniform in the inner
    80% of the box, semi-axes U[2,8] km, signs +,-,+ times 400)."""
    grid = Grid((n, n, n), (0.0, 0.0, -n * h), (h, h, h))
    rng = np.random.Generator(np.random.PCG64(seed))
    L = n * h
    rho = np.empty(grid.shape_zyx, dtype=dtype)
    t = n // 3
    rho[: n - 2 * t] = 2900.0          # bottom third (lowest z index)
    rho[n - 2 * t: n - t] = 2700.0
    rho[n - t:] = 2600.0               # top third
    cx = (np.arange(n) + 0.5) * h
    centres = rng.uniform(0.1 * L, 0.9 * L, size=(3, 3))
    axes = rng.uniform(2000.0, 8000.0, size=(3, 3))
    signs = (1.0, -1.0, 1.0)
    zc = cx - L  # voxel-centre z
    for e in range(3):
        c, a = centres[e], axes[e]
        qx = ((cx - c[0]) / a[0]) ** 2
        qy = ((cx - c[1]) / a[1]) ** 2
        qz = ((zc - (c[2] - L)) / a[2]) ** 2
        for k in np.nonzero(qz < 1.0)[0]:
            inside = (qx[None, :] + qy[:, None] + qz[k]) < 1.0
            rho[k][inside] += dtype(400.0 * signs[e])
    xi, w = gauss_rule(1)
    obs = station_plane(0.0, L, 0.0, L, stations, stations, grid.top)
    return Workload(f"layered_scale_{n}^3", grid, rho, xi, w, obs)


def serving_stream(n_requests: int = 512, seed: int = 4, nmin: int = 32, nmax: int = 256,
                   h: float = 250.0, stations: int = 256, rate_hz: float = 100.0):
    """Request descriptors for the serving workload: side n log-uniform in
    [nmin, nmax] (the voxel count is then log-uniform in [nmin^3, nmax^3]),
    Poisson arrival offsets at rate_hz, and a per-request density seed.
    Densities are generated lazily with :func:`serving_density`."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sides = np.rint(np.exp(rng.uniform(np.log(nmin), np.log(nmax), size=n_requests))).astype(int)
    gaps = rng.exponential(1.0 / rate_hz, size=n_requests)
    arrivals = np.cumsum(gaps) - gaps[0]
    reqs = []
    for i, n in enumerate(sides):
        grid = Grid((int(n), int(n), int(n)), (0.0, 0.0, -n * h), (h, h, h))
        obs = station_plane(0.0, n * h, 0.0, n * h, stations, stations, grid.top)
        reqs.append({"id": i, "grid": grid, "obs": obs, "arrival_s": float(arrivals[i]),
                     "seed": int(seed * 100003 + i)})
    return reqs


def serving_density(req, field=None, dtype=np.float32) -> np.ndarray:
    """Densities of one serving request: its own periodic random field
    (field None), or an n^3 window of a shared periodic field at an offset
    drawn from the request's seed (indices wrapped on the torus).  A window
    of a stationary field has the same covariance, so both are draws of the
    same distribution; the window is far cheaper for large streams."""
    n = req["grid"].n[0]
    if field is None:
        return periodic_grf(n, req["grid"].h[0], 2000.0, 150.0, req["seed"], dtype=dtype)
    m = field.shape[0]
    off = np.random.Generator(np.random.PCG64(req["seed"])).integers(0, m, size=3)
    idx = [(o + np.arange(n)) % m for o in off]
    return np.ascontiguousarray(field[np.ix_(idx[0], idx[1], idx[2])], dtype=dtype)


def adjoint_batch(n: int = 128, h: float = 250.0, stations: int = 256, batch: int = 16,
                  hidden_seed: int = 5, first_model_seed: int = 6):
    """Hidden density (seed 5) for synthesising data d, and `batch`
    candidate models (seeds 6, 7, ...), all exponential-covariance random
    fields on n^3 voxels of h; midpoint rule; stations^2 surface stations."""
    grid = Grid((n, n, n), (0.0, 0.0, -n * h), (h, h, h))
    hidden = exp_cov_grf(n, h, 2000.0, 150.0, hidden_seed)
    models = np.stack([exp_cov_grf(n, h, 2000.0, 150.0, first_model_seed + i)
                       for i in range(batch)])
    xi, w = gauss_rule(1)
    obs = station_plane(0.0, n * h, 0.0, n * h, stations, stations, grid.top)
    return Workload(f"adjoint_{n}^3_x{batch}", grid, models, xi, w, obs,
                    extra={"hidden": hidden})


def random_small(seed: int, n=(5, 4, 3), npts: int = 1, n_obs: int = 17, h=(1.0, 1.3, 0.9),
                 origin=(-2.0, 1.0, -3.5), obs_pad: float = 2.0, B: int = 1) -> Workload:
    """Small random problem for parity tests: random densities and random
    observers in a box padded around the grid."""
    rng = np.random.Generator(np.random.PCG64(seed))
    grid = Grid(tuple(int(v) for v in n), tuple(float(v) for v in origin),
                tuple(float(v) for v in h))
    shape = grid.shape_zyx if B == 1 else (B,) + grid.shape_zyx
    rho = rng.normal(0.0, 1.0, size=shape)
    lo = np.array(origin) - obs_pad
    hi = np.array(origin) + np.array(n) * np.array(h) + obs_pad
    obs = rng.uniform(lo, hi, size=(n_obs, 3))
    xi, w = gauss_rule(npts)
    return Workload(f"random_small_{seed}", grid, rho, xi, w, obs, G=1.0)


# ---------------------------------------------------------------- deformed cells and points
def hex_brick_mesh(n, lo, hi, warp: float = 0.0) -> np.ndarray:
    """Hexahedral mesh of the box [lo, hi] with n = (nx, ny, nz) cells.  Node
    (i, j, k) sits at the regular grid position moved, along every axis, by
    warp * extent * sin(pi u) sin(pi v) sin(pi w) with (u, v, w) its position
    in the box scaled to [0, 1]^3: boundary nodes stay put, so the deformed
    cells still tile the box.  Returns verts [ncell][8][3], cell
    c = (k ny + j) nx + i, corner a = i + 2 j + 4 k of the cell."""
    nx, ny, nz = (int(v) for v in n)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    u = [np.linspace(0.0, 1.0, m + 1) for m in (nx, ny, nz)]
    W, V, U = np.meshgrid(u[2], u[1], u[0], indexing="ij")         # [nz+1][ny+1][nx+1]
    bump = warp * np.sin(np.pi * U) * np.sin(np.pi * V) * np.sin(np.pi * W)
    ext = hi - lo
    nodes = np.stack([lo[0] + ext[0] * (U + bump), lo[1] + ext[1] * (V + bump),
                      lo[2] + ext[2] * (W + bump)], axis=-1)
    return _cells_of(nodes)


def _cells_of(nodes) -> np.ndarray:
    """Corners of the cells of a structured node array [nz+1][ny+1][nx+1][3]."""
    corners = [nodes[k:nodes.shape[0] - 1 + k, j:nodes.shape[1] - 1 + j, i:nodes.shape[2] - 1 + i]
               for k in (0, 1) for j in (0, 1) for i in (0, 1)]
    return np.ascontiguousarray(np.stack(corners, axis=3).reshape(-1, 8, 3))


def topo_surface(x, y, Lx, Ly, relief, seed):
    """Seeded topography: five Gaussian hills and valleys of widths
    U[0.08, 0.25] of the domain and heights U[-1, 1] * relief."""
    rng = np.random.Generator(np.random.PCG64(seed))
    z = np.zeros(np.broadcast(x, y).shape)
    for _ in range(5):
        cx, cy = rng.uniform(0.0, Lx), rng.uniform(0.0, Ly)
        wdt = rng.uniform(0.08, 0.25) * min(Lx, Ly)
        z += rng.uniform(-1.0, 1.0) * relief * np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / (2 * wdt * wdt))
    return z


def topo_mesh(nx: int = 64, ny: int = 64, nz: int = 32, Lx: float = 16000.0, Ly: float = 16000.0,
              depth: float = 8000.0, relief: float = 800.0, seed: int = 6):
    """Terrain-following hexahedral mesh (Sec. 4: topography): nodes on a
    regular horizontal grid over [0, Lx] x [0, Ly]; each node column runs from
    the flat bottom z = -depth to the topographic surface z_t(x, y)
    (:func:`topo_surface`) in nz equal steps.  Returns (verts
    [nx ny nz][8][3], surface node heights [ny+1][nx+1])."""
    xs = np.linspace(0.0, Lx, nx + 1)
    ys = np.linspace(0.0, Ly, ny + 1)
    Y, X = np.meshgrid(ys, xs, indexing="ij")
    zt = topo_surface(X, Y, Lx, Ly, relief, seed)
    t = np.linspace(0.0, 1.0, nz + 1)
    Z = -depth + (zt[None, :, :] + depth) * t[:, None, None]
    nodes = np.stack([np.broadcast_to(X, Z.shape), np.broadcast_to(Y, Z.shape), Z], axis=-1)
    return _cells_of(nodes), zt


def topo_workload(nx: int = 64, ny: int = 64, nz: int = 32, stations: int = 64, npts: int = 2,
                  seed: int = 6):
    """Deformed-cell workload: :func:`topo_mesh` (16 km x 16 km, 8 km deep,
    800 m relief), densities 2670 kg/m^3 plus a seeded anomaly field that
    follows depth below the surface (a +/-300 kg/m^3 band 1-3 km down), the
    npts^3 Gauss rule per cell, stations^2 stations draped 50 m above the
    surface.  Returns a dict with verts, rho [ncell], xi, w, obs."""
    Lx = Ly = 16000.0
    verts, _ = topo_mesh(nx, ny, nz, Lx, Ly, 8000.0, 800.0, seed)
    cen = verts.mean(axis=1)
    top = topo_surface(cen[:, 0], cen[:, 1], Lx, Ly, 800.0, seed)
    d = top - cen[:, 2]
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    phase = rng.uniform(0, 2 * np.pi, 2)
    band = np.exp(-((d - 2000.0) / 700.0) ** 2)
    rho = 2670.0 + 300.0 * band * np.sin(2 * np.pi * cen[:, 0] / Lx * 3 + phase[0]) * \
        np.cos(2 * np.pi * cen[:, 1] / Ly * 2 + phase[1])
    xi, w = gauss_rule(npts)
    sx = (np.arange(stations) + 0.5) * (Lx / stations)
    SY, SX = np.meshgrid(sx, sx, indexing="ij")
    obs = np.stack([SX.ravel(), SY.ravel(), topo_surface(SX, SY, Lx, Ly, 800.0, seed).ravel() + 50.0], axis=1)
    return {"name": "topo_hex_%dx%dx%d" % (nx, ny, nz), "verts": verts, "rho": rho, "xi": xi, "w": w,
            "obs": np.ascontiguousarray(obs), "G": G_PAPER}


def scattered_points(n: int, lo, hi, seed: int = 7) -> np.ndarray:
    """n density points uniform in the box [lo, hi] (seeded)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    return np.ascontiguousarray(lo + (hi - lo) * rng.random((int(n), 3)))


def voronoi_volumes(pts, lo, hi) -> np.ndarray:
    """Volume of each point's Voronoi cell clipped to the box [lo, hi] (the
    volume Sec. 4 associates with a scattered density point).  The points
    are mirrored across the six faces, which makes the faces bisectors, so
    every original cell is bounded by the box; each cell's volume is that of
    the convex hull of its vertices."""
    from scipy.spatial import ConvexHull, Voronoi
    pts = np.asarray(pts, dtype=np.float64)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    mirrored = [pts]
    for a in range(3):
        for face in (lo[a], hi[a]):
            m = pts.copy()
            m[:, a] = 2 * face - m[:, a]
            mirrored.append(m)
    vor = Voronoi(np.concatenate(mirrored))
    vol = np.empty(len(pts))
    for i in range(len(pts)):
        region = vor.regions[vor.point_region[i]]
        vol[i] = ConvexHull(vor.vertices[region]).volume
    return vol


def points_cloud(n: int = 1 << 24, stations: int = 512, seed: int = 8):
    """Scattered-density workload (Sec. 4: a random point distribution once
    each point carries a volume): n points uniform in a 16 km x 16 km x 4 km
    slab below the surface z = 0, densities 2670 kg/m^3 plus a seeded
    +/-250 kg/m^3 smooth field, stations^2 stations 50 m above the surface.
    Every point carries the slab volume / n, the mean volume of its Voronoi
    cell (the tests compute true Voronoi volumes on small clouds; at this
    size their construction would dominate).  Returns a dict with x, a, rho,
    per_cell = 1, obs."""
    Lx = Ly = 16000.0
    lo, hi = np.array([0.0, 0.0, -4000.0]), np.array([Lx, Ly, 0.0])
    x = scattered_points(n, lo, hi, seed)
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    ph = rng.uniform(0, 2 * np.pi, 3)
    rho = 2670.0 + 250.0 * np.sin(2 * np.pi * x[:, 0] / Lx * 2 + ph[0]) * \
        np.sin(2 * np.pi * x[:, 1] / Ly * 3 + ph[1]) * np.cos(np.pi * x[:, 2] / 4000.0 + ph[2])
    a = np.full(n, float(np.prod(hi - lo)) / n)
    sx = (np.arange(stations) + 0.5) * (Lx / stations)
    SY, SX = np.meshgrid(sx, sx, indexing="ij")
    obs = np.stack([SX.ravel(), SY.ravel(), np.full(SX.size, 50.0)], axis=1)
    return {"name": "points_cloud_%d" % n, "x": x, "a": a, "rho": rho, "per_cell": 1,
            "obs": np.ascontiguousarray(obs), "G": G_PAPER}
