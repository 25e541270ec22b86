"""Pins of the FP64 CPU oracle to facts fixed by the paper and by mathematics.

None of these compares the oracle with itself: each checks it against a value
the paper prints, a closed form, an exact-arithmetic brute force, a physical
law, or a convergence rate the paper reports.
"""
import math
from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np
import pytest

from conftest import golden
from oracle import direct
from paper_1107_5951_gb300 import workloads as wl

G = wl.G_PAPER
PRISM_LO = (250.0, 250.0, -200.0)
PRISM_HI = (350.0, 350.0, -100.0)
DOM_LO = (0.0, 0.0, -450.0)
DOM_HI = (600.0, 600.0, 150.0)


# ---------------------------------------------------------------- Table 10
@pytest.mark.parametrize("row", golden("table10_prism_norms.txt"),
                         ids=lambda r: f"M{r[0]}_m{r[1]}")
def test_table10_prism_norms(row):
    """Appendix A, Table 10: the analytic prism field integrated by a
    4-point Gauss rule on m^3 sub-cells reproduces every printed digit with
    G = 6.67428e-11.  Pins the closed-form prism field (SUM-AN) used by the
    other pins; the L1 column is linear in G and fixes G, the L2 and max
    columns then check the field's shape."""
    Mbar, m = int(row[0]), int(row[1])
    l1, l2, linf = (float(v) for v in row[2:5])
    out = direct.prism_norms(PRISM_LO, PRISM_HI, 2000.0, G, DOM_LO, DOM_HI, Mbar, m, 4)
    # the paper's L1 column itself scatters by +-5 units in the 13th digit
    assert out[0] == pytest.approx(l1, rel=2.5e-12)
    assert out[1] == pytest.approx(l2, rel=1.5e-12)
    assert out[2] == pytest.approx(linf, rel=1.5e-12)


def test_prism_point_mass_limit():
    """Far from a small prism its field tends to Newton's point-mass field
    with the sign of Eq. 1 (g points from the mass to the observer), with a
    relative correction O((a/d)^2)."""
    lo, hi = np.array([-1.0, -1.0, -1.0]), np.array([1.0, 1.0, 1.0])
    mass = 8.0
    pts = np.array([[0.0, 0.0, 200.0], [0.0, 0.0, -200.0], [120.0, 50.0, 90.0],
                    [-80.0, 130.0, -40.0]])
    gz = direct.prism_gz(lo, hi, 1.0, 1.0, pts)
    r = np.linalg.norm(pts, axis=1)
    newton = mass * pts[:, 2] / r ** 3
    assert np.all(np.abs(gz - newton) <= 1e-4 * mass / r ** 2)
    assert gz[0] > 0 and gz[1] < 0


def test_prism_inside_symmetry():
    """At the centre of the prism the field vanishes; at mirror points
    above and below the centre g_z is equal and opposite."""
    lo, hi = np.array(PRISM_LO), np.array(PRISM_HI)
    c = 0.5 * (lo + hi)
    pts = np.array([c, c + [0, 0, 30.0], c - [0, 0, 30.0], c + [10, -20, 70.0], c + [10, -20, -70.0]])
    gz = direct.prism_gz(lo, hi, 2000.0, G, pts)
    scale = abs(gz[1])
    assert abs(gz[0]) < 1e-14 * scale + 1e-25
    assert gz[1] == pytest.approx(-gz[2], rel=1e-13)
    assert gz[3] == pytest.approx(-gz[4], rel=1e-13)


# ---------------------------------------------------------------- Table 1
def _rates(npts, Mbars):
    errs = []
    for Mbar in Mbars:
        w = wl.prism_model(Mbar, npts)
        g = direct.forward(w.grid.n, w.grid.origin, w.grid.h, w.xi, w.w, w.rho, w.obs, G)
        exact = direct.prism_gz(PRISM_LO, PRISM_HI, 2000.0, G, w.obs)
        V = (600.0 / Mbar) ** 3
        e = np.abs(g[:, 2] - exact)
        errs.append((e.sum() * V, math.sqrt((e * e).sum() * V), e.max()))
    errs = np.log(np.array(errs))
    logh = np.log(600.0 / np.array(Mbars, dtype=float))
    return [np.polyfit(logh, errs[:, k], 1)[0] for k in range(3)]


def test_table1_summation_rates():
    """Sec. 3.1.1, Table 1: SUM-G1 and SUM-G2 error norms of g_z against the
    analytic field, measured by a 1-point rule at the cell centroids of the
    whole domain, converge at the printed rates.  Pins the oracle's
    quadrature (node placement, weights, masses) and the rule that an
    observer coinciding with a source point gets nothing from it (the E_inf
    rate of 1 comes from the cells next to the prism's edges)."""
    paper = {r[0]: (float(r[1]), float(r[2])) for r in golden("table1_sum_rates.txt")}
    g1 = _rates(1, [12, 24, 48, 96])
    g2 = _rates(2, [12, 24, 48])
    for k, name in enumerate(["E1", "E2", "Einf"]):
        assert g1[k] == pytest.approx(paper[name][0], abs=0.02), (name, g1[k])
        assert g2[k] == pytest.approx(paper[name][1], abs=0.02), (name, g2[k])


# ---------------------------------------------------------------- quadrature
def test_gauss_sum_converges_to_prism():
    """The 2x2x2 Gauss sum over a prism split into s^3 voxels converges to
    the closed form at fourth order (the rule integrates cubics exactly).
    So does the midpoint sum for an exterior observer: its h^2 error term is
    proportional to the volume integral of the Laplacian of the kernel,
    which vanishes because the kernel is harmonic away from the observer."""
    lo = np.array([0.0, 0.0, -100.0])
    obs = wl.station_plane(-50.0, 150.0, -50.0, 150.0, 5, 4, 60.0)
    exact = direct.prism_gz(lo, lo + 100.0, 2500.0, G, obs)
    for npts, order, s_list in ((2, 4.0, (2, 4, 8, 16)), (1, 4.0, (4, 8, 16, 32))):
        xi, w = wl.gauss_rule(npts)
        errs = []
        for s in s_list:
            h = 100.0 / s
            g = direct.forward((s, s, s), lo, (h, h, h), xi, w, np.full((s, s, s), 2500.0), obs, G)
            errs.append(np.max(np.abs(g[:, 2] - exact)) / np.max(np.abs(exact)))
        rates = -np.diff(np.log(errs)) / math.log(2.0)
        assert rates[-1] == pytest.approx(order, abs=0.15), (npts, rates)
        if npts == 2:
            assert errs[-1] < 5e-7


# ---------------------------------------------------------------- brute force
def _exact_sum(grid_n, origin, h, xi, w, rho, obs):
    """Eq. 1 discretised, in exact rational arithmetic for the differences
    and squares and 60-digit decimals for the square roots."""
    getcontext().prec = 60
    nx, ny, nz = grid_n
    wsum = sum(float(v) for v in w)
    vol = h[0] * h[1] * h[2]
    out = []
    mag = []
    for r in obs:
        acc = [Decimal(0)] * 3
        tot = [Decimal(0)] * 3
        for k in range(nz):
            for j in range(ny):
                for i in range(nx):
                    for q in range(len(w)):
                        c = [origin[0] + (i + 0.5) * h[0], origin[1] + (j + 0.5) * h[1],
                             origin[2] + (k + 0.5) * h[2]]
                        x = [c[a] + 0.5 * h[a] * xi[q][a] for a in range(3)]
                        d = [Fraction(float(r[a])) - Fraction(x[a]) for a in range(3)]
                        rr = d[0] * d[0] + d[1] * d[1] + d[2] * d[2]
                        if rr == 0:
                            continue
                        m = Fraction(float(rho[k, j, i]) * vol * (float(w[q]) / wsum))
                        rrd = Decimal(rr.numerator) / Decimal(rr.denominator)
                        inv3 = Decimal(1) / (rrd * rrd.sqrt())
                        for a in range(3):
                            t = (Decimal((m * d[a]).numerator) / Decimal((m * d[a]).denominator)) * inv3
                            acc[a] += t
                            tot[a] += abs(t)
        out.append([float(v) for v in acc])
        mag.append([float(v) for v in tot])
    return np.array(out), np.array(mag)


@pytest.mark.parametrize("npts,seed", [(1, 3), (2, 4)])
def test_bruteforce_exact_arithmetic(npts, seed):
    """<= 64 sources: the oracle's compensated FP64 sum agrees with the
    exact sum to the rounding of the individual terms (a few ulp of the sum
    of magnitudes), including an observer placed exactly on a source."""
    n = (4, 4, 4) if npts == 1 else (2, 2, 2)
    wk = wl.random_small(seed, n=n, npts=npts, n_obs=6, h=(0.75, 1.25, 1.0), origin=(-1.0, 0.5, -2.0))
    obs = wk.obs.copy()
    obs[0] = [-1.0 + 1.5 * 0.75, 0.5 + 0.5 * 1.25, -2.0 + 2.5 * 1.0] if npts == 1 else obs[0]
    g = direct.forward(wk.grid.n, wk.grid.origin, wk.grid.h, wk.xi, wk.w, wk.rho, obs, 1.0)
    exact, mag = _exact_sum(wk.grid.n, wk.grid.origin, wk.grid.h, wk.xi, wk.w, wk.rho, obs)
    assert np.all(np.abs(g - exact) <= 4e-16 * mag + 1e-300)


def test_single_voxel_centroid_is_zero():
    """An observer at the centroid of a lone voxel: the midpoint rule skips
    the coincident pair, the 2x2x2 rule cancels by symmetry."""
    for npts in (1, 2):
        xi, w = wl.gauss_rule(npts)
        g = direct.forward((1, 1, 1), (0.0, 0.0, 0.0), (2.0, 2.0, 2.0), xi, w,
                           np.full((1, 1, 1), 7.0), np.array([[1.0, 1.0, 1.0]]), 1.0)
        assert np.all(np.abs(g) < 1e-15)


# ---------------------------------------------------------------- sphere
def test_uniform_sphere_monopole():
    """A voxelised sphere with cubic symmetry: outside it, the field is the
    point-mass field of the total mass plus an l = 4 correction, so the
    relative error falls like d^-4."""
    R = 6
    c = np.arange(-R, R) + 0.5
    zz, yy, xx = np.meshgrid(c, c, c, indexing="ij")
    inside = (xx ** 2 + yy ** 2 + zz ** 2) <= R * R
    rho = inside.astype(float)
    mass = rho.sum()
    xi, w = wl.gauss_rule(1)
    dirs = np.array([[1.0, 0.3, 0.7], [-0.2, 1.0, 0.4], [0.5, -0.6, -1.0]])
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    errs = []
    for d in (30.0, 60.0, 120.0):
        pts = d * dirs
        g = direct.forward((2 * R,) * 3, (-R,) * 3, (1.0, 1.0, 1.0), xi, w, rho, pts, 1.0)
        mono = mass * pts / d ** 3
        errs.append(np.max(np.linalg.norm(g - mono, axis=1)) / (mass / d ** 2))
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all((ratios > 13.0) & (ratios < 19.0)), ratios
    assert errs[0] < 1e-4


# ---------------------------------------------------------------- Gauss's law
def _sphere_flux(centre, radius, wk, n_mu=40, n_phi=80):
    mu, wmu = np.polynomial.legendre.leggauss(n_mu)
    phi = (np.arange(n_phi) + 0.5) * (2 * np.pi / n_phi)
    MU, PHI = np.meshgrid(mu, phi, indexing="ij")
    s = np.sqrt(1 - MU ** 2)
    nrm = np.stack([s * np.cos(PHI), s * np.sin(PHI), MU], -1).reshape(-1, 3)
    wts = (wmu[:, None] * np.full(n_phi, 2 * np.pi / n_phi)[None, :]).ravel() * radius ** 2
    pts = np.asarray(centre) + radius * nrm
    g = direct.forward(wk.grid.n, wk.grid.origin, wk.grid.h, wk.xi, wk.w, wk.rho, pts, wk.G)
    return float(np.sum(wts * np.sum(g * nrm, axis=1)))


def test_gauss_law_flux():
    """The flux of g through a closed surface is +4 pi G times the enclosed
    mass (Eq. 2 with g = -grad phi), and zero through a surface that
    encloses no mass."""
    wk = wl.random_small(11, n=(4, 3, 3), npts=2, n_obs=1, h=(1.0, 1.0, 1.0), origin=(0.0, 0.0, 0.0))
    wk.rho = np.abs(wk.rho) + 0.5
    wk.G = G
    mass = wk.rho.sum() * 1.0
    centre = (2.0, 1.5, 1.5)
    flux = _sphere_flux(centre, 8.0, wk)
    assert flux == pytest.approx(4 * np.pi * G * mass, rel=1e-10)
    flux0 = _sphere_flux((30.0, 1.5, 1.5), 8.0, wk)
    assert abs(flux0) < 1e-10 * 4 * np.pi * G * mass


# ---------------------------------------------------------------- adjoint
@pytest.mark.parametrize("ncomp", [1, 3])
def test_adjoint_dot_product(ncomp):
    """<A x, y> = <x, A^T y>: the transpose sum is the exact adjoint of the
    forward sum (Eq. 1 is linear in rho)."""
    wk = wl.random_small(21, n=(5, 4, 3), npts=2, n_obs=23, B=2)
    g = direct.forward(wk.grid.n, wk.grid.origin, wk.grid.h, wk.xi, wk.w, wk.rho, wk.obs, 1.0)
    rng = np.random.default_rng(5)
    y = rng.normal(size=(2, wk.n_obs) if ncomp == 1 else (2, wk.n_obs, 3))
    at = direct.adjoint(wk.grid.n, wk.grid.origin, wk.grid.h, wk.xi, wk.w, wk.obs, y, 1.0, ncomp=ncomp)
    for b in range(2):
        lhs = np.sum((g[b, :, 2] if ncomp == 1 else g[b]) * y[b])
        rhs = np.sum(wk.rho[b] * at[b])
        assert lhs == pytest.approx(rhs, rel=1e-12)


def test_linearity_and_mirror_symmetry():
    """g is linear in rho; for a density symmetric under x -> -x about the
    grid's mid-plane, g_x is odd and g_y, g_z even under the mirror."""
    wk = wl.random_small(31, n=(4, 3, 3), npts=2, n_obs=5, h=(1.0, 1.0, 1.0), origin=(-2.0, 0.0, 0.0), B=2)
    a, b = 0.75, -1.5
    gb = direct.forward(wk.grid.n, wk.grid.origin, wk.grid.h, wk.xi, wk.w, wk.rho, wk.obs, 1.0)
    gc = direct.forward(wk.grid.n, wk.grid.origin, wk.grid.h, wk.xi, wk.w,
                        a * wk.rho[0] + b * wk.rho[1], wk.obs, 1.0)
    assert np.allclose(gc, a * gb[0] + b * gb[1], rtol=1e-13, atol=1e-13 * np.abs(gb).max())
    rho = wk.rho[0] + wk.rho[0][:, :, ::-1]
    obs = wk.obs
    mir = obs * np.array([-1.0, 1.0, 1.0])
    g1 = direct.forward(wk.grid.n, wk.grid.origin, wk.grid.h, wk.xi, wk.w, rho, obs, 1.0)
    g2 = direct.forward(wk.grid.n, wk.grid.origin, wk.grid.h, wk.xi, wk.w, rho, mir, 1.0)
    sc = np.abs(g1).max()
    assert np.allclose(g2[:, 0], -g1[:, 0], atol=1e-13 * sc)
    assert np.allclose(g2[:, 1:], g1[:, 1:], atol=1e-13 * sc)


def test_translation_invariance():
    """Moving the grid and the observers by the same vector leaves g
    unchanged: Eq. 1 depends on r - x only.  The shift is a multiple of
    the voxel size, so only the rounding of the coordinates differs."""
    wk = wl.random_small(51, n=(5, 4, 3), npts=2, n_obs=29, h=(0.5, 0.5, 0.5), origin=(0.0, 0.0, 0.0))
    t = np.array([64.0, -32.0, 128.0])
    g0 = direct.forward(wk.grid.n, wk.grid.origin, wk.grid.h, wk.xi, wk.w, wk.rho, wk.obs, 1.0)
    g1 = direct.forward(wk.grid.n, tuple(np.array(wk.grid.origin) + t), wk.grid.h, wk.xi, wk.w, wk.rho,
                        wk.obs + t, 1.0)
    assert np.max(np.abs(g1 - g0)) <= 1e-11 * np.max(np.abs(g0))
    g2 = direct.forward(wk.grid.n, tuple(np.array(wk.grid.origin) + t), wk.grid.h, wk.xi, wk.w, wk.rho,
                        wk.obs, 1.0)
    assert np.max(np.abs(g2 - g0)) > 1e-3 * np.max(np.abs(g0))


def test_adjoint_subset_matches_full_transpose():
    """The sampled transpose sum returns exactly the full transpose sum's
    values at the sampled voxels (same arithmetic, same order)."""
    wk = wl.random_small(41, n=(5, 4, 3), npts=2, n_obs=19, B=1)
    rng = np.random.default_rng(8)
    y = rng.normal(size=(2, wk.n_obs, 3))
    full = direct.adjoint(wk.grid.n, wk.grid.origin, wk.grid.h, wk.xi, wk.w, wk.obs, y, 1.0, ncomp=3)
    vox = np.array([0, 7, 33, 59])
    sub = direct.adjoint_subset(wk.grid.n, wk.grid.origin, wk.grid.h, wk.xi, wk.w, wk.obs, y, 1.0, vox, ncomp=3)
    assert np.array_equal(sub, full.reshape(2, -1)[:, vox])
