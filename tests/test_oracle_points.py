"""Oracle pins for weighted point sources: the quadrature points of deformed
hexahedral cells (the general SUM-G1 of Sec. 2.1, integration in reference
coordinates with the Jacobian of the cell's map) and scattered density
points with their volumes (Sec. 4).  Pinned by what the mathematics fixes:
undeformed cells reproduce the voxel sum, the 2x2x2 rule integrates the
trilinear cells' volumes exactly, a deformed tiling of a prism converges to
the prism's closed form at fourth order, Gauss's law, mirror symmetry, points
on a voxel lattice reproduce the midpoint sum, and 60-digit brute force."""
import math
from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np
import pytest

from oracle import direct
from paper_1107_5951_gb300 import workloads as wl

G = 6.67428e-11


def test_undeformed_cells_are_the_voxel_sum():
    """A regular brick mesh read as hexahedra gives the voxel quadrature
    points and weights, so the sums agree to rounding."""
    rng = np.random.default_rng(1)
    n, lo, h = (5, 4, 3), np.array([-2.0, 1.0, -3.0]), np.array([1.5, 1.0, 2.0])
    verts = wl.hex_brick_mesh(n, lo, lo + np.array(n) * h)
    rho = rng.normal(size=(n[2], n[1], n[0]))
    obs = rng.uniform(lo - 3, lo + np.array(n) * h + 3, size=(40, 3))
    for npts in (1, 2):
        xi, w = wl.gauss_rule(npts)
        want = direct.forward(n, lo, h, xi, w, rho, obs, G)
        got = direct.forward_hex(verts, xi, w, rho.ravel(), obs, G)
        assert np.linalg.norm(got - want) <= 1e-13 * np.linalg.norm(want)


def test_gauss_rule_integrates_trilinear_volumes_exactly():
    """|det J| of a trilinear cell is a polynomial of degree <= 2 per
    reference axis, so the 2x2x2 rule gives the exact volume: a terrain mesh
    holds the volume between its bilinear top surface and the flat bottom,
    sum over columns of the area times the mean of the four corner heights."""
    verts, zt = wl.topo_mesh(12, 10, 6, 6000.0, 5000.0, 3000.0, 600.0, seed=3)
    xi, w = wl.gauss_rule(2)
    _, a = direct.hex_sources(verts, xi, w)
    area = (6000.0 / 12) * (5000.0 / 10)
    h = zt + 3000.0
    exact = area * 0.25 * (h[:-1, :-1] + h[:-1, 1:] + h[1:, :-1] + h[1:, 1:]).sum()
    assert a.sum() == pytest.approx(exact, rel=1e-13)
    # the cells of a warped brick tile the brick
    vb = wl.hex_brick_mesh((6, 5, 4), (0.0, 0.0, 0.0), (3.0, 2.0, 1.0), warp=0.08)
    _, ab = direct.hex_sources(vb, xi, w)
    assert ab.sum() == pytest.approx(6.0, rel=1e-13)


def test_deformed_tiling_converges_to_the_prism_formula():
    """A prism tiled by warped hexahedra (interior nodes displaced, faces
    fixed) is still the prism: the 2x2x2 Gauss sum converges to the closed
    form at fourth order as the tiling is refined."""
    lo, hi = np.array([0.0, 0.0, -100.0]), np.array([100.0, 80.0, 0.0])
    obs = wl.station_plane(-40.0, 140.0, -40.0, 120.0, 4, 4, 40.0)
    exact = direct.prism_gz(lo, hi, 2500.0, G, obs)
    xi, w = wl.gauss_rule(2)
    errs = []
    for s in (4, 8, 16):
        verts = wl.hex_brick_mesh((s, s, s), lo, hi, warp=0.06)
        g = direct.forward_hex(verts, xi, w, np.full(s ** 3, 2500.0), obs, G)
        errs.append(np.max(np.abs(g[:, 2] - exact)) / np.max(np.abs(exact)))
    rates = -np.diff(np.log(errs)) / math.log(2.0)
    assert rates[-1] > 3.5, (errs, rates)
    assert errs[-1] < 1e-6


def _sphere_flux(centre, radius, x, a, per_cell, rho, n_mu=40, n_phi=80):
    mu, wmu = np.polynomial.legendre.leggauss(n_mu)
    phi = (np.arange(n_phi) + 0.5) * (2 * np.pi / n_phi)
    MU, PHI = np.meshgrid(mu, phi, indexing="ij")
    s = np.sqrt(1 - MU ** 2)
    nrm = np.stack([s * np.cos(PHI), s * np.sin(PHI), MU], -1).reshape(-1, 3)
    wts = (wmu[:, None] * np.full(n_phi, 2 * np.pi / n_phi)[None, :]).ravel() * radius ** 2
    g = direct.forward_points(x, a, per_cell, rho, np.asarray(centre) + radius * nrm, G)
    return float(np.sum(wts * np.sum(g * nrm, axis=1)))


def test_gauss_law_for_deformed_cells():
    """Flux through a sphere around the warped mesh = 4 pi G times the mass
    the sources carry; zero through a sphere that encloses none."""
    verts = wl.hex_brick_mesh((4, 3, 3), (0.0, 0.0, 0.0), (4.0, 3.0, 3.0), warp=0.1)
    xi, w = wl.gauss_rule(2)
    x, a = direct.hex_sources(verts, xi, w)
    rho = np.abs(np.random.default_rng(2).normal(size=36)) + 0.5
    mass = float(np.sum(np.repeat(rho, 8) * a))
    assert _sphere_flux((2.0, 1.5, 1.5), 8.0, x, a, 8, rho) == pytest.approx(4 * np.pi * G * mass, rel=1e-10)
    assert abs(_sphere_flux((30.0, 1.5, 1.5), 8.0, x, a, 8, rho)) < 1e-10 * 4 * np.pi * G * mass


def test_mirror_symmetry_of_deformed_cells():
    """Reflecting the mesh and the observers through x = 0 flips g_x and
    keeps g_y, g_z (|det J| is orientation-free)."""
    verts, _ = wl.topo_mesh(5, 4, 3, 2000.0, 1600.0, 900.0, 200.0, seed=9)
    xi, w = wl.gauss_rule(2)
    rho = np.random.default_rng(4).normal(size=60)
    obs = np.random.default_rng(5).uniform([-100, -100, 0], [2100, 1700, 400], size=(30, 3))
    g = direct.forward_hex(verts, xi, w, rho, obs, G)
    vm = verts.copy()
    vm[..., 0] *= -1
    om = obs.copy()
    om[:, 0] *= -1
    gm = direct.forward_hex(vm, xi, w, rho, om, G)
    scale = np.max(np.abs(g))
    assert np.max(np.abs(gm[:, 0] + g[:, 0])) <= 1e-13 * scale
    assert np.max(np.abs(gm[:, 1:] - g[:, 1:])) <= 1e-13 * scale


def test_points_on_a_voxel_lattice_are_the_midpoint_sum():
    rng = np.random.default_rng(6)
    n, lo, h = (4, 5, 3), np.array([0.5, -1.0, -2.0]), np.array([1.0, 1.0, 1.0])
    rho = rng.normal(size=(n[2], n[1], n[0]))
    pts = wl.voxel_centres(wl.Grid(n, tuple(lo), tuple(h)))
    obs = rng.uniform(lo - 2, lo + np.array(n) + 2, size=(30, 3))
    xi, w = wl.gauss_rule(1)
    want = direct.forward(n, lo, h, xi, w, rho, obs, G)
    got = direct.forward_points(pts, np.ones(len(pts)), 1, rho.ravel(), obs, G)
    assert np.linalg.norm(got - want) <= 1e-14 * np.linalg.norm(want)


def test_points_bruteforce_exact_arithmetic():
    """20 points with volumes and 5 observers (one on a point): the
    compensated FP64 sum equals the exact sum (rational differences and
    squares, 60-digit square roots) to the rounding of the terms (mass,
    reciprocal square root, cube and products: a few ulp of each)."""
    getcontext().prec = 60
    rng = np.random.default_rng(7)
    x = rng.uniform(-2, 2, size=(20, 3))
    a = rng.uniform(0.1, 1.0, size=20)
    rho = rng.normal(size=20)
    obs = rng.uniform(-3, 3, size=(5, 3))
    obs[0] = x[3]
    g = direct.forward_points(x, a, 1, rho, obs, 1.0)
    for j, r in enumerate(obs):
        acc = [Decimal(0)] * 3
        mag = [Decimal(0)] * 3
        for s in range(20):
            d = [Fraction(float(r[k])) - Fraction(float(x[s, k])) for k in range(3)]
            rr = d[0] * d[0] + d[1] * d[1] + d[2] * d[2]
            if rr == 0:
                continue
            m = Fraction(float(rho[s])) * Fraction(float(a[s]))
            rrd = Decimal(rr.numerator) / Decimal(rr.denominator)
            inv3 = Decimal(1) / (rrd * rrd.sqrt())
            for k in range(3):
                t = (Decimal((m * d[k]).numerator) / Decimal((m * d[k]).denominator)) * inv3
                acc[k] += t
                mag[k] += abs(t)
        for k in range(3):
            assert abs(g[j, k] - float(acc[k])) <= 1e-15 * float(mag[k]) + 1e-300
