"""Pins of the oracle's closed-form prism field (all three components) and of
its SUM-AN grid sum (Sec. 2.1: each constant-density voxel integrated in
closed form), against facts other than the formulas themselves: the vertical
component that Table 10 pins, the axis symmetry of Eq. 1, the point-mass
limit, Gauss's law (Eq. 2) outside and inside the body, fourth-order
convergence of the Gauss sums, additivity of the integral over voxels, and
the dot-product identity between the SUM-AN sum and its transpose.
"""
import numpy as np
import pytest

from oracle import direct
from paper_1107_5951_gb300 import workloads as wl

RNG = np.random.default_rng(20110728)


def _random_prisms(n):
    lo = RNG.uniform(-3.0, 3.0, size=(n, 3))
    return lo, lo + RNG.uniform(0.3, 2.5, size=(n, 3))


def test_vertical_component_is_the_table10_formula():
    """g_z of the vector routine is the same arithmetic as the g_z routine
    whose every Table 10 digit is pinned."""
    lo, hi = _random_prisms(8)
    for a, b in zip(lo, hi):
        pts = RNG.uniform(-6.0, 6.0, size=(40, 3))
        assert np.array_equal(direct.prism_g(a, b, 2.5, 0.7, pts)[:, 2], direct.prism_gz(a, b, 2.5, 0.7, pts))


def test_horizontal_components_by_axis_rotation():
    """Eq. 1 treats the axes alike: relabelling (x, y, z) -> (y, z, x) turns
    g_x into the vertical field of the relabelled prism, and (x, y, z) ->
    (z, x, y) turns g_y into it.  Observers outside, inside and on faces."""
    lo, hi = _random_prisms(6)
    for a, b in zip(lo, hi):
        pts = np.concatenate([RNG.uniform(-6.0, 6.0, size=(30, 3)),
                              RNG.uniform(a, b, size=(10, 3))])
        pts[-1] = [a[0], 0.5 * (a[1] + b[1]), b[2]]       # on an edge of the top face
        pts[-2] = [0.3 * a[0] + 0.7 * b[0], a[1], 0.5 * (a[2] + b[2])]   # on a side face
        g = direct.prism_g(a, b, 1.0, 1.0, pts)
        for comp, perm in ((0, [1, 2, 0]), (1, [2, 0, 1])):
            gz_rot = direct.prism_gz(a[perm], b[perm], 1.0, 1.0, pts[:, perm])
            scale = np.abs(g).max()
            assert np.max(np.abs(g[:, comp] - gz_rot)) <= 1e-13 * scale, comp


def test_point_mass_limit_of_a_cube():
    """Far from a cube the field is that of its mass at the centre; a cube
    has no quadrupole moment, so the relative residual falls like d^-4."""
    a = 1.0
    lo, hi = np.full(3, -a / 2), np.full(3, a / 2)
    dirs = np.array([[1.0, 0.3, 0.7], [-0.2, 1.0, 0.4], [0.5, -0.6, -1.0]])
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    errs = []
    for d in (5.0, 10.0, 20.0):
        pts = d * dirs
        g = direct.prism_g(lo, hi, 1.0, 1.0, pts)
        mono = a ** 3 * pts / d ** 3
        errs.append(np.max(np.linalg.norm(g - mono, axis=1)) / (a ** 3 / d ** 2))
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all((ratios > 14.0) & (ratios < 18.0)), ratios
    assert errs[0] < 2e-3


def _flux(fun, centre, radius, n_mu=48, n_phi=96):
    mu, wmu = np.polynomial.legendre.leggauss(n_mu)
    phi = (np.arange(n_phi) + 0.5) * (2 * np.pi / n_phi)
    MU, PHI = np.meshgrid(mu, phi, indexing="ij")
    s = np.sqrt(1 - MU ** 2)
    nrm = np.stack([s * np.cos(PHI), s * np.sin(PHI), MU], -1).reshape(-1, 3)
    wts = (wmu[:, None] * np.full(n_phi, 2 * np.pi / n_phi)[None, :]).ravel() * radius ** 2
    g = fun(np.asarray(centre) + radius * nrm)
    return float(np.sum(wts * np.sum(g * nrm, axis=1)))


def test_gauss_law_outside_and_inside_the_prism():
    """Flux of g through a sphere = +4 pi G times the enclosed mass (Eq. 2
    with g = -grad phi): the whole prism from outside, nothing from a sphere
    beside it, and a small ball of the uniform density from a sphere that
    lies inside the prism."""
    lo, hi = np.array([-1.0, -0.5, -0.75]), np.array([1.5, 0.5, 0.25])
    rho, G = 3.0, 0.5
    fun = lambda p: direct.prism_g(lo, hi, rho, G, p)   # noqa: E731
    mass = rho * np.prod(hi - lo)
    assert _flux(fun, (0.2, 0.1, -0.2), 4.0) == pytest.approx(4 * np.pi * G * mass, rel=1e-10)
    assert abs(_flux(fun, (9.0, 0.0, 0.0), 3.0)) < 1e-10 * 4 * np.pi * G * mass
    r = 0.3
    ball = rho * 4.0 / 3.0 * np.pi * r ** 3
    assert _flux(fun, (0.1, 0.05, -0.3), r) == pytest.approx(4 * np.pi * G * ball, rel=1e-10)


def test_gauss_sums_converge_to_the_closed_form_at_fourth_order():
    """The 2x2x2 Gauss sum over s^3 cells of a uniform prism approaches the
    closed-form vector field at order h^4 for an observer one side away
    (all three components nonzero)."""
    lo, hi = np.array([0.0, 0.0, -1.0]), np.array([1.0, 1.0, 0.0])
    obs = np.array([[1.7, 1.3, 0.8], [-0.6, 0.4, 0.9]])
    exact = direct.prism_g(lo, hi, 1.0, 1.0, obs)
    assert np.all(np.abs(exact) > 1e-3)
    xi, w = wl.gauss_rule(2)
    errs = []
    for s in (2, 4, 8):
        g = direct.forward((s, s, s), lo, (1.0 / s,) * 3, xi, w, np.ones((s, s, s)), obs, 1.0)
        errs.append(np.max(np.abs(g - exact)) / np.max(np.abs(exact)))
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all((ratios > 13.0) & (ratios < 19.0)), ratios


def test_sum_an_of_a_uniform_grid_is_one_prism():
    """The integral is additive over voxels: SUM-AN over a constant-density
    grid equals the closed form of the whole brick, for observers outside,
    inside, on voxel faces and at a voxel corner."""
    n, origin, h = (3, 4, 2), np.array([-1.0, 0.5, -2.0]), np.array([0.5, 0.25, 0.75])
    lo, hi = origin, origin + np.array(n) * h
    obs = np.concatenate([RNG.uniform(lo - 2.0, hi + 2.0, size=(40, 3)), RNG.uniform(lo, hi, size=(10, 3))])
    obs[-1] = origin + np.array([1, 2, 1]) * h                 # a corner shared by eight voxels
    obs[-2] = origin + np.array([1.5, 1, 0.5]) * h             # on a face between two voxels
    rho = np.full((n[2], n[1], n[0]), 2.0)
    g = direct.forward_analytic(n, origin, h, rho, obs, 0.3)
    ref = direct.prism_g(lo, hi, 2.0, 0.3, obs)
    assert np.max(np.abs(g - ref)) <= 1e-12 * np.abs(ref).max()


def test_sum_an_at_the_centre_of_a_symmetric_grid_is_zero():
    """An observer at the shared corner at the centre of a 2x2x2 grid whose
    densities are mirror-symmetric about it feels no field."""
    rho = np.full((2, 2, 2), 5.0)
    g = direct.forward_analytic((2, 2, 2), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), rho, np.array([[1.0, 1.0, 1.0]]), 1.0)
    assert np.all(np.abs(g) < 1e-14)


def test_sum_an_is_linear_and_tends_to_the_midpoint_sum():
    """SUM-AN is linear in rho, and far from a grid of cubic voxels it
    agrees with the one-point (SUM-G1) sum up to a relative O((h/d)^4):
    a cube's field is its point mass plus an l >= 4 correction."""
    n, origin, h = (3, 2, 2), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)
    rho = RNG.uniform(1.0, 3.0, size=(2, 2, 2, 3))
    dirs = np.array([[0.3, 1.0, 0.6], [-1.0, 0.2, 0.5]])
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    c = np.array([1.5, 1.0, 1.0])
    xi, w = wl.gauss_rule(1)
    ga = direct.forward_analytic(n, origin, h, rho, c + 5.0 * dirs, 1.0)
    gl = direct.forward_analytic(n, origin, h, 0.5 * rho[0] - 2.0 * rho[1], c + 5.0 * dirs, 1.0)
    assert np.allclose(gl, 0.5 * ga[0] - 2.0 * ga[1], rtol=0, atol=1e-14 * np.abs(ga).max())
    errs = []
    for d in (12.0, 24.0, 48.0):
        obs = c + d * dirs
        an = direct.forward_analytic(n, origin, h, rho[0], obs, 1.0)
        mid = direct.forward(n, origin, h, xi, w, rho[0], obs, 1.0)
        errs.append(np.max(np.abs(an - mid)) / np.max(np.abs(an)))
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all((ratios > 13.0) & (ratios < 19.0)), ratios


@pytest.mark.parametrize("ncomp", [1, 3])
def test_sum_an_adjoint_dot_product(ncomp):
    """<A x, y> = <x, A^T y> for the SUM-AN sum and its transpose (the sum is
    linear in rho), observers inside and outside the grid."""
    n, origin, h = (4, 3, 2), (-1.0, 0.5, -2.0), (0.5, 0.75, 1.0)
    rho = RNG.normal(size=(2, 2, 3, 4))
    obs = np.concatenate([RNG.uniform(-3.0, 3.0, size=(9, 3)), RNG.uniform((-1.0, 0.5, -2.0), (1.0, 2.75, 0.0),
                                                                            size=(4, 3))])
    g = direct.forward_analytic(n, origin, h, rho, obs, 0.3)
    y = RNG.normal(size=(2, len(obs)) if ncomp == 1 else (2, len(obs), 3))
    at = direct.adjoint_analytic(n, origin, h, obs, y, 0.3, ncomp=ncomp)
    for b in range(2):
        lhs = np.sum((g[b, :, 2] if ncomp == 1 else g[b]) * y[b])
        rhs = np.sum(rho[b] * at[b])
        assert lhs == pytest.approx(rhs, rel=1e-12)
