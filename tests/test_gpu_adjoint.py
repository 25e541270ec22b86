"""The adjoint (gf_adjoint): the exact transpose of the forward model, in
direct and FMM mode, against the FP64 CPU transpose sum, the dot-product
identity, central finite differences, and the autograd wrapper."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1107_5951_gb300 as pkg  # noqa: E402
from oracle import direct  # noqa: E402
from paper_1107_5951_gb300 import workloads as wl  # noqa: E402
from paper_1107_5951_gb300.autograd import gravity  # noqa: E402

DEV = "cuda:0"


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def case(seed, n=20, npts=1, n_obs=500, B=2, vol=200):
    wk = wl.random_small(seed, n=(n, n - 2, n - 4), npts=npts, n_obs=n_obs, h=(1.0, 1.0, 1.0),
                         origin=(-3.0, 2.0, -16.0), obs_pad=3.0, B=B)
    if vol:
        vc = wl.voxel_centres(wk.grid)
        rng = np.random.default_rng(seed)
        wk.obs = np.concatenate([wk.obs, vc[rng.choice(len(vc), vol, replace=False)]])
    return wk


def plan(wk, mode, precision, p=14, B=2):
    obs = torch.tensor(wk.obs, dtype=torch.float64, device=DEV)
    return pkg.Plan(wk.grid.n, wk.grid.origin, wk.grid.h, wk.xi, wk.w, obs, mode=mode, precision=precision,
                    p=p, max_batch=B, G=wk.G)


@pytest.mark.parametrize("mode,precision,p,tol", [("fmm", "fp64", 14, 1e-6), ("fmm", "mixed", 12, 1e-5),
                                                  ("direct", "fp64", 0, 1e-12)])
@pytest.mark.parametrize("ncomp", [1, 3])
@pytest.mark.parametrize("npts", [1, 2])
def test_adjoint_matches_oracle_transpose(mode, precision, p, tol, ncomp, npts):
    wk = case(101 + npts, npts=npts)
    rng = np.random.default_rng(7)
    r = rng.normal(size=(2, wk.n_obs) if ncomp == 1 else (2, wk.n_obs, 3))
    ref = direct.adjoint(wk.grid.n, wk.grid.origin, wk.grid.h, wk.xi, wk.w, wk.obs, r, wk.G, ncomp=ncomp)
    with plan(wk, mode, precision, p=max(p, 1)) as pl:
        grad = pl.adjoint(torch.tensor(r, device=DEV), ncomp=ncomp).cpu().numpy()
        pl.check()
    assert rel_l2(grad, ref) <= tol


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("mixed", 1e-5)])
def test_fmm_adjoint_is_the_exact_transpose(precision, tol):
    """<A x, y> = <x, A^T y> for the FMM operator itself (not just to the
    FMM's truncation error): the adjoint applies the transposed operators."""
    wk = case(111, npts=2)
    rng = np.random.default_rng(3)
    x = torch.tensor(rng.normal(size=(2,) + wk.grid.shape_zyx), device=DEV)
    y = rng.normal(size=(2, wk.n_obs, 3))
    with plan(wk, "fmm", precision, p=8) as pl:
        g, _ = pl.forward(x)
        at = pl.adjoint(torch.tensor(y, device=DEV), ncomp=3)
        lhs = float(torch.sum(g.cpu() * torch.tensor(y)))
        rhs = float(torch.sum(x.cpu() * at.cpu()))
    assert abs(lhs - rhs) <= tol * abs(lhs)


def test_autograd_misfit_gradient_against_central_differences():
    """d/drho of 0.5 ||g_z(rho) - d||^2 through the autograd wrapper equals
    central differences (h = 1e-3 |rho_v|) on 32 voxels; the misfit is
    quadratic and the FMM linear, so the differences are exact up to
    rounding."""
    wk = case(121, n=16, B=1, vol=0)
    rng = np.random.default_rng(11)
    rho0 = torch.tensor(wk.rho + 2.0, device=DEV)
    d = torch.tensor(rng.normal(size=wk.n_obs) * 1e-3, device=DEV)
    with plan(wk, "fmm", "fp64", p=10, B=16) as pl:
        rho = rho0.clone().requires_grad_(True)
        gz = gravity(rho, pl, "gz")
        J = 0.5 * torch.sum((gz - d) ** 2)
        J.backward()
        grad = rho.grad.cpu().numpy().ravel()
        vox = rng.choice(rho0.numel(), 32, replace=False)
        fd = []
        for chunk in np.array_split(vox, 4):
            hs = 1e-3 * np.abs(rho0.cpu().numpy().ravel()[chunk])
            for sgn in (1.0, -1.0):
                batch = rho0.repeat(len(chunk), 1, 1, 1).reshape(len(chunk), -1)
                batch[torch.arange(len(chunk)), torch.tensor(chunk)] += sgn * torch.tensor(hs, device=DEV)
                _, gzb = pl.forward(batch.reshape((len(chunk),) + wk.grid.shape_zyx), want_g=False, want_gz=True)
                Jb = 0.5 * torch.sum((gzb - d[None]) ** 2, dim=1).cpu().numpy()
                if sgn > 0:
                    jp = Jb
                else:
                    fd.append((jp - Jb) / (2 * hs))
        fd = np.concatenate(fd)
    assert rel_l2(grad[np.concatenate(np.array_split(vox, 4))], fd) <= 1e-6


def test_adjoint_batch_of_16_models_full_size_sampled():
    """The 128^3 inversion workload: data from a hidden random-field density
    at 256^2 stations, 16 candidate models in one batch; the misfit gradient
    from the mixed-precision transposed FMM against the FP64 CPU transpose
    sum on 24 sampled voxels, with the same residuals."""
    wk = wl.adjoint_batch()
    with plan(wk, "fmm", "mixed", p=12, B=16) as pl:
        _, dz = pl.forward(torch.tensor(wk.extra["hidden"], device=DEV), want_g=False, want_gz=True)
        models = torch.tensor(wk.rho, dtype=torch.float32, device=DEV).requires_grad_(True)
        gz = gravity(models, pl, "gz")
        J = 0.5 * torch.sum((gz - dz[None]) ** 2)
        J.backward()
        grad = models.grad.double().reshape(16, -1).cpu().numpy()
        resid = (gz - dz[None]).detach().cpu().numpy()
    rng = np.random.default_rng(5)
    vox = np.sort(rng.choice(wk.grid.nvox, 24, replace=False))
    ref = direct.adjoint_subset(wk.grid.n, wk.grid.origin, wk.grid.h, wk.xi, wk.w, wk.obs, resid, wk.G, vox)
    err = rel_l2(grad[:, vox], ref)
    print("adjoint 128^3 x16 mixed p=12 sampled rel L2 %.3e" % err)
    assert err <= 1e-5
