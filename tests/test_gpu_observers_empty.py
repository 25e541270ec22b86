"""Empty observer sets (M = 0) in every mode: the plan builds, the forward
returns empty outputs and the transpose returns zeros, through the C ABI."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1107_5951_gb300 as pkg  # noqa: E402
from paper_1107_5951_gb300 import workloads as wl  # noqa: E402

DEV = "cuda:0"


@pytest.mark.parametrize("mode,precision,voxels", [("direct", "fp64", "quadrature"), ("direct", "mixed", "quadrature"),
                                                   ("fmm", "fp64", "quadrature"), ("fmm", "mixed", "quadrature"),
                                                   ("direct", "fp64", "closed_form")])
def test_no_observers(mode, precision, voxels):
    wk = wl.random_small(3, n=(8, 8, 8), npts=1, n_obs=1, h=(1.0, 1.0, 1.0))
    obs = torch.zeros((0, 3), dtype=torch.float64, device=DEV)
    rho = torch.tensor(np.stack([wk.rho, -wk.rho]), device=DEV)
    with pkg.Plan(wk.grid.n, wk.grid.origin, wk.grid.h, wk.xi, wk.w, obs, mode=mode, precision=precision, p=8,
                  max_batch=2, G=1.0, voxels=voxels) as plan:
        g, gz = plan.forward(rho, want_gz=True)
        grad = plan.adjoint(torch.zeros((2, 0), dtype=torch.float64, device=DEV))
        torch.cuda.synchronize()
        plan.check()
        assert plan.info.M == 0
    assert tuple(g.shape) == (2, 0, 3) and tuple(gz.shape) == (2, 0)
    assert tuple(grad.shape) == (2,) + wk.grid.shape_zyx
    assert torch.count_nonzero(grad).item() == 0
