"""The Python binding refuses buffers the kernels would read or write out of
bounds (host tensors where device memory is expected, wrong dtypes, sizes or
devices, non-contiguous views) before any call into the library.  Runs
without a GPU: the plan and server objects are built without their C
handles, so a check that let a bad buffer through would fail on the NULL
handle instead of raising the binding's own error."""
import numpy as np
import pytest
import torch

from paper_1107_5951_gb300 import gf

CUDA0 = torch.device("cuda", 0)


def _plan(shape=(4, 3, 2), M=5):
    pl = object.__new__(gf.Plan)
    pl.shape = shape
    pl.M = M
    pl.max_batch = 4
    pl.device = CUDA0
    pl.handle = None
    return pl


def test_check_tensor_accepts_and_rejects():
    t = torch.zeros(6, dtype=torch.float64)
    gf._check_tensor(t, "t", 6, None)
    with pytest.raises(ValueError):
        gf._check_tensor(t, "t", 7, None)
    with pytest.raises(TypeError):
        gf._check_tensor(t.float(), "t", 6, None)
    with pytest.raises(TypeError):
        gf._check_tensor(t, "t", 6, CUDA0)              # host tensor where device memory is needed
    with pytest.raises(ValueError):
        gf._check_tensor(torch.zeros(3, 4, dtype=torch.float64).t(), "t", 12, None)
    with pytest.raises(TypeError):
        gf._check_tensor(np.zeros(6), "t", 6, None)
    gf._check_tensor(t.float(), "t", 6, None, (torch.float32, torch.float64))


def test_check_array_accepts_and_rejects():
    gf._check_array(np.zeros(5), "a", 5)
    with pytest.raises(ValueError):
        gf._check_array(np.zeros(4), "a", 5)
    with pytest.raises(TypeError):
        gf._check_array(np.zeros(5, dtype=np.float32), "a", 5)
    with pytest.raises(TypeError):
        gf._check_array(np.zeros((5, 2))[:, 0], "a", 5)
    ro = np.zeros(5)
    ro.setflags(write=False)
    with pytest.raises(TypeError):
        gf._check_array(ro, "a", 5)
    with pytest.raises(TypeError):
        gf._check_array(torch.zeros(5, dtype=torch.float64), "a", 5)


def test_plan_forward_refuses_host_and_misshapen_densities():
    pl = _plan()
    with pytest.raises(TypeError):
        pl.forward(torch.zeros((2, 3, 4), dtype=torch.float64))       # host memory
    with pytest.raises(ValueError):
        pl.forward(torch.zeros((3, 2, 4), dtype=torch.float64))       # (nz, ny, nx) is (2, 3, 4)
    with pytest.raises(ValueError):
        pl.forward(torch.zeros(24, dtype=torch.float64))


def test_plan_adjoint_refuses_host_weights_and_bad_sizes():
    pl = _plan()
    with pytest.raises(TypeError):
        pl.adjoint(torch.zeros(5, dtype=torch.float64))                 # host memory
    with pytest.raises(ValueError):
        pl.adjoint(torch.zeros(5, dtype=torch.float64), ncomp=2)


def test_server_submit_refuses_mismatched_outputs():
    srv = object.__new__(gf.Server)
    srv._device_index = 0
    srv._pending = {}
    srv.handle = None
    obs = np.zeros((5, 3))
    srv._geoms = {1: (None, None, obs, (4, 3, 2))}
    rho = np.zeros((2, 3, 4))
    with pytest.raises(ValueError):
        srv.submit(1, np.zeros((4, 3, 2)))
    with pytest.raises(ValueError):
        srv.submit(1, rho, gz=np.zeros(4))
    with pytest.raises(TypeError):
        srv.submit(1, rho, gz=np.zeros(5, dtype=np.float32))
    with pytest.raises(TypeError):
        srv.submit(1, rho.astype(np.int64))
    with pytest.raises(ValueError):
        srv.submit(1, torch.zeros((2, 3, 4), dtype=torch.float64), gz=torch.zeros(6, dtype=torch.float64))
    with pytest.raises(TypeError):
        srv.submit(1, torch.zeros((2, 3, 4), dtype=torch.float64), want_g=True,
                   g=torch.zeros(15, dtype=torch.float32))
    srv.handle = None
    srv._geoms = {}
