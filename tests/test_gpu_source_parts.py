"""Source-partitioned FMM (gf_plan_set_source_part): Eq. 1 is linear in the
sources, so the field is the sum of the fields of any partition of them, as
the summation method of Sec. 2.1 splits the voxels over processes and sums
the station vector.  Each part of a partitioned plan must equal the FP64
oracle evaluated on the densities of that part alone (the others zeroed),
and the sum of the parts must equal the unpartitioned plan to rounding --
in one process, and as two processes sharing the GPU whose fields are
summed over a gloo process group (the all-reduce a multi-GPU run does with
NCCL)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1107_5951_gb300 as pkg  # noqa: E402
from oracle import direct  # noqa: E402
from paper_1107_5951_gb300 import gf, workloads as wl  # noqa: E402

DEV = "cuda:0"
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def case(seed=3, n=(30, 26, 22)):
    wk = wl.random_small(seed, n=n, npts=1, n_obs=500, h=(1.0, 1.0, 1.0), origin=(-5.0, 3.0, -20.0), obs_pad=3.0)
    vc = wl.voxel_centres(wk.grid)
    rng = np.random.default_rng(seed)
    wk.obs = np.concatenate([wk.obs, vc[rng.choice(len(vc), 300, replace=False)]])
    return wk


def plan_for(wk, precision, p):
    obs = torch.tensor(wk.obs, dtype=torch.float64, device=DEV)
    return pkg.Plan(wk.grid.n, wk.grid.origin, wk.grid.h, wk.xi, wk.w, obs, mode="fmm", precision=precision, p=p,
                    G=wk.G)


def level2_codes(wk, info):
    """Morton code (x -> bit 0, y -> bit 1, z -> bit 2 per level) of the
    level-2 box that holds each voxel, [nz][ny][nx]."""
    side = int(info.leaf_vox) << (int(info.L) - 2)
    off = [int(v) for v in info.voxel_offset]
    nx, ny, nz = wk.grid.n
    bx = (np.arange(nx) + off[0]) // side
    by = (np.arange(ny) + off[1]) // side
    bz = (np.arange(nz) + off[2]) // side
    z, y, x = np.meshgrid(bz, by, bx, indexing="ij")
    return ((x & 1) | ((y & 1) << 1) | ((z & 1) << 2) | ((x & 2) << 2) | ((y & 2) << 3) | ((z & 2) << 4))


@pytest.mark.parametrize("precision,p,tol_sum,tol_ref", [("fp64", 14, 1e-12, 1e-6), ("mixed", 12, 1e-6, 1e-5)])
@pytest.mark.parametrize("nparts", [2, 3, 8])
def test_parts_sum_to_the_whole_and_each_part_meets_the_oracle(precision, p, tol_sum, tol_ref, nparts):
    wk = case()
    rho = torch.tensor(wk.rho, dtype=torch.float64 if precision == "fp64" else torch.float32, device=DEV)
    with plan_for(wk, precision, p) as plan:
        g_all, _ = plan.forward(rho)
        torch.cuda.synchronize()
        g_all = g_all.cpu().numpy()
        info = plan.info
    codes = level2_codes(wk, info)
    total = np.zeros_like(g_all)
    ranges = []
    for part in range(nparts):
        with plan_for(wk, precision, p) as plan:
            lo, hi = plan.set_source_part(part, nparts)
            ranges.append((lo, hi))
            g, _ = plan.forward(rho)
            torch.cuda.synchronize()
            plan.check()
            g = g.cpu().numpy()
        total += g
        mask = (codes >= lo) & (codes < hi)
        ref = direct.forward(wk.grid.n, wk.grid.origin, wk.grid.h, wk.xi, wk.w, np.where(mask, wk.rho, 0.0),
                             wk.obs, wk.G)
        if mask.any():
            assert rel_l2(g, ref) <= tol_ref, (part, lo, hi)
        else:
            assert np.all(g == 0.0)
    # the parts are consecutive ranges that cover every level-2 box holding voxels
    cover = np.zeros(64, bool)
    for lo, hi in ranges:
        assert not cover[lo:hi].any()
        cover[lo:hi] = True
    assert cover[np.unique(codes)].all()
    assert rel_l2(total, g_all) <= tol_sum


def test_parts_are_balanced_by_voxels():
    wk = wl.layered_scale(n=96, stations=64)
    rho = torch.tensor(wk.rho, dtype=torch.float32, device=DEV)
    with plan_for(wk, "mixed", 8) as plan:
        info = plan.info
    codes = level2_codes(wk, info)
    counts = []
    for part in range(4):
        with plan_for(wk, "mixed", 8) as plan:
            lo, hi = plan.set_source_part(part, 4)
        counts.append(int(((codes >= lo) & (codes < hi)).sum()))
    assert sum(counts) == codes.size
    assert max(counts) <= 1.5 * codes.size / 4
    del rho


def test_partition_limits():
    wk = case(5, (12, 10, 9))
    with plan_for(wk, "fp64", 8) as plan:
        for bad in ((2, 2), (-1, 2), (0, 0), (0, 65)):
            with pytest.raises(gf.GfError) as e:
                plan.set_source_part(*bad)
            assert e.value.status == gf.GF_ERR_INVALID_ARG
        plan.set_source_part(1, 2)
        r = torch.zeros(wk.n_obs, dtype=torch.float64, device=DEV)
        with pytest.raises(gf.GfError) as e:
            plan.adjoint(r)
        assert e.value.status == gf.GF_ERR_UNSUPPORTED
        assert plan.set_source_part(0, 1) == (0, 64)
    obs = torch.tensor(wk.obs, dtype=torch.float64, device=DEV)
    with pkg.Plan(wk.grid.n, wk.grid.origin, wk.grid.h, wk.xi, wk.w, obs, mode="direct", precision="fp64") as plan:
        with pytest.raises(gf.GfError) as e:
            plan.set_source_part(0, 2)
        assert e.value.status == gf.GF_ERR_UNSUPPORTED


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wk = case()
        rho = torch.tensor(wk.rho, dtype=torch.float64, device=DEV)
        with plan_for(wk, "fp64", 14) as plan:
            plan.set_source_part(rank, world)
            g, _ = plan.forward(rho)
            torch.cuda.synchronize()
            g = g.cpu()
        dist.all_reduce(g, op=dist.ReduceOp.SUM)
        out.put((rank, g.numpy()))
    finally:
        dist.destroy_process_group()


def test_two_ranks_on_one_gpu_summed_over_gloo():
    """Two processes each solve their half of the sources (independent
    kernels, no kernel waits on the other process) and sum the fields over a
    gloo group; both end with the single-process field to rounding."""
    import torch.multiprocessing as mp
    wk = case()
    with plan_for(wk, "fp64", 14) as plan:
        g_all, _ = plan.forward(torch.tensor(wk.rho, dtype=torch.float64, device=DEV))
        torch.cuda.synchronize()
        g_all = g_all.cpu().numpy()
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(2)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for _, g in res:
        assert rel_l2(g, g_all) <= 1e-12
