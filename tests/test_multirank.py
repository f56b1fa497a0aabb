"""Replica timing over several ranks (gloo, CPU): every rank sees the slowest rank's time."""
import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(10.0 * (rank + 1), device="cpu")
    out[rank] = t
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_max_over_ranks_with_gloo(world):
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert dict(out) == {r: 10.0 * world for r in range(world)}


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5


def _shard_worker(rank, world, port, out):
    import numpy as np
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import jacobian as jb
    from oracle.nufft import KBNufft
    from paper_2111_02912_gb300.shard import allreduce_vjp, coil_slice
    from paper_2111_02912_gb300.workloads import gaussian_bump_maps, random_image, random_omega, rng
    g = rng(77)
    shape, M, C = (16, 12), 300, 5
    x = random_image(g, shape)
    om = random_omega(g, 2, M)
    S = gaussian_bump_maps(shape, C)
    v = g.standard_normal((C, M)) + 1j * g.standard_normal((C, M))
    op = KBNufft(shape, om)
    sl = coil_slice(C, rank, world)
    go, gx = jb.vjp_omega_x(op, x, v[sl], S[sl])        # this rank's coils only
    go_t, gx_t = torch.from_numpy(np.ascontiguousarray(go)), torch.from_numpy(np.ascontiguousarray(gx))
    allreduce_vjp(go_t, gx_t)
    if rank == 0:
        go_all, gx_all = jb.vjp_omega_x(op, x, v, S)
        out["err_omega"] = float(np.abs(go_t.numpy() - go_all).max() / np.abs(go_all).max())
        out["err_x"] = float(np.abs(gx_t.numpy() - gx_all).max() / np.abs(gx_all).max())
    dist.barrier()
    dist.destroy_process_group()


def test_coil_shard_reduction_with_gloo():
    """Two ranks, each the VJP of its block of 5 coils (3 + 2); one all-reduce gives the all-coil
    gradients of Eq. (e,jac,Ax,v) (Sec. II-G sums over coils)."""
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = 30500 + os.getpid() % 1000
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        assert p.exitcode == 0
    assert out["err_omega"] < 1e-12 and out["err_x"] < 1e-12


def test_coil_slices_cover_every_coil_once():
    sys.path.insert(0, ROOT)
    from paper_2111_02912_gb300.shard import coil_slice
    for C in (1, 5, 16, 33):
        for world in (1, 2, 3, 8):
            seen = [c for r in range(world) for c in range(C)[coil_slice(C, r, world)]]
            assert seen == list(range(C))
