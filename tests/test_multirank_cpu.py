"""Multi-rank domain decomposition on CPU ranks (gloo, world size 2).

The single-problem path ships as replicas only (every box has one GPU); the natural
multi-GPU form is a slab decomposition along the slowest axis with a halo of depth K
exchanged every K steps (a ring for periodic boundaries; the end ranks apply the
Neumann / Dirichlet rule themselves).  These tests run that exchange between two gloo
processes, each stepping its slab plus halos with the FP64 oracle, and check that the
gathered state is bit-identical to the single-domain oracle run -- the property a GPU
implementation of the decomposition must keep.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from workloads import dt_rule, uniform_field


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, shape, bc, steps, K, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n0 = shape[0]
        eps = 0.03
        h = 1.0 / max(shape)
        dt = dt_rule(len(shape), eps, h)
        full = uniform_field(shape, -1, 1, 123)
        r0, r1 = rank * n0 // world, (rank + 1) * n0 // world
        periodic = bc == 0
        has_lo = periodic or rank > 0
        has_hi = periodic or rank < world - 1
        own = full[r0:r1].copy()
        lo_nb, hi_nb = (rank - 1) % world, (rank + 1) % world
        done = 0
        while done < steps:
            k = min(K, steps - done)
            # exchange k boundary slabs with the neighbours (ring for periodic)
            parts = []
            reqs = []
            recv_lo = torch.empty((k,) + own.shape[1:], dtype=torch.float64)
            recv_hi = torch.empty((k,) + own.shape[1:], dtype=torch.float64)
            send_lo = torch.from_numpy(own[:k].copy())
            send_hi = torch.from_numpy(own[-k:].copy())
            if has_lo:
                reqs.append(dist.isend(send_lo, lo_nb, tag=1))
                reqs.append(dist.irecv(recv_lo, lo_nb, tag=2))
            if has_hi:
                reqs.append(dist.isend(send_hi, hi_nb, tag=2))
                reqs.append(dist.irecv(recv_hi, hi_nb, tag=1))
            for r in reqs:
                r.wait()
            if has_lo:
                parts.append(recv_lo.numpy())
            parts.append(own)
            if has_hi:
                parts.append(recv_hi.numpy())
            ext = np.concatenate(parts, axis=0)
            # k steps on the extended slab; the array edges that are rank boundaries get
            # a wrong ghost, but its error travels one row per step and never reaches
            # the owned rows within k steps
            ext = oracle.run_fd(ext, eps, dt, h, bc, k)
            a = k if has_lo else 0
            own = ext[a:a + (r1 - r0)].copy()
            done += k
        t = torch.from_numpy(own.copy())
        sizes = [(i + 1) * n0 // world - i * n0 // world for i in range(world)]
        buf = [torch.empty((sz,) + own.shape[1:], dtype=torch.float64) for sz in sizes]
        for i, b in enumerate(buf):  # slabs may differ in size: one broadcast per rank
            if i == rank:
                b.copy_(t)
            dist.broadcast(b, i)
        if rank == 0:
            np.save(out_path, torch.cat(buf, 0).numpy())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("shape,bc,K", [((24, 20), 0, 1), ((24, 20), 1, 2), ((16, 12, 10), 2, 3),
                                        ((17, 9, 8), 0, 2)], ids=str)
def test_slab_decomposition_is_bitwise(tmp_path, shape, bc, K):
    steps = 7
    out = str(tmp_path / "gathered.npy")
    mp.start_processes(_rank_main, args=(2, _free_port(), shape, bc, steps, K, out), nprocs=2, join=True,
                       start_method="spawn")
    got = np.load(out)
    eps = 0.03
    h = 1.0 / max(shape)
    ref = oracle.run_fd(uniform_field(shape, -1, 1, 123), eps, dt_rule(len(shape), eps, h), h, bc, steps)
    assert np.array_equal(got, ref)
