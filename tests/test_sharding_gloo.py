"""Multi-rank path on CPU: two gloo ranks each take a contiguous channel shard,
compute the FP64 oracle gradient of their shard with the design-wide loss
normalisation, and sum with one all-reduce; the result equals the gradient
and loss of the whole design."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import dos_oracle as O
from paper_2604_02624_gb300 import sharding
from paper_2604_02624_gb300 import workloads as W


def _design():
    w = W.workload("tiny")
    return w, W.thickness(w, 0), W.targets(w, 1)


def _shard_grad(w, h, T, lo, hi):
    ws = w.subset(np.arange(lo, hi))
    model = dict(lambdas=ws.lambdas, gaps=ws.gaps, pitch=ws.pitch, m=ws.m, fov=ws.fov,
                 n_index=ws.n_index, kappa=ws.kappa)
    fwd = O.forward(h, aperture=ws.aperture, **model)
    norm = w.n_lambda * w.fov * w.fov           # design-wide normalisation
    dLdI = 2.0 * (fwd["I"] - T[lo:hi]) / norm
    loss = float(np.sum((fwd["I"] - T[lo:hi]) ** 2) / norm)
    return loss, O.backward(h, fwd, dLdI, **model)


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, h, T = _design()
    lo, hi = sharding.shard_range(w.n_lambda, rank, world)
    loss, g = _shard_grad(w, h, T, lo, hi)
    gt = torch.tensor(g)
    total = sharding.reduce_step(gt, loss)
    if rank == 0:
        out.put((total, gt.numpy()))
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_shard_ranges_partition_the_channels():
    for n in (1, 5, 4096, 4097):
        for world in (1, 2, 3, 8):
            r = [sharding.shard_range(n, k, world) for k in range(world)]
            assert r[0][0] == 0 and r[-1][1] == n
            assert all(r[k][1] == r[k + 1][0] for k in range(world - 1))
            sizes = [b - a for a, b in r]
            assert max(sizes) - min(sizes) <= 1


def test_two_gloo_ranks_reproduce_the_full_gradient():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    total, g = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    w, h, T = _design()
    L, _, g_ref, _ = O.loss_and_grad(h, T, lambdas=w.lambdas, gaps=w.gaps, pitch=w.pitch, m=w.m,
                                     fov=w.fov, aperture=w.aperture, n_index=w.n_index, kappa=w.kappa)
    assert abs(total - L) <= 1e-12 * abs(L)
    assert np.max(np.abs(g - g_ref)) <= 1e-12 * np.max(np.abs(g_ref))
