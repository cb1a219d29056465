"""Multi-rank logic of the data-parallel path on CPU ranks (gloo, world size 2).

Each rank computes the checker's hypergradient over its shard of a small batch; the all-reduced,
pair-weighted mean must equal the full-batch hypergradient of eq. (5.2)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2412_08264_gb300.parallel import allreduce_mean, shard_pairs


def test_shard_pairs_balances_and_covers():
    pixels = [128 * 128, 512 * 512, 256 * 256, 192 * 192, 384 * 384, 128 * 128, 512 * 512]
    for world in [1, 2, 3]:
        sh = shard_pairs(pixels, world)
        assert sorted(sum(sh, [])) == list(range(len(pixels)))
        loads = [sum(pixels[k] for k in s) for s in sh]
        assert max(loads) - min(loads) <= max(pixels)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2412_08264_gb300 import synth
    from oracle.bilevel import BilevelProblem
    wl = synth.uneven_foe([(9, 10), (8, 12), (11, 9), (10, 10), (7, 13)], n_filters=2, f=3, blur_radius=2, seed=5)
    full = BilevelProblem(wl)
    th = wl.theta0
    shards = shard_pairs([p.height * p.width for p in wl.pairs], world)
    mine = shards[rank]
    grads = []
    for k in mine:
        ll = full.lowers[k]
        from oracle.lbfgs import lbfgs
        x, _ = lbfgs(lambda v: ll.value(v.reshape(ll.h, ll.w), th), lambda v: ll.grad(v.reshape(ll.h, ll.w), th).reshape(-1),
                     np.zeros(ll.n), 1e-7)
        x = x.reshape(ll.h, ll.w)
        w = full.reference_w(k, x, th)
        grads.append(full.Jw(k, x, th, w))
    local = torch.tensor(np.mean(grads, axis=0), dtype=torch.float64)
    g = allreduce_mean(local, len(mine))
    if rank == 0:
        out_q.put(g.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_mean_hypergradient_equals_full_batch():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = q.get(timeout=240)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    from paper_2412_08264_gb300 import synth
    from oracle.bilevel import BilevelProblem
    wl = synth.uneven_foe([(9, 10), (8, 12), (11, 9), (10, 10), (7, 13)], n_filters=2, f=3, blur_radius=2, seed=5)
    prob = BilevelProblem(wl)
    xs, _ = prob.solve_lower(wl.theta0, gtol=1e-7)
    ws = [prob.reference_w(k, xs[k], wl.theta0) for k in range(prob.K)]
    ref = prob.hypergradient(wl.theta0, xs, ws)
    np.testing.assert_allclose(got, ref, rtol=1e-6, atol=1e-9 * np.abs(ref).max())
