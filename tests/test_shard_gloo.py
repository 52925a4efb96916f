"""Sharding of the fitness path across ranks, checked on CPU with the gloo
backend (world size 2): population ranges partition the trees,
point-sharded MSEs combined by one all-reduce equal the unsharded MSE, and a
generation whose fitness is sharded by population (one all-gather) and whose
selection and operators are replicated gives every rank the same children as
one process."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2501_17168_gb300 import shard, workloads as W


def test_population_and_point_ranges_partition():
    for n in (0, 1, 7, 100, 5001):
        for world in (1, 2, 3, 8):
            rs = [shard.population_range(n, r, world) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
            sizes = [b - a for a, b in rs]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    prob = W.sr_small(3)
    y = np.random.default_rng(0).standard_normal((prob.D, 1)).astype(np.float32)
    a, b = shard.point_range(prob.D, rank, world)
    m, _ = oracle.mse(prob.pop.type, prob.pop.val, prob.pop.size, prob.X[a:b], y[a:b], threads=1)
    # each rank contributes its sum of squared residuals (what the library's
    # TGP_FLAG_SSE mode returns); the oracle's mean times the local count is it
    full = shard.combine_point_shards(torch.from_numpy(m * float(b - a)), prob.D)
    if rank == 0:
        ref, _ = oracle.mse(prob.pop.type, prob.pop.val, prob.pop.size, prob.X, y, threads=1)
        q.put(float(np.nanmax(np.abs(full.numpy() - ref) / np.maximum(np.abs(ref), 1e-300))))
    torch.distributed.destroy_process_group()


def test_point_sharded_mse_equals_unsharded():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert q.get(timeout=10) < 1e-12


def _generation_worker(rank, world, port, q):
    import oracle
    from oracle import genetic
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    prob = W.sr_small(4)
    pop3 = (prob.pop.type, prob.pop.val, prob.pop.size)
    y = np.random.default_rng(1).standard_normal((prob.D, 1)).astype(np.float32)
    a, b = shard.population_range(prob.pop.pop, rank, world)
    m, _ = oracle.mse(*(t[a:b] for t in pop3), prob.X, y, threads=1)
    fit = shard.gather_fitness(torch.from_numpy(m[:, 0]), prob.pop.pop).numpy()
    P = prob.pop.pop
    words = W.random_words(5, (2 * P, 20))
    win = genetic.tournament(fit, words)
    k, j = W.random_words(6, P), W.random_words(7, P)
    kids = genetic.subtree_exchange(pop3, pop3, win[:P], k, win[P:], j, genetic.RANDOM,
                                    prob.pop.max_len, prob.pop.max_len)
    q.put((rank, fit, kids[0], kids[2], kids[3]))
    torch.distributed.destroy_process_group()


def test_population_sharded_generation_matches_one_process():
    import oracle
    from oracle import genetic
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_generation_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    prob = W.sr_small(4)
    pop3 = (prob.pop.type, prob.pop.val, prob.pop.size)
    y = np.random.default_rng(1).standard_normal((prob.D, 1)).astype(np.float32)
    m, _ = oracle.mse(*pop3, prob.X, y, threads=1)
    P = prob.pop.pop
    win = genetic.tournament(m[:, 0], W.random_words(5, (2 * P, 20)))
    kids = genetic.subtree_exchange(pop3, pop3, win[:P], W.random_words(6, P), win[P:],
                                    W.random_words(7, P), genetic.RANDOM, prob.pop.max_len,
                                    prob.pop.max_len)
    for rank, fit, t, s, st in got:
        assert np.array_equal(fit, m[:, 0], equal_nan=True)
        assert np.array_equal(t, kids[0], equal_nan=True) and np.array_equal(s, kids[2], equal_nan=True)
        assert (st == kids[3]).all()


def _gather_worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    for P in (1, 2, 7, 64):
        a, b = shard.population_range(P, rank, world)
        local = torch.arange(a, b, dtype=torch.float64) * 0.5
        full = shard.gather_fitness(local, P)
        q.put((rank, P, full.tolist()))
    torch.distributed.destroy_process_group()


def test_gather_fitness_with_uneven_slices():
    """Three ranks, populations that do not divide evenly (and one smaller
    than the world): every rank gets the whole vector in tree order."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    world = 3
    procs = [ctx.Process(target=_gather_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(4 * world)]
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for rank, P, full in got:
        assert full == [0.5 * i for i in range(P)], (rank, P)
