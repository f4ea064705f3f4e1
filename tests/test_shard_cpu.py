"""The multi-rank path on the CPU: the cost partition of independent units
(selective query rows, batch problems) and the final all-gather, with two gloo
ranks in separate processes. Each rank computes its share with a stand-in
executor (the oracle on the host, in place of its GPU); the gathered outputs
must equal the single-process result bit for bit."""
import itertools
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle
import workloads as wl
from paper_2408_10369_gb300 import shard


def test_lpt_partition_covers_every_unit_once_and_is_deterministic():
    rng = np.random.default_rng(0)
    for world in (1, 2, 3, 8):
        costs = rng.exponential(1.0, 101)
        parts = shard.lpt_partition(costs, world)
        assert len(parts) == world
        assert sorted(itertools.chain.from_iterable(parts)) == list(range(101))
        assert parts == shard.lpt_partition(costs, world)
    assert shard.lpt_partition([], 3) == [[], [], []]
    with pytest.raises(ValueError):
        shard.lpt_partition([1.0], 0)


def test_lpt_makespan_within_graham_bound_of_brute_force():
    """Graham's bound for LPT: makespan <= (4/3 - 1/(3m)) OPT, against the
    optimum found by trying every assignment of 9 jobs to 2 and 3 machines."""
    rng = np.random.default_rng(1)
    for trial in range(20):
        costs = rng.integers(1, 50, 9).astype(float)
        for m in (2, 3):
            parts = shard.lpt_partition(costs, m)
            got = max(shard.part_loads(costs, parts))
            opt = min(max(sum(c for c, a in zip(costs, assign) if a == k) for k in range(m))
                      for assign in itertools.product(range(m), repeat=len(costs)))
            assert got <= (4.0 / 3.0 - 1.0 / (3 * m)) * opt + 1e-9, (trial, m, got, opt)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _queries_worker(rank, world, port, n, ip, ix, src, q, res):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        parts = shard.lpt_partition(shard.query_costs(src), world)
        mine = parts[rank]
        # stand-in executor: v_q R1+ for this rank's rows, as packed bit rows
        rows, _ = oracle.smp(n, ip, ix, src[mine]) if mine else (np.zeros((0, n), np.uint8), None)
        local = torch.from_numpy(wl.pack_rows(rows).view(np.int64) if mine
                                 else np.zeros((0, src.shape[1]), np.int64))
        full = shard.gather_rows(local, parts, rank, q)
        res[rank] = full.numpy().copy()
    finally:
        dist.destroy_process_group()


def _problems_worker(rank, world, port, graphs, res):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ns = [g[0] for g in graphs]
        numel = [n * wl.words(n) for n in ns]

        def execute(idx):
            return [torch.from_numpy(wl.pack_rows(oracle.closure(*graphs[i])).view(np.int64).copy()) for i in idx]

        outs, parts = shard.run_sharded(len(graphs), shard.problem_costs(ns), world, rank, execute, numel)
        res[rank] = [o.numpy().copy() for o in outs]
    finally:
        dist.destroy_process_group()


def test_query_rows_sharded_over_two_gloo_ranks():
    n, q = 1500, 37
    ip, ix = wl.powerlaw_csr(n, 2.1, 200, 3)
    src = wl.query_rows(n, q, 1, 9, 4)
    want = wl.pack_rows(oracle.smp(n, ip, ix, src)[0]).view(np.int64)
    with mp.get_context("spawn").Manager() as man:
        res = man.dict()
        mp.spawn(_queries_worker, args=(2, _free_port(), n, ip, ix, src, q, res), nprocs=2, join=True)
        for r in range(2):
            np.testing.assert_array_equal(res[r], want)


def test_problems_sharded_over_two_gloo_ranks():
    sizes = [(300, 1.5, 1), (64, 2.0, 2), (1000, 1.2, 3), (5, 1.0, 4), (777, 1.7, 5), (129, 3.0, 6), (1, 0.0, 7)]
    graphs = []
    for n, d, seed in sizes:
        ip, ix = wl.er_graph(n, d, seed)
        graphs.append((n, ip, ix))
    want = [wl.pack_rows(oracle.closure(*g)).view(np.int64).ravel() for g in graphs]
    with mp.get_context("spawn").Manager() as man:
        res = man.dict()
        mp.spawn(_problems_worker, args=(2, _free_port(), graphs, res), nprocs=2, join=True)
        for r in range(2):
            assert len(res[r]) == len(graphs)
            for got, w in zip(res[r], want):
                np.testing.assert_array_equal(got, w)


def _flat_worker(rank, world, port, numel, parts_costs, res):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        parts = shard.lpt_partition(parts_costs, world)
        offs, cap = shard.share_layout(parts, rank, numel)
        buf = torch.zeros(cap, dtype=torch.int64)
        for i in parts[rank]:  # unit i's output: numel[i] words of value 1000 * i + k
            buf[offs[i]:offs[i] + numel[i]] = 1000 * i + torch.arange(numel[i])
        out = shard.gather_flat(buf, parts, numel)
        res[rank] = [o.numpy().copy() for o in out]
    finally:
        dist.destroy_process_group()


def test_gather_flat_over_two_gloo_ranks():
    numel = [5, 1, 17, 3, 8, 2, 11]
    costs = [3.0, 9.0, 1.0, 4.0, 4.0, 7.0, 2.0]
    with mp.get_context("spawn").Manager() as man:
        res = man.dict()
        mp.spawn(_flat_worker, args=(2, _free_port(), numel, costs, res), nprocs=2, join=True)
        for r in range(2):
            for i, w in enumerate(numel):
                np.testing.assert_array_equal(res[r][i], 1000 * i + np.arange(w))
