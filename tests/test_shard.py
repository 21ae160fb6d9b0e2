"""Sharding a batch of independent instances over ranks: the ranges, and a
world-size-2 run over gloo on the CPU in which each rank computes one Wave-ADR
cycle of its instances (the oracle stands in for the GPU here) and the results
are gathered on the host, compared with one process doing the whole batch."""
import os
import socket

import numpy as np
import pytest

from paper_2404_02493_gb300.shard import gather_to_host, my_shard, shard_ranges


def test_ranges_cover_contiguously_and_balance():
    work = [n * n for n in (255, 511, 1023) * 21 + (255,)]
    for world in (1, 2, 3, 4, 8):
        rs = shard_ranges(work, world)
        assert len(rs) == world and rs[0][0] == 0 and rs[-1][1] == len(work)
        assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
        share = sum(work) / world
        for lo, hi in rs:
            assert abs(sum(work[lo:hi]) - share) <= max(work) + 1e-9
        assert sorted(i for r in range(world) for i in my_shard(work, r, world)) == list(range(len(work)))


def test_more_ranks_than_instances():
    rs = shard_ranges([1.0, 1.0], 4)
    assert [hi - lo for lo, hi in rs].count(1) == 2 and sum(hi - lo for lo, hi in rs) == 2
    with pytest.raises(ValueError):
        shard_ranges([1.0], 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _instances():
    import synth
    return [synth.config_lognormal(n=n, omega=0.4 * n * np.pi / 5, seed=60 + i)
            for i, n in enumerate((31, 47, 23, 39, 31))]


def _cycle_all(idx):
    from oracle.cycle import CycleParams, Hierarchy
    out = {}
    for i in idx:
        I = _instances()[i]
        H = Hierarchy(I.n, I.k, I.phi, I.omega, I.bc, CycleParams(n_cmax=7))
        out[i] = H.cycle(np.zeros_like(I.g), I.g)
    return out


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        work = [I.n * I.n for I in _instances()]
        mine = my_shard(work, rank, world)
        res = gather_to_host(_cycle_all(mine), world)
        if rank == 0:
            q.put({k: v.tolist() for k, v in res.items()})
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo_gather_equals_single_process():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=180)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ref = _cycle_all(range(len(_instances())))
    assert sorted(got) == sorted(ref)
    for k, v in ref.items():
        assert np.array_equal(np.asarray(got[k]), v)
