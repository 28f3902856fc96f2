"""Multi-rank host logic on CPU: world-size-2 gloo ranks shard the samples of
the same work items and merge their sums; the result equals one rank's sums
over the union of the samples (exactly for integer estimators)."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2502_07123_gb300 import distributed as D
from paper_2502_07123_gb300 import workloads as W


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _oracle_sums(items, seed):
    from oracle import core
    out = []
    for it in items:
        s, _ = core.level(it["p"], it["level"], it["first_sample"], it["N"], it["variant"], seed,
                          fmt=W.default_format(it["p"], it["level"]))
        out.append(s)
    return out


ITEMS = [dict(p=W.params(), level=0, variant=W.FIXED_APPROX, N=1001),
         dict(p=W.params(payoff=W.DIGITAL), level=3, variant=W.FIXED_APPROX, N=333),
         dict(p=W.params(), level=2, variant=W.CORR_FIXED, N=250)]


def _worker(rank, world, port, mode, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = D.shard_weak(ITEMS, rank) if mode == "weak" else D.shard_strong(ITEMS, rank, world)
    merged = D.allgather_merge(_oracle_sums(mine, 5))
    if rank == 0:
        q.put(merged)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("mode", ["weak", "strong"])
def test_two_rank_merge_equals_single_rank(mode):
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, mode, q)) for r in range(world)]
    for p in procs:
        p.start()
    merged = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    union = []
    for it in ITEMS:
        d = dict(it)
        d["first_sample"] = 0
        d["N"] = it["N"] * world if mode == "weak" else it["N"]
        union.append(d)
    ref = _oracle_sums(union, 5)
    for mm, rr, it in zip(merged, ref, ITEMS):
        assert mm["n"] == rr["n"]
        if it["variant"] == W.FIXED_APPROX:
            assert mm["isum"] == rr["isum"] and mm["isum2"] == rr["isum2"]
        assert abs(mm["sum"] - rr["sum"]) <= 1e-12 * max(1.0, abs(rr["sum"])) * 10
        assert abs(mm["sum2"] - rr["sum2"]) <= 1e-12 * abs(rr["sum2"]) * 10


def test_shards_are_disjoint_and_cover():
    items = [dict(N=10, first_sample=3), dict(N=7)]
    for world in (1, 2, 3, 4):
        for i, it in enumerate(items):
            got = []
            for r in range(world):
                s = D.shard_strong(items, r, world)[i]
                got.extend(range(s["first_sample"], s["first_sample"] + s["N"]))
            f = it.get("first_sample", 0)
            assert got == list(range(f, f + it["N"]))
            weak = [D.shard_weak(items, r)[i]["first_sample"] for r in range(world)]
            assert weak == [f + r * it["N"] for r in range(world)]
