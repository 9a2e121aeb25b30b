"""The multi-rank path of the benchmark on CPU ranks (gloo, world size 2):
replicas draw distinct seeded instances, whole instances are sharded over
ranks disjointly and completely, and the job's time is the slowest rank's
(no collective touches the data path; only the timing is reduced)."""
import importlib.util
import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b = _bench()
    w, r, lr = b.rank_env()
    items = list(range(11))
    mine = b.shard(items, r, w)
    t = 1.5 + r  # rank 1 is the slow one
    res = {"world": w, "rank": r, "local": lr, "seed": b.rank_seed(7, r), "mine": mine,
           "max": b.max_over_ranks(t, w), "sum": b.sum_over_ranks(len(mine), w)}
    dist.barrier()
    dist.destroy_process_group()
    out.put(res)


def test_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=120) for _ in procs], key=lambda x: x["rank"])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [x["world"] for x in res] == [2, 2] and [x["local"] for x in res] == [0, 1]
    assert res[0]["seed"] != res[1]["seed"]
    assert sorted(res[0]["mine"] + res[1]["mine"]) == list(range(11))
    assert not set(res[0]["mine"]) & set(res[1]["mine"])
    assert res[0]["max"] == res[1]["max"] == 2.5
    assert res[0]["sum"] == res[1]["sum"] == 11


def test_single_rank_defaults(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    b = _bench()
    assert b.rank_env() == (1, 0, 0)
    assert b.shard([1, 2, 3], 0, 1) == [1, 2, 3]
    assert b.max_over_ranks(3.0, 1) == 3.0
