"""Host-side logic of the multi-GPU replica path, run as two gloo ranks on CPU: distinct
chain seeds per rank, max-over-ranks timing, and the barrier (bench.py)."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    w, r, lr = bench.dist_env()
    t = bench.max_over_ranks(1.0 + rank, w)
    bench.barrier(w)
    q.put((r, lr, w, t, bench.chain_seed(0, r)))
    dist.destroy_process_group()


def test_two_rank_replica_helpers():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1] and all(r[2] == 2 for r in res)
    assert all(r[3] == 2.0 for r in res)              # max over ranks of (1 + rank)
    assert res[0][4] != res[1][4]                     # independent chains


def test_single_rank_defaults(monkeypatch):
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_env() == (1, 0, 0)
    assert bench.max_over_ranks(3.5, 1) == 3.5
