"""world_size-2 gloo test of the multi-rank path (replicas only): barriers,
max-over-ranks timing, unique replica ids, weak-scaling aggregate. CPU only."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    from paper_2602_14975_gb300 import dist as D
    ws = D.init("gloo")
    D.barrier()
    t = D.max_over_ranks(1.5 + rank)          # slowest rank sets the time
    rid = D.replica_id(rank, 3)
    ids = [None] * world
    dist.all_gather_object(ids, rid)
    agg = D.aggregate(100.0, t, ws)
    D.barrier()
    dist.destroy_process_group()
    q.put((rank, ws, t, ids, agg))


def test_two_rank_replicas_only_path():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ws, t, ids, agg in out:
        assert ws == 2
        assert t == 2.5
        assert len(set(ids)) == 2
        assert agg == pytest.approx(100.0 * 2 / 2.5)


def test_single_process_defaults(monkeypatch):
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    from paper_2602_14975_gb300 import dist as D
    assert D.world()[0] == 1
    assert D.max_over_ranks(3.0) == 3.0
