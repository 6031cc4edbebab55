"""Multi-process host logic on CPU: two gloo ranks run the same setup, barrier
and max-over-ranks timing reduction the bench uses under torchrun (one process
per GPU; ECB shards by buffer with no data-path collective)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    from paper_1201_0398_gb300 import dist

    r = dist.setup(backend="gloo")
    dist.barrier(r)
    elapsed = 1.0 + rank  # rank 1 is the slower one
    job = dist.max_over_ranks(r, elapsed)
    seed = dist.shard_seed(1, r)
    dist.barrier(r)
    dist.teardown(r)
    q.put((rank, job, seed, r.world, r.distributed))


def test_two_gloo_ranks_share_max_time_and_distinct_shards():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(i, 2, port, q)) for i in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [2.0, 2.0]  # every rank sees the slowest rank's time
    assert out[0][2] != out[1][2]  # each rank enciphers its own data
    assert all(o[3] == 2 and o[4] for o in out)


def test_single_process_needs_no_group(monkeypatch):
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    from paper_1201_0398_gb300 import dist

    r = dist.setup()
    assert not r.distributed and dist.max_over_ranks(r, 3.5) == 3.5
    dist.barrier(r)
    dist.teardown(r)
