"""Continuous-batching server.

CPU (dry run, no GPU): admission order and budget, batching, injected faults,
open-loop replay, a producer stopped mid-run, draining and argument errors.
GPU: every request's output equals the single-message kernel's output for the
same request alone (and the oracle on a sample), the budget is never exceeded,
and batches overlap on the device."""
import numpy as np
import pytest

import oracle


def fake_requests(g, n, rng, max_blocks=64, nkeys=4, rate=None):
    r = np.zeros(n, g.REQUEST)
    r["id"] = np.arange(n)
    r["nblocks"] = rng.integers(1, max_blocks + 1, n)
    r["in_ptr"] = 1 << 20
    r["out_ptr"] = 2 << 20
    r["key_index"] = rng.integers(0, nkeys, n)
    r["decrypt"] = rng.integers(0, 2, n)
    if rate:
        r["arrival_s"] = np.cumsum(rng.exponential(1.0 / rate, n))
    return r


def keyset(g, n=4):
    return [g.Key(bytes([i]) * (16, 24, 32)[i % 3]) for i in range(n)]


def test_dryrun_submit_drain_and_stats(gbaes):
    srv = gbaes.Server(keyset(gbaes), budget_bytes=1 << 20, nstreams=3, dryrun=True)
    rng = np.random.default_rng(0)
    reqs = fake_requests(gbaes, 500, rng)
    for r in reqs:
        srv.submit(int(r["id"]), int(r["key_index"]), int(r["in_ptr"]), int(r["out_ptr"]), int(r["nblocks"]),
                   bool(r["decrypt"]))
    srv.drain(10.0)
    done = srv.poll_all()
    assert sorted(done["id"].tolist()) == list(range(500))
    assert (done["status"] == 0).all()
    st = srv.stats()
    assert st["submitted"] == st["completed"] == 500 and st["failed"] == 0
    assert 1 <= st["batches"] <= 500
    assert st["max_inflight_bytes"] <= 1 << 20
    assert (done["done_s"] >= done["launch_s"]).all() and (done["launch_s"] >= done["arrival_s"]).all()
    srv.close()


def test_budget_refusal_and_admission_limit(gbaes):
    srv = gbaes.Server(keyset(gbaes), budget_bytes=32 * 100, nstreams=2, dryrun=True)
    with pytest.raises(gbaes.AesError) as e:  # 101 blocks need 3,232 bytes in+out > 3,200
        srv.submit(1, 0, 1 << 20, 2 << 20, 101)
    assert e.value.name == "AES_ERR_BUDGET"
    for i in range(50):
        srv.submit(i, 0, 1 << 20, 2 << 20, 100)  # each fills the whole budget: one per batch
    srv.drain(10.0)
    st = srv.stats()
    assert st["rejected"] == 1 and st["completed"] == 50
    assert st["max_inflight_bytes"] <= 3200 and st["max_batch_msgs"] == 1
    srv.close()


def test_injected_fault_fails_one_batch_and_server_continues(gbaes):
    srv = gbaes.Server(keyset(gbaes), budget_bytes=32 * 10, nstreams=1, dryrun=True)
    srv.inject_fault(3)
    for i in range(20):
        srv.submit(i, 0, 1 << 20, 2 << 20, 10)  # one request per batch
    srv.drain(10.0)
    done = srv.poll_all()
    assert len(done) == 20
    failed = done[done["status"] != 0]
    assert len(failed) == 1 and failed["status"][0] == -7
    assert srv.stats()["failed"] == 1
    srv.close()


def test_open_loop_replay_and_producer_stop(gbaes):
    rng = np.random.default_rng(1)
    srv = gbaes.Server(keyset(gbaes), dryrun=True)
    reqs = fake_requests(gbaes, 20_000, rng, rate=200_000.0)  # ~0.1 s of arrivals
    srv.replay(reqs)
    srv.replay_join()
    srv.drain(10.0)
    done = srv.poll_all()
    assert len(done) == 20_000 and (done["status"] == 0).all()
    # FIFO admission: nobody waits behind later arrivals for long (no starvation)
    assert float((done["done_s"] - done["arrival_s"]).max()) < 1.0
    # arrivals are the scheduled times: strictly increasing like the schedule
    order = np.argsort(done["id"])
    arr = done["arrival_s"][order]
    assert np.all(np.diff(arr) >= 0)
    assert np.allclose(np.diff(arr), np.diff(reqs["arrival_s"]), atol=1e-9)
    # a producer stopped early: the server drains what was submitted
    slow = fake_requests(gbaes, 1000, rng, rate=1000.0)  # 1 s of arrivals
    srv.replay(slow)
    import time

    time.sleep(0.05)
    srv.replay_join(stop_early=True)
    srv.drain(10.0)
    got = srv.poll_all()
    assert 0 < len(got) < 1000
    srv.close()


def test_cancel_waiting_requests(gbaes):
    # Budget for one request at a time: later submissions wait for admission
    # and can be cancelled; the running one cannot.
    srv = gbaes.Server(keyset(gbaes), budget_bytes=32 * 100, nstreams=1, dryrun=True, dryrun_batch_us=2000)
    for i in range(200):
        srv.submit(i, 0, 1 << 20, 2 << 20, 100)
    for i in range(100, 200):
        srv.cancel(i)
    srv.cancel(10_000)  # unknown id: ignored
    srv.drain(10.0)
    done = srv.poll_all()
    assert len(done) == 200
    st = dict(zip(done["id"].tolist(), done["status"].tolist()))
    assert all(st[i] == 0 for i in range(50))  # well before the cancels arrived
    cancelled = [i for i in range(200) if st[i] == -8]
    assert cancelled and all(i >= 100 for i in cancelled)
    srv.close()


def test_idle_server_sleeps_and_wakes(gbaes):
    import time

    srv = gbaes.Server(keyset(gbaes), dryrun=True)
    time.sleep(0.05)  # idle: the scheduler waits on its condition variable
    t0 = time.perf_counter()
    srv.submit(1, 0, 1 << 20, 2 << 20, 4)
    srv.drain(5.0)
    assert time.perf_counter() - t0 < 0.5
    assert len(srv.poll_all()) == 1
    srv.close()


def test_server_argument_errors(gbaes):
    srv = gbaes.Server(keyset(gbaes, 2), dryrun=True)
    with pytest.raises(gbaes.AesError):
        srv.submit(0, 5, 1 << 20, 2 << 20, 4)  # key index out of range
    with pytest.raises(gbaes.AesError) as e:
        srv.submit(0, 0, (1 << 20) + 8, 2 << 20, 4)
    assert e.value.name == "AES_ERR_ALIGN"
    bad = fake_requests(gbaes, 3, np.random.default_rng(2), rate=10.0)[::-1].copy()  # decreasing arrivals
    with pytest.raises(gbaes.AesError):
        srv.replay(bad)
    srv.close()
    with pytest.raises(gbaes.AesError):
        gbaes.Server([], dryrun=True)


# ------------------------------------------------------------------------- GPU

torch = pytest.importorskip("torch")


def device_requests(g, rng, n, keys_bits, pool_bytes, max_len, rate):
    """Requests over one input pool and disjoint output slices."""
    lengths = (np.exp(rng.uniform(np.log(64), np.log(max_len), n)) // 16 * 16).astype(np.int64)
    lengths = np.maximum(lengths, 16)
    x = torch.from_numpy(rng.integers(0, 256, pool_bytes, dtype=np.uint8)).cuda()
    out_off = np.concatenate([[0], np.cumsum(lengths)[:-1]])
    y = torch.zeros(int(lengths.sum()), dtype=torch.uint8, device="cuda")
    in_off = (rng.integers(0, (pool_bytes - lengths) // 16 + 1) * 16).astype(np.int64)
    r = np.zeros(n, g.REQUEST)
    r["id"] = np.arange(n)
    r["in_ptr"] = x.data_ptr() + in_off
    r["out_ptr"] = y.data_ptr() + out_off
    r["nblocks"] = lengths // 16
    r["key_index"] = rng.integers(0, len(keys_bits), n)
    r["decrypt"] = rng.integers(0, 2, n)
    r["arrival_s"] = np.cumsum(rng.exponential(1.0 / rate, n))
    return r, x, y, in_off, out_off, lengths


@pytest.mark.gpu
@pytest.mark.parametrize("budget,nstreams,threads,bpt", [(8 << 30, 4, 512, 1), (1 << 20, 2, 1024, 2),
                                                          (64 << 20, 8, 256, 4)])
def test_server_results_equal_alone_and_oracle(gbaes, budget, nstreams, threads, bpt):
    rng = np.random.default_rng(budget % 1000 + nstreams)
    nkeys = 64
    bits = rng.choice([128, 192, 256], nkeys)
    raw_keys = [rng.integers(0, 256, b // 8, dtype=np.uint8).tobytes() for b in bits]
    keys = [gbaes.Key(k) for k in raw_keys]
    reqs, x, y, in_off, out_off, lengths = device_requests(gbaes, rng, 4000, bits, 8 << 20, 256 << 10, 100_000.0)
    srv = gbaes.Server(keys, budget_bytes=budget, nstreams=nstreams, threads=threads, blocks_per_thread=bpt)
    srv.replay(reqs)
    srv.replay_join()
    srv.drain(60.0)
    done = srv.poll_all()
    st = srv.stats()
    srv.close()
    assert len(done) == len(reqs) and (done["status"] == 0).all()
    assert st["max_inflight_bytes"] <= budget
    # every request alone through the single-message kernel
    alone = torch.zeros_like(y)
    for i in range(len(reqs)):
        a, b, n = int(in_off[i]), int(out_off[i]), int(lengths[i])
        gbaes.ecb_ex(keys[int(reqs["key_index"][i])], x[a:a + n], alone[b:b + n], decrypt=bool(reqs["decrypt"][i]))
    torch.cuda.synchronize()
    assert torch.equal(alone, y)
    xs = x.cpu().numpy()
    ys = y.cpu().numpy()
    for i in rng.choice(len(reqs), 40, replace=False):
        a, b, n = int(in_off[i]), int(out_off[i]), int(lengths[i])
        k = int(reqs["key_index"][i])
        want = oracle.ecb(raw_keys[k], int(bits[k]), xs[a:a + n], decrypt=bool(reqs["decrypt"][i]))
        assert np.array_equal(ys[b:b + n], want)
    assert gbaes.device_status() == 0


@pytest.mark.gpu
def test_server_batches_overlap_on_device(gbaes):
    rng = np.random.default_rng(9)
    bits = np.array([128, 256])
    keys = [gbaes.Key(rng.integers(0, 256, b // 8, dtype=np.uint8).tobytes()) for b in bits]
    reqs, x, y, *_ = device_requests(gbaes, rng, 3000, bits, 64 << 20, 4 << 20, 50_000.0)
    srv = gbaes.Server(keys, nstreams=4, max_batch_msgs=16)
    srv.replay(reqs)
    srv.replay_join()
    srv.drain(60.0)
    done = srv.poll_all()
    srv.close()
    assert (done["status"] == 0).all()
    batches = np.unique(np.stack([done["launch_s"], done["done_s"]], 1), axis=0)
    assert len(batches) > 10
    starts, ends = batches[:, 0], batches[:, 1]
    # some batch is launched while an earlier one is still running
    overlapping = sum(int(np.any((starts < e) & (starts > s))) for s, e in batches)
    assert overlapping > 0
