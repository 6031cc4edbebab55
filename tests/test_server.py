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


def test_completions_oldest_first_across_chunks(gbaes):
    """The completion store (chunks of 16,384, made ahead and reused) hands out
    every completion once, oldest first, when polls of odd sizes interleave with
    new requests across chunk boundaries."""
    rng = np.random.default_rng(5)
    srv = gbaes.Server(keyset(gbaes), dryrun=True)
    buf = np.zeros(7777, gbaes.COMPLETION)
    total, parts = 0, []
    for burst in range(4):
        reqs = fake_requests(gbaes, 12_345, rng, max_blocks=4)  # all due at once
        reqs["id"] += total
        total += len(reqs)
        srv.replay(reqs)
        srv.replay_join()
        srv.drain(30.0)
        for _ in range(burst + 1):  # leaves some behind for the next burst
            parts.append(srv.poll(buf.size, out=buf).copy())
    parts.append(srv.poll_all())
    done = np.concatenate(parts)
    assert len(done) == total and (done["status"] == 0).all()
    assert np.array_equal(np.sort(done["id"]), np.arange(total))
    assert np.all(np.diff(done["done_s"]) >= 0)  # observation order
    assert srv.poll().size == 0
    srv.close()


@pytest.mark.parametrize("resident", [False, True])
def test_scheduler_page_faults_do_not_grow_with_completions(gbaes, resident):
    """A replay's completions land in memory made (and touched) before it
    starts: the scheduler and replay threads take a handful of page faults for
    100,000 requests, not one per page of completions (~1,000 pages)."""
    rng = np.random.default_rng(2)
    kw = dict(threads=64, blocks_per_thread=1) if resident else {}
    srv = gbaes.Server(keyset(gbaes), dryrun=True, resident=resident, **kw)
    reqs = fake_requests(gbaes, 100_000, rng, max_blocks=4, rate=400_000.0)
    srv.replay(reqs)
    srv.replay_join()
    srv.drain(30.0)
    d = srv.diag()
    assert len(srv.poll_all()) == 100_000
    assert d["sched_minflt"] < 200 and d["producer_minflt"] < 200, d
    assert srv.stats()["lost_completions"] == 0
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


def test_resident_dryrun_ring_wraps(gbaes):
    """Resident mode's ring protocol (the kernel's stand-in is a host thread):
    a ring of 64 tile records and 16 request slots per direction serves 3,000
    requests of 1-300 blocks (64-block tiles), so records and slots are reused
    many times; every request completes once, in budget."""
    rng = np.random.default_rng(11)
    srv = gbaes.Server(keyset(gbaes), budget_bytes=1 << 20, dryrun=True, resident=True, threads=64,
                       blocks_per_thread=1, ring_tiles=64, ring_items=16, max_batch_blocks=4096)
    reqs = fake_requests(gbaes, 3000, rng, max_blocks=300)
    for r in reqs:
        srv.submit(int(r["id"]), int(r["key_index"]), int(r["in_ptr"]), int(r["out_ptr"]), int(r["nblocks"]),
                   bool(r["decrypt"]))
    srv.drain(30.0)
    done = srv.poll_all()
    st = srv.stats()
    srv.close()
    assert sorted(done["id"].tolist()) == list(range(3000))
    assert (done["status"] == 0).all() and (done["batch_msgs"] == 1).all()
    assert st["completed"] == 3000 and st["failed"] == 0 and st["max_inflight_bytes"] <= 1 << 20
    assert st["batches"] >= 1  # kernel launches
    assert (done["done_s"] >= done["launch_s"]).all() and (done["launch_s"] >= done["arrival_s"]).all()


def test_resident_dryrun_idle_exit_and_relaunch(gbaes):
    """The kernel leaves after resident_idle_us without work; the next request
    relaunches it.  A short lifetime under steady load also ends kernels that
    are busy, and the scheduler relaunches them with nothing lost."""
    import time

    srv = gbaes.Server(keyset(gbaes), dryrun=True, resident=True, resident_idle_us=500)
    for i in range(10):
        srv.submit(i, i % 4, 1 << 20, 2 << 20, 8, bool(i & 1))
    srv.drain(10.0)
    time.sleep(0.03)  # well past the idle limit: the stand-in kernel has left
    for i in range(10, 20):
        srv.submit(i, i % 4, 1 << 20, 2 << 20, 8, bool(i & 1))
    srv.drain(10.0)
    assert len(srv.poll_all()) == 20
    assert srv.stats()["batches"] >= 2
    srv.close()

    rng = np.random.default_rng(12)
    srv = gbaes.Server(keyset(gbaes), dryrun=True, resident=True, resident_lifetime_ms=5)
    srv.replay(fake_requests(gbaes, 5000, rng, rate=50_000.0))  # ~0.1 s of arrivals
    srv.replay_join()
    srv.drain(10.0)
    done = srv.poll_all()
    assert len(done) == 5000 and (done["status"] == 0).all()
    assert srv.stats()["batches"] >= 5
    srv.close()


def test_resident_dryrun_recovery_after_kernel_bound(gbaes):
    """The scheduler restarts the kernel only after its own lifetime bound has
    ended it (restart at 1000% of a 3 ms lifetime), while requests keep
    arriving: tiles published after the kernel left are recovered from its
    abandoned tickets and re-published, and every request completes once."""
    rng = np.random.default_rng(13)
    srv = gbaes.Server(keyset(gbaes), dryrun=True, resident=True, resident_lifetime_ms=3, resident_restart_pct=1000)
    reqs = fake_requests(gbaes, 20_000, rng, rate=100_000.0)  # ~0.2 s: dozens of kernel lifetimes
    srv.replay(reqs)
    srv.replay_join()
    srv.drain(30.0)
    done = srv.poll_all()
    st = srv.stats()
    srv.close()
    assert sorted(done["id"].tolist()) == list(range(20_000)) and (done["status"] == 0).all()
    assert st["batches"] >= 20  # kernel launches
    assert st["recovered_tiles"] > 0  # the re-publishing path ran


def test_resident_config_errors(gbaes):
    with pytest.raises(gbaes.AesError):  # not a power of two
        gbaes.Server(keyset(gbaes), dryrun=True, resident=True, ring_tiles=100)
    with pytest.raises(gbaes.AesError):  # restart point above 1000% of the lifetime
        gbaes.Server(keyset(gbaes), dryrun=True, resident=True, resident_restart_pct=1001)
    with pytest.raises(gbaes.AesError):  # the largest request (2^22 blocks) needs 4,096 tiles of 512 x 2
        gbaes.Server(keyset(gbaes), dryrun=True, resident=True, ring_tiles=2048)
    srv = gbaes.Server(keyset(gbaes), dryrun=True, resident=True, ring_tiles=2048, max_batch_blocks=2048 * 1024)
    srv.close()


def test_resident_dryrun_fault_cancel_budget(gbaes):
    """An injected fault fails one request; requests still waiting for admission
    (the budget admits one at a time) can be cancelled; the rest complete."""
    srv = gbaes.Server(keyset(gbaes), budget_bytes=32 * 100, dryrun=True, resident=True, dryrun_batch_us=2000,
                       threads=64, blocks_per_thread=1)
    srv.inject_fault(3)
    for i in range(60):
        srv.submit(i, 0, 1 << 20, 2 << 20, 100)
    for i in range(40, 60):
        srv.cancel(i)
    srv.drain(30.0)
    done = srv.poll_all()
    st = dict(zip(done["id"].tolist(), done["status"].tolist()))
    assert len(st) == 60
    assert st[3] == -7 and sum(v == -7 for v in st.values()) == 1
    assert all(st[i] == 0 for i in range(10) if i != 3)
    assert any(st[i] == -8 for i in range(40, 60))
    assert srv.stats()["max_inflight_bytes"] <= 32 * 100
    srv.close()


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


@pytest.mark.gpu
@pytest.mark.parametrize("threads,bpt,ring_tiles,ring_items", [(512, 1, 0, 0), (256, 2, 256, 64), (512, 4, 64, 16)])
def test_resident_results_equal_alone_and_oracle(gbaes, threads, bpt, ring_tiles, ring_items):
    """Resident mode: 4,000 requests (64 B - 256 KiB, 64 keys of all sizes, both
    directions) at 100k req/s through one kernel that stays on the GPU; small
    rings in two cases so tile records and request slots are reused."""
    rng = np.random.default_rng(threads + bpt)
    nkeys = 64
    bits = rng.choice([128, 192, 256], nkeys)
    raw_keys = [rng.integers(0, 256, b // 8, dtype=np.uint8).tobytes() for b in bits]
    keys = [gbaes.Key(k) for k in raw_keys]
    reqs, x, y, in_off, out_off, lengths = device_requests(gbaes, rng, 4000, bits, 8 << 20, 256 << 10, 100_000.0)
    torch.cuda.synchronize()
    max_blocks = (ring_tiles or 1 << 16) * threads * bpt
    srv = gbaes.Server(keys, resident=True, threads=threads, blocks_per_thread=bpt, ring_tiles=ring_tiles,
                       ring_items=ring_items, max_batch_blocks=min(max_blocks, 1 << 22))
    srv.replay(reqs)
    srv.replay_join()
    srv.drain(60.0)
    done = srv.poll_all()
    st = srv.stats()
    srv.close()
    assert len(done) == len(reqs) and (done["status"] == 0).all()
    assert st["batches"] >= 1
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
def test_resident_sees_rewritten_inputs_and_in_place(gbaes):
    """One resident kernel (long idle limit) serves requests on buffers that
    change between them: an input rewritten from the host, and in-place
    requests on a buffer it wrote itself.  Each result must reflect the data at
    submission, not anything cached from earlier requests.  (While the kernel
    runs it holds every SM, so the test moves data with copies only.)"""
    rng = np.random.default_rng(21)
    key = bytes(range(32))
    k = gbaes.Key(key)
    n = 1 << 16  # 1 MiB
    x0 = rng.integers(0, 256, 16 * n, dtype=np.uint8)
    x1 = rng.integers(0, 256, 16 * n, dtype=np.uint8)
    x = torch.from_numpy(x0).cuda()
    y = torch.zeros_like(x)
    torch.cuda.synchronize()
    srv = gbaes.Server([k], resident=True, resident_idle_us=2_000_000)

    def run(i, src, dst, decrypt=False):
        srv.submit(i, 0, src.data_ptr(), dst.data_ptr(), src.numel() // 16, decrypt)
        srv.drain(10.0)
        return dst.cpu().numpy()  # a device-to-host copy

    first = run(0, x, y)
    x.copy_(torch.from_numpy(x1))  # rewrite the input (host-to-device copy)
    torch.cuda.current_stream().synchronize()  # (a device-wide sync would wait for the resident kernel)
    second = run(1, x, y)
    third = run(2, y, y)  # in place on the buffer the kernel just wrote
    fourth = run(3, y, y, decrypt=True)
    done = srv.poll_all()
    launches = srv.stats()["batches"]
    srv.close()
    assert (done["status"] == 0).all() and len(done) == 4
    assert launches == 1  # one kernel served all four
    assert np.array_equal(first, oracle.ecb(key, 256, x0))
    c = oracle.ecb(key, 256, x1)
    assert np.array_equal(second, c)
    assert np.array_equal(third, oracle.ecb(key, 256, c))
    assert np.array_equal(fourth, c)


@pytest.mark.gpu
def test_resident_kernel_leaves_when_idle_and_is_relaunched(gbaes):
    import time

    rng = np.random.default_rng(5)
    key = rng.integers(0, 256, 16, dtype=np.uint8).tobytes()
    k = gbaes.Key(key)
    x = torch.from_numpy(rng.integers(0, 256, 1 << 20, dtype=np.uint8)).cuda()
    y = torch.zeros_like(x)
    torch.cuda.synchronize()
    srv = gbaes.Server([k], resident=True, resident_idle_us=300)
    srv.submit(0, 0, x.data_ptr(), y.data_ptr(), 1 << 15)
    srv.drain(10.0)
    time.sleep(0.05)  # past the idle limit: the kernel has left
    srv.submit(1, 0, x.data_ptr() + (1 << 19), y.data_ptr() + (1 << 19), 1 << 15)
    srv.drain(10.0)
    done = srv.poll_all()
    launches = srv.stats()["batches"]
    srv.close()
    assert len(done) == 2 and (done["status"] == 0).all()
    assert launches == 2
    assert np.array_equal(y.cpu().numpy(), oracle.ecb(key, 128, x.cpu().numpy()))
    assert gbaes.device_status() == 0


def test_resident_dryrun_ring_sized_requests(gbaes):
    """Requests that need the whole tile ring (64 tiles of 64 blocks) alternate
    with zero-length requests (which complete at once without touching the
    ring) and single-block ones; all complete, in budget."""
    srv = gbaes.Server(keyset(gbaes), dryrun=True, resident=True, threads=64, blocks_per_thread=1, ring_tiles=64,
                       ring_items=4, max_batch_blocks=64 * 64)
    ids = []
    for i in range(60):
        n = (64 * 64, 0, 1)[i % 3]
        srv.submit(i, i % 4, 1 << 20, 2 << 20, n, bool(i & 1))
        ids.append(i)
    srv.drain(30.0)
    done = srv.poll_all()
    srv.close()
    assert sorted(done["id"].tolist()) == ids and (done["status"] == 0).all()


@pytest.mark.gpu
def test_resident_ring_sized_zero_length_and_in_place(gbaes):
    """On the GPU: requests that fill the whole (small) tile ring, zero-length
    requests, and in-place requests of both directions on one buffer, through
    one server; every output equals the oracle's."""
    rng = np.random.default_rng(31)
    key = rng.integers(0, 256, 24, dtype=np.uint8).tobytes()
    k = gbaes.Key(key)
    tile = 64 * 2  # 64 threads x 2 blocks
    big = 16 * tile  # blocks: the whole ring of 16 tiles
    data = rng.integers(0, 256, 16 * big * 4, dtype=np.uint8)
    x = torch.from_numpy(data).cuda()
    y = torch.zeros_like(x)
    torch.cuda.synchronize()
    srv = gbaes.Server([k], resident=True, threads=64, blocks_per_thread=2, ring_tiles=16, ring_items=4,
                       max_batch_blocks=big)
    for i in range(4):  # four ring-sized requests, x -> y
        off = 16 * big * i
        srv.submit(i, 0, x.data_ptr() + off, y.data_ptr() + off, big)
        srv.submit(100 + i, 0, x.data_ptr(), y.data_ptr(), 0)  # zero-length
    srv.drain(30.0)
    for i in range(4):  # in place on y: decrypt halves 0 and 2, encrypt halves 1 and 3 again
        off = 16 * big * i
        srv.submit(10 + i, 0, y.data_ptr() + off, y.data_ptr() + off, big, bool(i % 2 == 0))
    srv.drain(30.0)
    done = srv.poll_all()
    srv.close()
    assert len(done) == 12 and (done["status"] == 0).all()
    got = y.cpu().numpy().reshape(4, -1)
    parts = data.reshape(4, -1)
    for i in range(4):
        c = oracle.ecb(key, 192, parts[i])
        want = parts[i] if i % 2 == 0 else oracle.ecb(key, 192, c)
        assert np.array_equal(got[i], want), i
    assert gbaes.device_status() == 0


@pytest.mark.gpu
def test_resident_recovery_after_kernel_bound(gbaes):
    """On the GPU: the kernel's own 20 ms lifetime bound ends it while requests
    keep arriving (the scheduler would restart it only at 1000%); the tickets
    its CTAs abandoned are recovered and re-published.  Every output equals the
    single-message kernel's and the oracle's on a sample."""
    rng = np.random.default_rng(41)
    nkeys = 16
    bits = rng.choice([128, 192, 256], nkeys)
    raw_keys = [rng.integers(0, 256, b // 8, dtype=np.uint8).tobytes() for b in bits]
    keys = [gbaes.Key(k) for k in raw_keys]
    reqs, x, y, in_off, out_off, lengths = device_requests(gbaes, rng, 6000, bits, 8 << 20, 64 << 10, 30_000.0)
    torch.cuda.synchronize()
    srv = gbaes.Server(keys, resident=True, resident_lifetime_ms=20, resident_restart_pct=1000)
    srv.replay(reqs)  # ~0.2 s of arrivals: about ten kernel lifetimes
    srv.replay_join()
    srv.drain(60.0)
    done = srv.poll_all()
    st = srv.stats()
    srv.close()
    assert len(done) == len(reqs) and (done["status"] == 0).all()
    assert st["batches"] >= 5
    print("kernel launches", st["batches"], "recovered tiles", st["recovered_tiles"])
    alone = torch.zeros_like(y)
    for i in range(len(reqs)):
        a, b, n = int(in_off[i]), int(out_off[i]), int(lengths[i])
        gbaes.ecb_ex(keys[int(reqs["key_index"][i])], x[a:a + n], alone[b:b + n], decrypt=bool(reqs["decrypt"][i]))
    torch.cuda.synchronize()
    assert torch.equal(alone, y)
    xs, ys = x.cpu().numpy(), y.cpu().numpy()
    for i in rng.choice(len(reqs), 20, replace=False):
        a, b, n = int(in_off[i]), int(out_off[i]), int(lengths[i])
        k = int(reqs["key_index"][i])
        assert np.array_equal(ys[b:b + n], oracle.ecb(raw_keys[k], int(bits[k]), xs[a:a + n], decrypt=bool(reqs["decrypt"][i])))
    assert gbaes.device_status() == 0


@pytest.mark.parametrize("resident", (False, True))
def test_dryrun_thread_diagnostics_and_pinning(gbaes, resident):
    """Host-thread diagnostics after a replay (both modes): scheduler passes
    and windows, lock waits, replay lateness; with pin_threads the scheduler
    and replay threads sit on distinct CPUs of the process's affinity set."""
    import os

    allowed = sorted(os.sched_getaffinity(0))
    srv = gbaes.Server(keyset(gbaes), dryrun=True, resident=resident, threads=64, blocks_per_thread=1,
                       pin_threads=True)
    rng = np.random.default_rng(11)
    reqs = fake_requests(gbaes, 3000, rng, max_blocks=32, rate=100_000.0)
    srv.replay(reqs)
    srv.replay_join()
    srv.drain(30.0)
    assert len(srv.poll_all()) == 3000
    d = srv.diag()
    srv.close()
    assert d["sched_passes"] > 0
    assert d["sched_worst_window_ns"] > 0
    assert d["sched_worst_window_cpu_ns"] <= d["sched_worst_window_ns"] + 10_000_000  # (CPU clock granularity)
    assert d["producer_late_max_ns"] > 0 and d["producer_check_max_ns"] > 0
    assert d["producer_late_at_ns"] <= 2e9 and len(d["lock_wait_max_ns"]) == 3
    assert max(d["sched_phase_max_ns"]) > 0 and d["inbox_hold_max_ns"][1] > 0
    assert d["sched_cpu"] == allowed[-1]
    assert d["producer_cpu"] == (allowed[-2] if len(allowed) > 1 else -1)


def test_dryrun_unpinned_threads_report_no_cpu(gbaes):
    srv = gbaes.Server(keyset(gbaes), dryrun=True)
    srv.submit(1, 0, 1 << 20, 2 << 20, 4)
    srv.drain(10.0)
    d = srv.diag()
    srv.close()
    assert d["sched_cpu"] == -1 and d["producer_cpu"] == -1


@pytest.mark.parametrize("resident", [False, True])
def test_concurrent_submitters_and_replay(gbaes, resident):
    """Four client threads submit while a replay runs and completions are polled:
    the server's shared queues and its memory pool take allocations from several
    threads at once; every request completes exactly once."""
    import threading

    kw = dict(threads=64, blocks_per_thread=1) if resident else {}
    srv = gbaes.Server(keyset(gbaes), dryrun=True, resident=resident, **kw)
    rng = np.random.default_rng(9)
    reqs = fake_requests(gbaes, 20_000, rng, max_blocks=4, rate=200_000.0)
    reqs["id"] += 1_000_000
    srv.replay(reqs)

    def client(c):
        for i in range(3000):
            srv.submit(c * 10_000 + i, i % 4, 1 << 20, 2 << 20, 1 + i % 3, decrypt=bool(i & 1))

    ths = [threading.Thread(target=client, args=(c,)) for c in range(4)]
    for t in ths:
        t.start()
    got = []
    buf = np.zeros(4096, gbaes.COMPLETION)
    while any(t.is_alive() for t in ths):
        got.append(srv.poll(buf.size, out=buf).copy())
    for t in ths:
        t.join()
    srv.replay_join()
    srv.drain(30.0)
    got.append(srv.poll_all())
    done = np.concatenate(got)
    want = np.concatenate([np.arange(c * 10_000, c * 10_000 + 3000) for c in range(4)] + [reqs["id"]])
    assert (done["status"] == 0).all()
    assert np.array_equal(np.sort(done["id"]), np.sort(want))
    srv.close()


def test_server_threads_are_named(gbaes):
    """The scheduler and replay threads carry names (gbaes-sched, gbaes-replay) for ps, top and
    /proc/<pid>/task, where a watchdog finds them."""
    import os
    import time

    task = "/proc/self/task"
    if not os.path.isdir(task):
        pytest.skip("no /proc task list")

    def names():
        out = set()
        for t in os.listdir(task):
            try:
                with open(f"{task}/{t}/comm") as f:
                    out.add(f.read().strip())
            except OSError:
                pass
        return out

    srv = gbaes.Server(keyset(gbaes), dryrun=True)
    rng = np.random.default_rng(8)
    srv.replay(fake_requests(gbaes, 2000, rng, rate=10_000.0))  # ~0.2 s of arrivals
    time.sleep(0.05)
    seen = names()
    srv.replay_join()
    srv.drain(10.0)
    srv.close()
    assert {"gbaes-sched", "gbaes-replay"} <= seen, seen


@pytest.mark.gpu
@pytest.mark.parametrize("resident", (False, True))
def test_server_with_payloads_in_page_locked_host_memory(gbaes, resident):
    """Requests whose inputs and outputs live in page-locked host memory (the
    kernels read and write them over the host link): both server modes, every
    request against the oracle."""
    rng = np.random.default_rng(77 + int(resident))
    nkeys = 16
    bits = rng.choice([128, 192, 256], nkeys)
    raw_keys = [rng.integers(0, 256, b // 8, dtype=np.uint8).tobytes() for b in bits]
    keys = [gbaes.Key(k) for k in raw_keys]
    n = 2000
    lengths = np.maximum((np.exp(rng.uniform(np.log(64), np.log(256 << 10), n)) // 16 * 16).astype(np.int64), 16)
    pool = 8 << 20
    x = torch.from_numpy(rng.integers(0, 256, pool, dtype=np.uint8)).pin_memory()
    y = torch.zeros(int(lengths.sum()), dtype=torch.uint8).pin_memory()
    in_off = (rng.integers(0, (pool - lengths) // 16 + 1) * 16).astype(np.int64)
    out_off = np.concatenate([[0], np.cumsum(lengths)[:-1]])
    reqs = np.zeros(n, gbaes.REQUEST)
    reqs["id"] = np.arange(n)
    reqs["in_ptr"] = x.data_ptr() + in_off
    reqs["out_ptr"] = y.data_ptr() + out_off
    reqs["nblocks"] = lengths // 16
    reqs["key_index"] = rng.integers(0, nkeys, n)
    reqs["decrypt"] = rng.integers(0, 2, n)
    reqs["arrival_s"] = np.cumsum(rng.exponential(1.0 / 50_000.0, n))
    srv = gbaes.Server(keys, resident=resident, threads=512, blocks_per_thread=2)
    srv.replay(reqs)
    srv.replay_join()
    srv.drain(60.0)
    done = srv.poll_all()
    srv.close()
    assert len(done) == n and (done["status"] == 0).all()
    xs, ys = x.numpy(), y.numpy()
    for i in range(n):
        a, b, m = int(in_off[i]), int(out_off[i]), int(lengths[i])
        k = int(reqs["key_index"][i])
        want = oracle.ecb(raw_keys[k], int(bits[k]), xs[a:a + m], decrypt=bool(reqs["decrypt"][i]), nthreads=1)
        assert np.array_equal(ys[b:b + m], want), i
    assert gbaes.device_status() == 0
