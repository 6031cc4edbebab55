"""Several servers behind one router (independent replicas; one per GPU in a
multi-GPU machine).  CPU: dry-run servers of different speeds, errors.  GPU: two
launch-per-batch servers sharing this GPU behind the by-device policy."""
import numpy as np
import pytest

import oracle


def keyset(g, n=2):
    return [g.Key(bytes([i + 1]) * 16) for i in range(n)]


def test_router_least_loaded_favours_the_faster_server(gbaes):
    fast = gbaes.Server(keyset(gbaes), dryrun=True, dryrun_batch_us=20, nstreams=1, max_batch_msgs=1)
    slow = gbaes.Server(keyset(gbaes), dryrun=True, dryrun_batch_us=2000, nstreams=1, max_batch_msgs=1)
    router = gbaes.Router([fast, slow])
    picks = []
    import time

    for i in range(600):
        picks.append(router.submit(i, i % 2, 1 << 20, 2 << 20, 4))
        if i % 20 == 19:
            time.sleep(0.002)  # arrivals spread over ~60 ms
    router.drain(30.0)
    done = router.poll_all()
    assert sorted(done["id"].tolist()) == list(range(600)) and (done["status"] == 0).all()
    picks = np.array(picks)
    assert set(picks.tolist()) <= {0, 1}
    assert (picks == 0).sum() > 2 * (picks == 1).sum()  # the faster server takes most requests
    router.close()
    fast.close()
    slow.close()


def test_router_by_device_without_device_memory_falls_back(gbaes):
    a = gbaes.Server(keyset(gbaes), dryrun=True)
    b = gbaes.Server(keyset(gbaes), dryrun=True)
    router = gbaes.Router([a, b], gbaes.ROUTE_BY_DEVICE)
    picks = [router.submit(i, 0, 1 << 20, 2 << 20, 4) for i in range(50)]
    router.drain(10.0)
    assert len(router.poll_all()) == 50 and set(picks) <= {0, 1}
    router.close()
    a.close()
    b.close()


def test_router_argument_errors(gbaes):
    a = gbaes.Server(keyset(gbaes), dryrun=True)
    with pytest.raises(gbaes.AesError):
        gbaes.Router([])
    with pytest.raises(gbaes.AesError):
        gbaes.Router([a, a])  # the same server twice
    with pytest.raises(gbaes.AesError):
        gbaes.Router([a], policy=7)
    router = gbaes.Router([a])
    with pytest.raises(gbaes.AesError):
        router.submit(0, 9, 1 << 20, 2 << 20, 4)  # the server's own check: key index out of range
    router.close()
    a.close()


# ------------------------------------------------------------------------- GPU

torch = pytest.importorskip("torch")


@pytest.mark.gpu
def test_router_two_servers_on_this_gpu(gbaes):
    rng = np.random.default_rng(51)
    raw = [rng.integers(0, 256, n, dtype=np.uint8).tobytes() for n in (16, 32)]
    keys = [gbaes.Key(k) for k in raw]
    n = 400
    lengths = (rng.integers(1, 257, n) * 16).astype(np.int64)
    off = np.concatenate([[0], np.cumsum(lengths)[:-1]])
    data = rng.integers(0, 256, int(lengths.sum()), dtype=np.uint8)
    x = torch.from_numpy(data).cuda()
    y = torch.zeros_like(x)
    torch.cuda.synchronize()
    servers = [gbaes.Server(keys, nstreams=2), gbaes.Server(keys, nstreams=2)]
    router = gbaes.Router(servers, gbaes.ROUTE_BY_DEVICE)
    kidx = rng.integers(0, 2, n)
    dec = rng.integers(0, 2, n)
    picks = [router.submit(i, int(kidx[i]), x.data_ptr() + int(off[i]), y.data_ptr() + int(off[i]),
                           int(lengths[i]) // 16, bool(dec[i])) for i in range(n)]
    router.drain(30.0)
    done = router.poll_all()
    router.close()
    for s in servers:
        s.close()
    assert sorted(done["id"].tolist()) == list(range(n)) and (done["status"] == 0).all()
    assert set(picks) == {0, 1}  # both servers on this device took work
    ys = y.cpu().numpy()
    for i in range(n):
        a, m = int(off[i]), int(lengths[i])
        want = oracle.ecb(raw[int(kidx[i])], 8 * len(raw[int(kidx[i])]), data[a:a + m], decrypt=bool(dec[i]))
        assert np.array_equal(ys[a:a + m], want), i
