"""Batched multi-key launch: host tiling (CPU) and GPU parity.

Every message of a batch must come out exactly as the CPU oracle computes it
and exactly as the single-message kernel computes it alone (AES output is
unique, so "the same alone and in the mix" is bit equality)."""
import numpy as np
import pytest

import oracle
from paper_1201_0398_gb300 import workloads

NR = {128: 10, 192: 12, 256: 14}


def random_batch(rng, n, nkeys, max_blocks, zero_frac=0.05):
    bits = rng.choice([128, 192, 256], nkeys)
    keys = [rng.integers(0, 256, b // 8, dtype=np.uint8).tobytes() for b in bits]
    nblocks = np.exp(rng.uniform(0, np.log(max_blocks), n)).astype(np.int64)
    nblocks[rng.random(n) < zero_frac] = 0
    key_index = rng.integers(0, nkeys, n)
    decrypt = rng.integers(0, 2, n)
    return bits, keys, nblocks, key_index, decrypt


def model_tiles(nblocks, key_index, decrypt, key_bits, tb):
    """Plain model of the plan's tiling: groups (dir, Nr) in order enc128..dec256."""
    out = []
    for d in (0, 1):
        for nr in (10, 12, 14):
            msgs = [i for i in range(len(nblocks)) if nblocks[i] > 0 and decrypt[i] == d
                    and NR[int(key_bits[key_index[i]])] == nr]
            starts, blk = [], 0
            for i in msgs:
                starts.append(blk)
                blk += int(nblocks[i])
            ntiles = -(-blk // tb)
            for t in range(ntiles):
                first = t * tb
                j = max(k for k in range(len(msgs)) if starts[k] <= first)
                out.append(msgs[j])
    return np.array(out, np.uint32)


def test_batch_tiles_match_model(gbaes):
    rng = np.random.default_rng(1)
    for tb in (1, 7, 64, 2048):
        bits, keys, nblocks, key_index, decrypt = random_batch(rng, 200, 13, 3000)
        ks = [gbaes.Key(k) for k in keys]
        off = np.concatenate([[0], np.cumsum(nblocks)[:-1]]) * 16
        d = gbaes.make_descs(off, off, nblocks, key_index, decrypt)
        got = gbaes.batch_tiles(d, ks, tb)
        assert np.array_equal(got, model_tiles(nblocks, key_index, decrypt, bits, tb))


def test_batch_plan_shape_errors(gbaes):
    ks = [gbaes.Key(bytes(16))]
    d = gbaes.make_descs([0], [0], [4], [0], [0])
    for threads, bpt, text in ((1024, 8, "512"), (512, 3, "1, 2, 4 or 8"), (48, 2, "multiple of 32")):
        with pytest.raises(gbaes.AesError) as e:
            gbaes.BatchPlan(d, ks, threads, bpt)
        assert text in str(e.value), (threads, bpt, str(e.value))


def test_batch_descriptor_errors(gbaes):
    ks = [gbaes.Key(bytes(16))]
    bad_key = gbaes.make_descs([0], [0], [4], [1], [0])
    with pytest.raises(gbaes.AesError):
        gbaes.batch_tiles(bad_key, ks, 64)
    bad_dir = gbaes.make_descs([0], [0], [4], [0], [2])
    with pytest.raises(gbaes.AesError):
        gbaes.batch_tiles(bad_dir, ks, 64)
    bad_align = gbaes.make_descs([8], [0], [4], [0], [0])
    with pytest.raises(gbaes.AesError) as e:
        gbaes.batch_tiles(bad_align, ks, 64)
    assert e.value.name == "AES_ERR_ALIGN"
    overflow = gbaes.make_descs([(1 << 64) - 16], [0], [4], [0], [0])
    with pytest.raises(gbaes.AesError):
        gbaes.batch_tiles(overflow, ks, 64)
    assert gbaes.batch_tiles(gbaes.make_descs([], [], [], [], []), ks, 64).size == 0


# ------------------------------------------------------------------------- GPU

torch = pytest.importorskip("torch")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def oracle_batch(data, keys, bits, nblocks, key_index, decrypt, in_off, out_off, out_size):
    out = np.zeros(out_size, np.uint8)
    for i in range(len(nblocks)):
        n = int(nblocks[i])
        if n == 0:
            continue
        k = int(key_index[i])
        src = data[int(in_off[i]):int(in_off[i]) + 16 * n]
        out[int(out_off[i]):int(out_off[i]) + 16 * n] = oracle.ecb(keys[k], int(bits[k]), src,
                                                                   decrypt=bool(decrypt[i]), nthreads=1 if n < 4096 else None)
    return out


@pytest.mark.gpu
@pytest.mark.parametrize("threads,bpt", [(1024, 2), (1024, 1), (1024, 4), (512, 2), (256, 4), (64, 1), (512, 8),
                                         (64, 8)])
def test_batch_vs_oracle_and_single_kernel(gbaes, threads, bpt):
    rng = np.random.default_rng(threads + bpt)
    bits, keys, nblocks, key_index, decrypt = random_batch(rng, 400, 37, 5000)
    ks = [gbaes.Key(k) for k in keys]
    total = int(nblocks.sum())
    in_off = np.concatenate([[0], np.cumsum(nblocks)[:-1]]) * 16
    perm = rng.permutation(len(nblocks))  # outputs laid out in a different order
    out_off = np.zeros_like(in_off)
    out_off[perm] = np.concatenate([[0], np.cumsum(nblocks[perm])[:-1]]) * 16
    data = rng.integers(0, 256, 16 * total + 16, dtype=np.uint8)
    x = torch.from_numpy(data).cuda()
    y = torch.zeros_like(x)
    plan = gbaes.BatchPlan(gbaes.make_descs(in_off, out_off, nblocks, key_index, decrypt), ks, threads, bpt)
    assert plan.info()["total_blocks"] == total
    plan.launch(x, y)
    got = host(y)
    want = oracle_batch(data, keys, bits, nblocks, key_index, decrypt, in_off, out_off, data.size)
    assert np.array_equal(got, want)
    # each message alone through the single-message kernel
    alone = torch.zeros_like(x)
    for i in range(len(nblocks)):
        n = int(nblocks[i])
        if n:
            a, b = int(in_off[i]), int(out_off[i])
            gbaes.ecb_ex(ks[int(key_index[i])], x[a:a + 16 * n], alone[b:b + 16 * n], decrypt=bool(decrypt[i]))
    assert torch.equal(alone, y)
    assert gbaes.device_status() == 0


@pytest.mark.gpu
def test_batch_graph_rebase_one_shot_and_in_place(gbaes):
    rng = np.random.default_rng(42)
    bits, keys, nblocks, key_index, decrypt = random_batch(rng, 150, 9, 20000)
    ks = [gbaes.Key(k) for k in keys]
    total = int(nblocks.sum())
    off = np.concatenate([[0], np.cumsum(nblocks)[:-1]]) * 16
    d = gbaes.make_descs(off, off, nblocks, key_index, decrypt)
    data = rng.integers(0, 256, 16 * total, dtype=np.uint8)
    want = oracle_batch(data, keys, bits, nblocks, key_index, decrypt, off, off, data.size)
    plan = gbaes.BatchPlan(d, ks)
    x1 = torch.from_numpy(data).cuda()
    x2 = x1.clone()
    y1, y2 = torch.zeros_like(x1), torch.zeros_like(x1)
    plan.launch(x1, y1, graph=True)   # capture
    plan.launch(x2, y2, graph=True)   # replay with new bases
    plan.launch(x1, y1, graph=True)   # and back
    assert np.array_equal(host(y1), want) and np.array_equal(host(y2), want)
    y3 = torch.zeros_like(x1)
    gbaes.ecb_batch(d, ks, x1, y3)
    assert np.array_equal(host(y3), want)
    plan.launch(x2, x2)  # in place: every message reads and writes its own range
    assert np.array_equal(host(x2), want)
    with pytest.raises(gbaes.AesError):  # buffers smaller than the messages need
        plan.launch(x1[:-16], y1)


@pytest.mark.gpu
@pytest.mark.parametrize("shape", __import__("paper_1201_0398_gb300.autotune", fromlist=["x"]).BATCH_CANDIDATES)
def test_batch_full_workload_10k_messages(gbaes, shape):
    """10,000 messages, log-uniform 16 B - 4 MiB, keys 2:1:1 over 128/192/256,
    mixed directions, one launch, in every plan shape the autotuner may pick for
    the bench; sampled messages against the oracle and every message against the
    single-message kernel."""
    w = workloads.batch_workload()
    ks = [gbaes.Key(k) for k in w.keys]
    nblocks = w.lengths // 16
    off = np.concatenate([[0], np.cumsum(w.lengths)[:-1]])
    d = gbaes.make_descs(off, off, nblocks, np.arange(len(ks)), w.decrypt)
    x = workloads.device_bytes(workloads.SEED_BATCH, w.total_bytes)
    y = torch.empty_like(x)
    plan = gbaes.BatchPlan(d, ks, *shape)
    plan.launch(x, y)
    alone = torch.empty_like(x)
    for i in range(len(ks)):
        a, n = int(off[i]), int(w.lengths[i])
        gbaes.ecb_ex(ks[i], x[a:a + n], alone[a:a + n], decrypt=bool(w.decrypt[i]))
    assert torch.equal(alone, y)
    rng = np.random.default_rng(shape[0] + shape[1])
    for i in rng.choice(len(ks), 30, replace=False):
        a, n = int(off[i]), int(w.lengths[i])
        take = min(n, 1 << 16)
        src = host(x[a:a + take])
        got = host(y[a:a + take])
        assert np.array_equal(got, oracle.ecb(w.keys[i], int(w.bits[i]), src, decrypt=bool(w.decrypt[i])))
    assert gbaes.device_status() == 0


@pytest.mark.gpu
def test_one_shot_batch_refuses_stream_capture(gbaes):
    """aes_ecb_batch uploads its tables from a host copy that is freed when the
    call returns, so it refuses a stream that is being captured into a graph
    (plans have their own graph path)."""
    ks = [gbaes.Key(bytes(16))]
    d = gbaes.make_descs([0], [0], [4], [0], [0])
    x = torch.zeros(64, dtype=torch.uint8, device="cuda")
    y = torch.zeros_like(x)
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=s, capture_error_mode="relaxed"):
        with pytest.raises(gbaes.AesError) as e:
            gbaes.ecb_batch(d, ks, x, y)
        y.add_(1)  # the graph captures this alone
    assert e.value.name == "AES_ERR_STATE"
    assert int(y.sum()) == 0  # captured, not run
