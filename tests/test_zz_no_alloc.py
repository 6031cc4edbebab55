"""The allocation-free batch entry point, called through the C ABI.

aes_ecb_batch_noalloc serves callers that cannot call cudaMalloc (their device
memory belongs to another runtime or allocator, or the call sits on a latency
path that must not allocate).  It must produce exactly what aes_ecb_batch and
the CPU oracle produce, call after call, although every call reuses one fixed
device array.  This file is named to be collected last."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1201_0398_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _setup(gbaes, seed, nmsg, nkeys, max_blocks):
    rng = np.random.default_rng(seed)
    bits = rng.choice([128, 192, 256], nkeys)
    raw = [rng.integers(0, 256, b // 8, dtype=np.uint8).tobytes() for b in bits]
    keys = [gbaes.Key(r) for r in raw]
    nblocks = np.exp(rng.uniform(0, np.log(max_blocks), nmsg)).astype(np.int64)
    off = np.concatenate([[0], np.cumsum(nblocks)[:-1]]) * 16
    kidx = rng.integers(0, nkeys, nmsg)
    dec = rng.integers(0, 2, nmsg)
    descs = gbaes.make_descs(off, off, nblocks, kidx, dec)
    data = rng.integers(0, 256, 16 * int(nblocks.sum()), dtype=np.uint8)
    want = np.empty_like(data)
    for o, n, k, d in zip(off, nblocks, kidx, dec):
        o, n = int(o), 16 * int(n)
        want[o:o + n] = oracle.ecb(raw[k], int(bits[k]), data[o:o + n], decrypt=bool(d))
    return keys, descs, torch.from_numpy(data).cuda(), want


def _call(lib, name, keys, descs, x, y, stream):
    ctxs = (ctypes.c_void_p * len(keys))(*[k.handle.value for k in keys])
    fn = getattr(lib, name)
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                   ctypes.c_size_t, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
    return fn(ctypes.c_void_p(descs.ctypes.data), descs.size, ctxs, len(keys), ctypes.c_void_p(x.data_ptr()),
              x.numel(), ctypes.c_void_p(y.data_ptr()), y.numel(), ctypes.c_void_p(stream.cuda_stream))


CASES = [(1, 700, 300, 40_000), (2, 2500, 2500, 3000)]


def test_noalloc_batch_matches_allocating_batch_and_oracle_twice(gbaes):
    lib = gbaes.load()
    stream = torch.cuda.current_stream()
    for call, case in enumerate(CASES):
        keys, descs, x, want = _setup(gbaes, *case)
        ref = torch.zeros_like(x)
        got = torch.full_like(x, 0xA5)
        assert _call(lib, "aes_ecb_batch", keys, descs, x, ref, stream) == 0
        assert _call(lib, "aes_ecb_batch_noalloc", keys, descs, x, got, stream) == 0, lib.aes_last_error()
        torch.cuda.synchronize()
        assert torch.equal(got, ref), f"call {call}"
        assert np.array_equal(got.cpu().numpy(), want), f"call {call}"
    assert gbaes.device_status() == 0


def test_noalloc_back_to_back_on_one_stream(gbaes):
    """Two different batches queued on one stream with no synchronisation in
    between: the second call's table upload is ordered after the first call's
    kernel on that stream, so both outputs are exact."""
    lib = gbaes.load()
    s = torch.cuda.Stream()
    a = _setup(gbaes, *CASES[0])
    b = _setup(gbaes, *CASES[1])
    outs = [torch.full_like(x, 0x5A) for _, _, x, _ in (a, b)]
    torch.cuda.synchronize()  # inputs and outputs are ready before the side stream reads them
    for (keys, descs, x, _), y in zip((a, b), outs):
        assert _call(lib, "aes_ecb_batch_noalloc", keys, descs, x, y, s) == 0, lib.aes_last_error()
    s.synchronize()
    for (_, _, _, want), y, name in zip((a, b), outs, "ab"):
        assert np.array_equal(y.cpu().numpy(), want), name
    assert gbaes.device_status() == 0


def test_noalloc_holds_the_ten_thousand_message_batch(gbaes):
    """The batched workload (10,000 messages of 16 B - 4 MiB, one key context
    each, key sizes 2:1:1, mixed directions) fits the fixed array and gives the
    allocating entry point's bytes."""
    w = workloads.batch_workload()
    keys = [gbaes.Key(k) for k in w.keys]
    off = np.concatenate([[0], np.cumsum(w.lengths)[:-1]])
    descs = gbaes.make_descs(off, off, w.lengths // 16, np.arange(len(keys)), w.decrypt)
    x = workloads.device_bytes(workloads.SEED_BATCH, w.total_bytes)
    lib = gbaes.load()
    stream = torch.cuda.current_stream()
    ref = torch.zeros_like(x)
    assert _call(lib, "aes_ecb_batch", keys, descs, x, ref, stream) == 0
    got = torch.full_like(x, 0xA5)
    assert _call(lib, "aes_ecb_batch_noalloc", keys, descs, x, got, stream) == 0, lib.aes_last_error()
    torch.cuda.synchronize()
    assert torch.equal(got, ref)
    del x, ref, got
    torch.cuda.empty_cache()


def test_noalloc_batch_rejects_tables_beyond_its_array(gbaes):
    lib = gbaes.load()
    stream = torch.cuda.current_stream()
    # 20,000 key contexts need 20,000 x 512 B of schedule slots: more than 8 MiB.
    keys, descs, x, _ = _setup(gbaes, 3, 4, 20_000, 8)
    y = torch.zeros_like(x)
    rc = _call(lib, "aes_ecb_batch_noalloc", keys, descs, x, y, stream)
    assert rc == -1
    lib.aes_last_error.restype = ctypes.c_char_p
    assert b"at most" in lib.aes_last_error()
