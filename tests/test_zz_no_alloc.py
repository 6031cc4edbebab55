"""The allocation-free batch entry point, called through the C ABI.

aes_ecb_batch_noalloc serves callers that cannot call cudaMalloc (their device
memory belongs to another runtime or allocator, or the call sits on a latency
path that must not allocate).  It must produce exactly what aes_ecb_batch
produces, call after call, although both calls reuse one fixed device array.
This file is named to be collected last."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _setup(gbaes, seed, nmsg, nkeys, max_blocks):
    rng = np.random.default_rng(seed)
    bits = rng.choice([128, 192, 256], nkeys)
    keys = [gbaes.Key(rng.integers(0, 256, b // 8, dtype=np.uint8).tobytes()) for b in bits]
    nblocks = np.exp(rng.uniform(0, np.log(max_blocks), nmsg)).astype(np.int64)
    off = np.concatenate([[0], np.cumsum(nblocks)[:-1]]) * 16
    descs = gbaes.make_descs(off, off, nblocks, rng.integers(0, nkeys, nmsg), rng.integers(0, 2, nmsg))
    x = torch.from_numpy(rng.integers(0, 256, 16 * int(nblocks.sum()), dtype=np.uint8)).cuda()
    return keys, descs, x


def _call(lib, name, keys, descs, x, y, stream):
    ctxs = (ctypes.c_void_p * len(keys))(*[k.handle.value for k in keys])
    fn = getattr(lib, name)
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                   ctypes.c_size_t, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
    return fn(ctypes.c_void_p(descs.ctypes.data), descs.size, ctxs, len(keys), ctypes.c_void_p(x.data_ptr()),
              x.numel(), ctypes.c_void_p(y.data_ptr()), y.numel(), ctypes.c_void_p(stream.cuda_stream))


def test_noalloc_batch_matches_allocating_batch_twice(gbaes):
    lib = gbaes.load()
    stream = torch.cuda.current_stream()
    for call, (seed, nmsg, nkeys, max_blocks) in enumerate([(1, 700, 300, 40_000), (2, 2500, 2500, 3000)]):
        keys, descs, x = _setup(gbaes, seed, nmsg, nkeys, max_blocks)
        want = torch.zeros_like(x)
        got = torch.full_like(x, 0xA5)
        assert _call(lib, "aes_ecb_batch", keys, descs, x, want, stream) == 0
        assert _call(lib, "aes_ecb_batch_noalloc", keys, descs, x, got, stream) == 0, lib.aes_last_error()
        torch.cuda.synchronize()
        assert torch.equal(got, want), f"call {call}"
    assert gbaes.device_status() == 0


def test_noalloc_batch_rejects_tables_beyond_its_array(gbaes):
    lib = gbaes.load()
    stream = torch.cuda.current_stream()
    # 20,000 key contexts need 20,000 x 512 B of schedule slots: more than 8 MiB.
    keys, descs, x = _setup(gbaes, 3, 4, 20_000, 8)
    y = torch.zeros_like(x)
    rc = _call(lib, "aes_ecb_batch_noalloc", keys, descs, x, y, stream)
    assert rc == -1
    lib.aes_last_error.restype = ctypes.c_char_p
    assert b"at most" in lib.aes_last_error()
