"""Host-buffer pipeline against the oracle: staged (chunks through device
staging slots and copy engines) and direct (the kernel on the host buffers)."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def pinned(a: np.ndarray):
    t = torch.empty(a.size, dtype=torch.uint8, pin_memory=True)
    t.numpy()[:] = a
    return t


@pytest.mark.parametrize("chunk,depth", [(1 << 20, 1), (1 << 20, 2), (3 << 20, 3), (16, 4), (64 << 20, 4)])
def test_pipeline_vs_oracle(gbaes, chunk, depth):
    rng = np.random.default_rng(chunk + depth)
    n = (5 << 20) // 16 + 7 if chunk > 16 else 1000  # several chunks and a ragged last one
    for bits in (128, 192, 256):
        key = rng.integers(0, 256, bits // 8, dtype=np.uint8).tobytes()
        k = gbaes.Key(key)
        data = rng.integers(0, 256, 16 * n, dtype=np.uint8)
        pipe = gbaes.Pipeline(chunk, depth)
        for decrypt in (False, True):
            hin = pinned(data)
            hout = pipe.ecb(k, hin, decrypt=decrypt)
            torch.cuda.synchronize()
            assert np.array_equal(hout.numpy(), oracle.ecb(key, bits, data, decrypt=decrypt))


@pytest.mark.parametrize("n", [1, 7, 2048 * 152 + 5, (5 << 20) // 16 + 7])
def test_direct_pipeline_vs_oracle(gbaes, n):
    """Direct mode at sizes below one tile, with a ragged last tile, and over several grid passes."""
    rng = np.random.default_rng(n)
    for bits in (128, 192, 256):
        key = rng.integers(0, 256, bits // 8, dtype=np.uint8).tobytes()
        k = gbaes.Key(key)
        data = rng.integers(0, 256, 16 * n, dtype=np.uint8)
        pipe = gbaes.Pipeline(mode=gbaes.PIPE_DIRECT)
        for decrypt in (False, True):
            hout = pipe.ecb(k, pinned(data), decrypt=decrypt)
            torch.cuda.synchronize()
            assert np.array_equal(hout.numpy(), oracle.ecb(key, bits, data, decrypt=decrypt))
        h = pinned(data)  # in place
        pipe.ecb(k, h, h)
        torch.cuda.synchronize()
        assert np.array_equal(h.numpy(), oracle.ecb(key, bits, data))


def test_pipeline_in_place_and_errors(gbaes):
    rng = np.random.default_rng(3)
    key = rng.integers(0, 256, 16, dtype=np.uint8).tobytes()
    k = gbaes.Key(key)
    data = rng.integers(0, 256, 16 * 300_001, dtype=np.uint8)
    h = pinned(data)
    pipe = gbaes.Pipeline(1 << 20, 3)
    pipe.ecb(k, h, h)
    torch.cuda.synchronize()
    assert np.array_equal(h.numpy(), oracle.ecb(key, 128, data))
    pipe.ecb(k, h, h, decrypt=True)
    torch.cuda.synchronize()
    assert np.array_equal(h.numpy(), data)
    pageable = torch.from_numpy(data.copy())  # not page-locked: refused on the host
    with pytest.raises(gbaes.AesError):
        pipe.ecb(k, pageable, h)
    with pytest.raises(gbaes.AesError):
        gbaes.Pipeline(24, 2)  # chunk not a multiple of 16
    direct = gbaes.Pipeline(mode=gbaes.PIPE_DIRECT)
    with pytest.raises(gbaes.AesError):
        direct.ecb(k, pageable, h)


def test_zero_copy_on_pinned_memory(gbaes):
    """The device-memory calls also accept page-locked host memory (the GPU reads
    and writes it over the host link)."""
    rng = np.random.default_rng(4)
    key = rng.integers(0, 256, 32, dtype=np.uint8).tobytes()
    k = gbaes.Key(key)
    data = rng.integers(0, 256, 16 * 100_000, dtype=np.uint8)
    hin, hout = pinned(data), pinned(np.zeros_like(data))
    gbaes.encrypt_ecb(k, hin, hout)
    torch.cuda.synchronize()
    assert np.array_equal(hout.numpy(), oracle.ecb(key, 256, data))
