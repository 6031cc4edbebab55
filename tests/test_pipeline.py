"""Host-buffer pipeline (chunks through device staging slots) against the oracle."""
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
