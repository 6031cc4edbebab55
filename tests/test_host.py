"""CPU-only checks of the CUDA library: it builds, loads, exports every symbol
that include/gbaes.h declares, and its host-side tables and key schedules match
the oracle and exhaustive GF(2^8) arithmetic.  No kernel runs here."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from tests.test_oracle import clmul_mod

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w\s\*]*?\b(aes_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol(gbaes):
    lib = ctypes.CDLL(gbaes.library_path())
    names = declared_functions()
    assert len(names) >= 14
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def rotl32(v, n):
    return ((v << n) | (v >> (32 - n))) & 0xFFFFFFFF if n else v


def test_tables_by_brute_force(gbaes):
    te0, td0, s, si = gbaes.host_tables()
    os_, osi = oracle.sbox()
    assert np.array_equal(s, os_) and np.array_equal(si, osi)
    for x in range(256):
        a = int(s[x])
        want = clmul_mod(a, 2) | (a << 8) | (a << 16) | (clmul_mod(a, 3) << 24)
        assert int(te0[x]) == want
        b = int(si[x])
        want = clmul_mod(b, 14) | (clmul_mod(b, 9) << 8) | (clmul_mod(b, 13) << 16) | (clmul_mod(b, 11) << 24)
        assert int(td0[x]) == want


def inv_mix_column(col):
    m = [[14, 11, 13, 9], [9, 14, 11, 13], [13, 9, 14, 11], [11, 13, 9, 14]]
    return [clmul_mod(col[0], m[r][0]) ^ clmul_mod(col[1], m[r][1]) ^ clmul_mod(col[2], m[r][2])
            ^ clmul_mod(col[3], m[r][3]) for r in range(4)]


@pytest.mark.parametrize("bits", (128, 192, 256))
def test_key_schedules_match_oracle(gbaes, bits):
    rng = np.random.default_rng(bits)
    for _ in range(20):
        key = rng.integers(0, 256, bits // 8, dtype=np.uint8).tobytes()
        enc, dec = gbaes.key_schedule(key, bits)
        w = oracle.key_expansion(key, bits)  # (Nr+1, 16) bytes
        assert enc.astype("<u4").tobytes() == w.tobytes()
        nr = oracle.nrounds(bits)
        for r in range(nr + 1):
            src = w[nr - r]
            want = src.tobytes() if r in (0, nr) else bytes(
                sum((inv_mix_column([int(v) for v in src[4 * j:4 * j + 4]]) for j in range(4)), []))
            assert dec[r].astype("<u4").tobytes() == want


def test_bad_key_size_is_an_error(gbaes):
    with pytest.raises(gbaes.AesError) as e:
        gbaes.Key(bytes(20), 160)
    assert e.value.code == -2


def test_no_device_means_error_not_fallback(gbaes):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lib = gbaes.load()
    k = gbaes.Key(bytes(16))
    buf = ctypes.create_string_buffer(64)
    rc = lib.aes_encrypt_ecb(k.handle, ctypes.cast(buf, ctypes.c_void_p), ctypes.cast(buf, ctypes.c_void_p), 4, None)
    assert rc in (-1, -3, -4)
    # zero blocks is a no-op success even without a device
    assert lib.aes_encrypt_ecb(k.handle, None, None, 0, None) == 0


def test_kernel_and_tuning_argument_checks(gbaes):
    lib = gbaes.load()
    assert lib.aes_set_kernel(7) == -1
    assert lib.aes_set_tuning(160, 0, 1024, 2) == -2
    assert lib.aes_set_tuning(128, 0, 1000, 2) == -1
    assert lib.aes_set_tuning(128, 0, 1024, 3) == -1
    assert lib.aes_set_tuning(128, 0, 1024, 2) == 0


def test_argument_checks_before_any_cuda_call(gbaes):
    """NULL pointers, byte-count overflow and bad flags are refused on the host
    (no device is touched; these run on a machine without a GPU)."""
    lib = gbaes.load()
    k = gbaes.Key(bytes(16))
    big = ctypes.c_void_p(1 << 20)
    assert lib.aes_encrypt_ecb(k.handle, None, big, 4, None) == -1  # NULL in
    assert lib.aes_decrypt_ecb(k.handle, big, None, 4, None) == -1  # NULL out
    assert lib.aes_encrypt_ecb(k.handle, big, big, (1 << 64) // 16 + 1, None) == -1  # bytes overflow size_t
    assert lib.aes_encrypt_ecb(None, big, big, 4, None) == -1  # no context
    assert lib.aes_ecb_ex(k.handle, 2, big, big, 4, 0, 0, 0, None) == -1  # decrypt flag not 0/1
    assert lib.aes_ecb_ex(k.handle, 0, big, big, 4, 9, 0, 0, None) == -1  # unknown kernel
    iv = (ctypes.c_uint8 * 16)()
    assert lib.aes_ctr_xcrypt(k.handle, iv, 5, 0, big, big, 4, None) == -1  # unknown counter kind
    assert lib.aes_ctr_xcrypt(k.handle, None, 0, 0, big, big, 4, None) == -1  # NULL iv
    assert lib.aes_cbc_decrypt(k.handle, None, big, big, 4, None) == -1
    assert lib.aes_ctx_bits(k.handle) == 128 and lib.aes_ctx_bits(None) == -1
    assert not lib.aes_pipeline_create_ex(0, 0, 2)  # unknown pipeline mode
    assert b"mode" in lib.aes_last_error()
    assert not lib.aes_pipeline_create_ex(24, 2, gbaes.PIPE_DIRECT)  # chunk not a multiple of 16
    msg = lib.aes_last_error()
    assert isinstance(msg, bytes) and len(msg) > 0
