"""Pins for the CPU oracle (no GPU).

Each test checks the oracle against something other than itself: exhaustive
GF(2^8) arithmetic written a different way, permutation/design properties of the
S-box, the installed ``cryptography`` package and the ``openssl`` command line as
black-box known-answer sources (AES per FIPS-197, which Section 2.1 of the paper
defers to), and plain integer arithmetic for CTR counters.  The planted-mistake
test shows that a dropped term, a wrong index or a missing step in the oracle is
caught by these pins.
"""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import oracle

ciphers = pytest.importorskip("cryptography.hazmat.primitives.ciphers")
Cipher, algorithms, modes = ciphers.Cipher, ciphers.algorithms, ciphers.modes

BITS = (128, 192, 256)


def clmul_mod(a: int, b: int) -> int:
    """GF(2^8) product as polynomial product then long division by 0x11B."""
    p = 0
    for i in range(8):
        if (b >> i) & 1:
            p ^= a << i
    for deg in range(14, 7, -1):
        if (p >> deg) & 1:
            p ^= 0x11B << (deg - 8)
    return p


def lib_ecb(key: bytes, data: bytes, decrypt=False) -> bytes:
    c = Cipher(algorithms.AES(key), modes.ECB())
    op = c.decryptor() if decrypt else c.encryptor()
    return op.update(data) + op.finalize()


def test_gf_mul_exhaustive():
    # Every one of the 65,536 products, against shift-and-reduce long division.
    for a in range(256):
        for b in range(0, 256, 1):
            assert oracle.gf_mul(a, b) == clmul_mod(a, b)


def test_sbox_independent_formulation():
    # S[x] = affine(x^254): exponentiation instead of the oracle's search, and the
    # affine map as rotations b ^ rotl1 ^ rotl2 ^ rotl3 ^ rotl4 ^ 0x63.
    def power(x, e):
        r = 1
        while e:
            if e & 1:
                r = clmul_mod(r, x)
            x = clmul_mod(x, x)
            e >>= 1
        return r

    def rotl8(v, n):
        return ((v << n) | (v >> (8 - n))) & 0xFF

    s, si = oracle.sbox()
    for x in range(256):
        inv = power(x, 254) if x else 0
        aff = inv ^ rotl8(inv, 1) ^ rotl8(inv, 2) ^ rotl8(inv, 3) ^ rotl8(inv, 4) ^ 0x63
        assert s[x] == aff


def test_sbox_permutation_properties():
    s, si = oracle.sbox()
    assert sorted(s.tolist()) == list(range(256))
    assert all(si[s[x]] == x for x in range(256))
    # design property of the AES S-box: no fixed points and no opposite fixed points
    assert all(s[x] != x and s[x] != (x ^ 0xFF) for x in range(256))


def test_key_expansion_shape_and_prefix():
    rng = np.random.default_rng(11)
    for bits in BITS:
        key = rng.integers(0, 256, bits // 8, dtype=np.uint8)
        w = oracle.key_expansion(key, bits)
        assert w.shape == (oracle.nrounds(bits) + 1, 16)
        assert w.reshape(-1)[: bits // 8].tobytes() == key.tobytes()


@pytest.mark.parametrize("bits", BITS)
def test_ecb_vs_cryptography(bits):
    rng = np.random.default_rng(bits)
    for _ in range(64):
        key = rng.integers(0, 256, bits // 8, dtype=np.uint8).tobytes()
        data = rng.integers(0, 256, 16 * 37, dtype=np.uint8).tobytes()
        enc = oracle.ecb(key, bits, data)
        assert enc.tobytes() == lib_ecb(key, data)
        dec = oracle.ecb(key, bits, data, decrypt=True)
        assert dec.tobytes() == lib_ecb(key, data, decrypt=True)


@pytest.mark.parametrize("bits", BITS)
def test_ecb_special_keys_vs_cryptography(bits):
    # all-zero / all-one keys and blocks exercise the degenerate S-box input 0
    for kb in (0x00, 0xFF):
        key = bytes([kb]) * (bits // 8)
        for db in (0x00, 0xFF):
            data = bytes([db]) * 32
            assert oracle.ecb(key, bits, data).tobytes() == lib_ecb(key, data)
            assert oracle.ecb(key, bits, data, decrypt=True).tobytes() == lib_ecb(key, data, True)


@pytest.mark.skipif(shutil.which("openssl") is None, reason="no openssl CLI")
@pytest.mark.parametrize("bits", BITS)
def test_ecb_vs_openssl_cli(bits):
    rng = np.random.default_rng(100 + bits)
    key = rng.integers(0, 256, bits // 8, dtype=np.uint8).tobytes()
    data = rng.integers(0, 256, 16 * 256, dtype=np.uint8).tobytes()
    for decrypt in (False, True):
        cmd = ["openssl", "enc", f"-aes-{bits}-ecb", "-nopad", "-K", key.hex()]
        if decrypt:
            cmd.append("-d")
        out = subprocess.run(cmd, input=data, capture_output=True, check=True).stdout
        assert oracle.ecb(key, bits, data, decrypt=decrypt).tobytes() == out


@pytest.mark.parametrize("bits", BITS)
def test_round_trip_multithreaded(bits):
    rng = np.random.default_rng(7 + bits)
    key = rng.integers(0, 256, bits // 8, dtype=np.uint8)
    data = rng.integers(0, 256, 16 * 10007, dtype=np.uint8)
    enc1 = oracle.ecb(key, bits, data, nthreads=1)
    enc8 = oracle.ecb(key, bits, data, nthreads=8)
    assert np.array_equal(enc1, enc8)
    assert np.array_equal(oracle.ecb(key, bits, enc8, decrypt=True, nthreads=5), data)


def test_empty_input():
    assert oracle.ecb(bytes(16), 128, b"").size == 0


def test_bad_key_size():
    with pytest.raises((ValueError, KeyError)):
        oracle.ecb(bytes(20), 160, bytes(16))


@pytest.mark.parametrize("bits", BITS)
def test_ctr_be128_vs_cryptography(bits):
    rng = np.random.default_rng(300 + bits)
    key = rng.integers(0, 256, bits // 8, dtype=np.uint8).tobytes()
    data = rng.integers(0, 256, 16 * 300, dtype=np.uint8).tobytes()
    ivs = [rng.integers(0, 256, 16, dtype=np.uint8).tobytes(),
           b"\xff" * 15 + b"\xf0",  # wraps past 2^128 within the message
           b"\x00" * 8 + b"\xff" * 8]  # carries out of the low 64 bits
    for iv in ivs:
        enc = Cipher(algorithms.AES(key), modes.CTR(iv)).encryptor()
        ref = enc.update(data) + enc.finalize()
        assert oracle.ctr(key, bits, iv, data, oracle.CTR_BE128).tobytes() == ref


def le32_carry_counter(iv: bytes, i: int) -> bytes:
    # The paper's counter (four little-endian 32-bit words x, y, z, w with a carry
    # chain) is a 128-bit little-endian integer addition.
    v = (int.from_bytes(iv, "little") + i) % (1 << 128)
    return v.to_bytes(16, "little")


@pytest.mark.parametrize("bits", BITS)
def test_ctr_le32_carry_vs_integer_counter(bits):
    rng = np.random.default_rng(400 + bits)
    key = rng.integers(0, 256, bits // 8, dtype=np.uint8).tobytes()
    n = 200
    data = rng.integers(0, 256, 16 * n, dtype=np.uint8).tobytes()
    ivs = [rng.integers(0, 256, 16, dtype=np.uint8).tobytes(),
           (0xFFFFFFF0).to_bytes(4, "little") + (0xFFFFFFFF).to_bytes(4, "little") * 3,  # carry x->y->z->w->wrap
           (0xFFFFFF80).to_bytes(4, "little") + (0xFFFFFFFF).to_bytes(4, "little") + bytes(8)]
    for iv in ivs:
        ctrs = b"".join(le32_carry_counter(iv, i) for i in range(n))
        ks = lib_ecb(key, ctrs)
        ref = bytes(a ^ b for a, b in zip(data, ks))
        assert oracle.ctr(key, bits, iv, data, oracle.CTR_LE32_CARRY).tobytes() == ref
        for i in (0, 1, 17, n - 1, 1 << 32, (1 << 40) + 5):
            assert oracle.counter_block(iv, i, oracle.CTR_LE32_CARRY) == le32_carry_counter(iv, i)
            assert oracle.counter_block(iv, i, oracle.CTR_BE128) == (
                (int.from_bytes(iv, "big") + i) % (1 << 128)).to_bytes(16, "big")


@pytest.mark.parametrize("bits", BITS)
def test_cbc_decrypt_vs_cryptography(bits):
    rng = np.random.default_rng(500 + bits)
    key = rng.integers(0, 256, bits // 8, dtype=np.uint8).tobytes()
    iv = rng.integers(0, 256, 16, dtype=np.uint8).tobytes()
    data = rng.integers(0, 256, 16 * 123, dtype=np.uint8).tobytes()
    dec = Cipher(algorithms.AES(key), modes.CBC(iv)).decryptor()
    ref = dec.update(data) + dec.finalize()
    assert oracle.cbc_decrypt(key, bits, iv, data, nthreads=3).tobytes() == ref


def test_golden_kat_file_matches_library_and_oracle():
    import json

    path = os.path.join(os.path.dirname(__file__), "golden", "ecb_kat.json")
    with open(path) as f:
        kat = json.load(f)
    assert len(kat["vectors"]) >= 12
    for v in kat["vectors"]:
        key, pt, ct = bytes.fromhex(v["key"]), bytes.fromhex(v["plaintext"]), bytes.fromhex(v["ciphertext"])
        assert lib_ecb(key, pt) == ct
        assert oracle.ecb(key, v["bits"], pt).tobytes() == ct


# --------------------------------------------------------------- planted mistakes

MUTATIONS = {
    # ShiftRows rotating right instead of left
    "shiftrows_direction": ("row[c] = s[r][(c + r) % 4];", "row[c] = s[r][(c + 4 - r) % 4];"),
    # MixColumns with the 3*a_{r+1} term reduced to xtime only (dropped "^ a1")
    "mixcolumns_dropped_term": ("(xtime(a1) ^ a1)", "(xtime(a1))"),
    # AES-256 key schedule without the extra SubWord at i mod Nk == 4
    "keyexp_missing_subword": ("nk > 6 && i % nk == 4", "nk > 6 && i % nk == 99"),
    # InvMixColumns with two coefficients swapped
    "invmix_swapped": ("oracle_gf_mul(a[(r + 1) % 4], 0x0b)", "oracle_gf_mul(a[(r + 1) % 4], 0x0d)"),
    # affine constant off by one bit
    "affine_constant": ("const uint8_t c = 0x63;", "const uint8_t c = 0x62;"),
    # CBC chaining with the wrong previous block
    "cbc_prev_index": ("(in - 16)", "(in)"),
}


def _mutant_lib(tmpdir, name):
    import ctypes

    src = os.path.join(os.path.dirname(oracle.__file__), "aes_oracle.c")
    text = open(src).read()
    old, new = MUTATIONS[name]
    assert text.count(old) == 1, name
    path = os.path.join(tmpdir, f"{name}.c")
    with open(path, "w") as f:
        f.write(text.replace(old, new))
    so = os.path.join(tmpdir, f"{name}.so")
    subprocess.run(["gcc", "-O1", "-fPIC", "-shared", "-pthread", path, "-o", so], check=True)
    return ctypes.CDLL(so)


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name):
    import ctypes

    u8 = ctypes.POINTER(ctypes.c_uint8)
    rng = np.random.default_rng(9)
    with tempfile.TemporaryDirectory() as d:
        lib = _mutant_lib(d, name)
        caught = False
        for bits in BITS:
            key = rng.integers(0, 256, bits // 8, dtype=np.uint8)
            iv = rng.integers(0, 256, 16, dtype=np.uint8)
            data = rng.integers(0, 256, 16 * 8, dtype=np.uint8)
            out = np.empty_like(data)
            kb, db = key.tobytes(), data.tobytes()
            for decrypt in (0, 1):
                lib.oracle_ecb(key.ctypes.data_as(u8), bits, decrypt, data.ctypes.data_as(u8),
                               out.ctypes.data_as(u8), ctypes.c_uint64(8), 1)
                caught |= out.tobytes() != lib_ecb(kb, db, bool(decrypt))
            lib.oracle_cbc_decrypt(key.ctypes.data_as(u8), bits, iv.ctypes.data_as(u8), data.ctypes.data_as(u8),
                                   out.ctypes.data_as(u8), ctypes.c_uint64(8), 1)
            dec = Cipher(algorithms.AES(kb), modes.CBC(iv.tobytes())).decryptor()
            caught |= out.tobytes() != dec.update(db) + dec.finalize()
        assert caught, f"mutation {name} was not detected by the library cross-check"
