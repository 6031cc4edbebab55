"""GPU parity: the T-table kernels against the CPU oracle, bit for bit.

AES is a permutation per key, so the result is unique and the tolerance is zero
(Section 2.1's cipher; Eq. 1 is a re-arrangement of the same arithmetic).
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1201_0398_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BITS = (128, 192, 256)


def dev(a: np.ndarray):
    a = np.ascontiguousarray(a)
    return torch.from_numpy(a if a.flags.writeable else a.copy()).cuda()


def host(t) -> np.ndarray:
    torch.cuda.synchronize()
    return t.cpu().numpy()


def sms():
    return torch.cuda.get_device_properties(0).multi_processor_count


def test_small_workload_encrypt_then_decrypt(gbaes):
    key, data = workloads.small_workload()
    k = gbaes.Key(key)
    x = dev(data)
    c = gbaes.encrypt_ecb(k, x)
    p = gbaes.decrypt_ecb(k, c)
    want_c = oracle.ecb(key, 128, data)
    assert np.array_equal(host(c), want_c)
    assert np.array_equal(host(p), data)
    assert np.array_equal(host(p), oracle.ecb(key, 128, want_c, decrypt=True))
    assert gbaes.device_status() == 0


def edge_sizes():
    tile = 1024 * 2
    full = sms() * tile
    return sorted({1, 2, 3, 31, 32, 33, 1023, 1024, 1025, tile - 1, tile, tile + 1, full - 1, full, full + 1,
                   3 * full + 17})


@pytest.mark.parametrize("bits", BITS)
@pytest.mark.parametrize("decrypt", (False, True))
def test_edge_sizes_vs_oracle(gbaes, bits, decrypt):
    rng = np.random.default_rng(bits + 7 * decrypt)
    key = rng.integers(0, 256, bits // 8, dtype=np.uint8).tobytes()
    k = gbaes.Key(key)
    for n in edge_sizes():
        data = rng.integers(0, 256, 16 * n, dtype=np.uint8)
        out = (gbaes.decrypt_ecb if decrypt else gbaes.encrypt_ecb)(k, dev(data))
        assert np.array_equal(host(out), oracle.ecb(key, bits, data, decrypt=decrypt)), n


@pytest.mark.parametrize("threads", (64, 256, 512, 768, 1024))
@pytest.mark.parametrize("bpt", (1, 2, 4))
def test_every_launch_shape(gbaes, threads, bpt):
    rng = np.random.default_rng(threads * 10 + bpt)
    n = sms() * threads * bpt + threads + 5  # all CTAs busy, a second pass, a ragged tail
    for bits in (128, 256):
        key = rng.integers(0, 256, bits // 8, dtype=np.uint8).tobytes()
        k = gbaes.Key(key)
        data = rng.integers(0, 256, 16 * n, dtype=np.uint8)
        for decrypt in (False, True):
            out = gbaes.ecb_ex(k, dev(data), decrypt=decrypt, threads=threads, blocks_per_thread=bpt)
            assert np.array_equal(host(out), oracle.ecb(key, bits, data, decrypt=decrypt))


def test_in_place_and_side_stream(gbaes):
    rng = np.random.default_rng(5)
    key = rng.integers(0, 256, 32, dtype=np.uint8).tobytes()
    k = gbaes.Key(key)
    data = rng.integers(0, 256, 16 * 100_003, dtype=np.uint8)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        x = dev(data)
        gbaes.encrypt_ecb(k, x, out=x)
        s.synchronize()
    assert np.array_equal(host(x), oracle.ecb(key, 256, data))
    gbaes.decrypt_ecb(k, x, out=x, stream=s)
    s.synchronize()
    assert np.array_equal(host(x), data)


def test_golden_known_answers(gbaes):
    path = os.path.join(os.path.dirname(__file__), "golden", "ecb_kat.json")
    for v in json.load(open(path))["vectors"]:
        k = gbaes.Key(bytes.fromhex(v["key"]))
        pt = np.frombuffer(bytes.fromhex(v["plaintext"]), np.uint8)
        ct = np.frombuffer(bytes.fromhex(v["ciphertext"]), np.uint8)
        assert host(gbaes.encrypt_ecb(k, dev(pt))).tobytes() == ct.tobytes()
        assert host(gbaes.decrypt_ecb(k, dev(ct))).tobytes() == pt.tobytes()


def test_argument_errors(gbaes):
    k = gbaes.Key(bytes(16))
    buf = torch.zeros(16 * 64 + 16, dtype=torch.uint8, device="cuda")
    with pytest.raises(gbaes.AesError) as e:  # misaligned
        gbaes.encrypt_ecb(k, buf[1:1 + 16 * 8], out=buf[32:32 + 16 * 8].clone())
    assert e.value.name == "AES_ERR_ALIGN"
    with pytest.raises(gbaes.AesError) as e:  # partial overlap
        gbaes.encrypt_ecb(k, buf[0:16 * 8], out=buf[16:16 * 9])
    assert e.value.name == "AES_ERR_ARG"
    lib = gbaes.load()
    import ctypes

    base = ctypes.c_void_p(buf.data_ptr())
    # a range running past the end of its allocation is rejected on the host
    big = torch.zeros(16 * 4, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    rc = lib.aes_encrypt_ecb(k.handle, ctypes.c_void_p(big.data_ptr()), ctypes.c_void_p(big.data_ptr()),
                             1 << 40, None)
    assert rc == -1
    assert lib.aes_encrypt_ecb(k.handle, base, base, 0, None) == 0  # empty input: no-op
    with pytest.raises(gbaes.AesError):
        gbaes.ecb_ex(k, buf[:16 * 8], threads=100)
    with pytest.raises(gbaes.AesError):
        gbaes.ecb_ex(k, buf[:16 * 8], blocks_per_thread=3)
    assert gbaes.device_status() == 0


@pytest.mark.parametrize("bits", BITS)
def test_ctr_vs_oracle(gbaes, bits):
    rng = np.random.default_rng(600 + bits)
    key = rng.integers(0, 256, bits // 8, dtype=np.uint8).tobytes()
    k = gbaes.Key(key)
    n = 3 * sms() * 2048 + 77
    data = rng.integers(0, 256, 16 * n, dtype=np.uint8)
    ivs = [rng.integers(0, 256, 16, dtype=np.uint8).tobytes(), b"\xff" * 16,
           (0xFFFFFF00).to_bytes(4, "little") + b"\xff" * 4 + bytes(8)]
    for iv in ivs:
        for kind in (oracle.CTR_BE128, oracle.CTR_LE32_CARRY):
            out = gbaes.ctr_xcrypt(k, iv, dev(data), kind=kind)
            assert np.array_equal(host(out), oracle.ctr(key, bits, iv, data, kind)), (iv.hex(), kind)
    # a message processed in two pieces equals one call (first_block offsets the counter)
    iv = ivs[0]
    x = dev(data)
    half = (n // 2) * 16
    a = gbaes.ctr_xcrypt(k, iv, x[:half])
    b = gbaes.ctr_xcrypt(k, iv, x[half:], first_block=n // 2)
    assert np.array_equal(np.concatenate([host(a), host(b)]), oracle.ctr(key, bits, iv, data))
    # in place
    gbaes.ctr_xcrypt(k, iv, x, out=x)
    assert np.array_equal(host(x), oracle.ctr(key, bits, iv, data))


@pytest.mark.parametrize("bits", BITS)
def test_cbc_decrypt_vs_oracle(gbaes, bits):
    rng = np.random.default_rng(700 + bits)
    key = rng.integers(0, 256, bits // 8, dtype=np.uint8).tobytes()
    iv = rng.integers(0, 256, 16, dtype=np.uint8).tobytes()
    k = gbaes.Key(key)
    for n in (1, 2, 33, 2 * sms() * 2048 + 5):
        data = rng.integers(0, 256, 16 * n, dtype=np.uint8)
        out = gbaes.cbc_decrypt(k, iv, dev(data))
        assert np.array_equal(host(out), oracle.cbc_decrypt(key, bits, iv, data)), n
    x = dev(data)
    with pytest.raises(gbaes.AesError):
        gbaes.cbc_decrypt(k, iv, x, out=x)
    # two pieces chained through the iv argument
    h = (n // 2) * 16
    a = gbaes.cbc_decrypt(k, iv, x[:h])
    b = gbaes.cbc_decrypt(k, data[h - 16:h].tobytes(), x[h:])
    assert np.array_equal(np.concatenate([host(a), host(b)]), oracle.cbc_decrypt(key, bits, iv, data))


def sampled_parity(key, bits, x, out, decrypt, nsample=1 << 15, seed=0):
    """Compares out against the oracle on nsample random blocks of x."""
    nblocks = x.numel() // 16
    idx = np.random.default_rng(seed).choice(nblocks, size=min(nsample, nblocks), replace=False)
    idx = np.concatenate([idx, [0, nblocks - 1]])
    ti = torch.from_numpy(idx).cuda()
    xs = host(x.view(-1, 16)[ti]).reshape(-1)
    os_ = host(out.view(-1, 16)[ti]).reshape(-1)
    assert np.array_equal(os_, oracle.ecb(key, bits, xs, decrypt=decrypt))


@pytest.mark.parametrize("bits", BITS)
def test_one_gib_single_launch(gbaes, bits):
    """1 GiB device-resident buffer per key size, one launch per direction:
    sampled blocks against the oracle, and decrypt(encrypt(x)) == x everywhere."""
    key = workloads.random_key(workloads.SEED_BULK[bits], bits)
    k = gbaes.Key(key)
    x = workloads.device_bytes(workloads.SEED_BULK[bits], workloads.GiB)
    c = gbaes.encrypt_ecb(k, x)
    sampled_parity(key, bits, x, c, False)
    p = gbaes.decrypt_ecb(k, c)
    sampled_parity(key, bits, c, p, True, seed=1)
    assert torch.equal(p, x)
    del c, p, x
    torch.cuda.empty_cache()


@pytest.mark.parametrize("bits", (128, 256))
@pytest.mark.parametrize("kind", (oracle.CTR_BE128, oracle.CTR_LE32_CARRY))
def test_ctr_and_cbc_one_gib(gbaes, bits, kind):
    """The modes at the bench's size (1 GiB, 2^26 blocks, one launch each): the
    CTR keystream (output XOR input) on 2^14 sampled blocks equals the oracle's
    encryption of those blocks' counter blocks, and CTR applied twice gives the
    input back everywhere; CBC decryption on sampled blocks (the first, whose
    predecessor is the IV, and the last included) equals the oracle's
    decryption of the block XOR the previous ciphertext block."""
    key = workloads.random_key(90 + bits, bits)
    k = gbaes.Key(key)
    x = workloads.device_bytes(91 + bits, workloads.GiB)
    n = x.numel() // 16
    iv = bytes(range(0xF0, 0x100))  # low bytes near a carry
    rng = np.random.default_rng(bits + kind)
    idx = np.concatenate([[0, 1, n - 1], rng.choice(n, 1 << 14, replace=False)])
    ti = torch.from_numpy(idx).cuda()
    xb = host(x.view(-1, 16)[ti])
    c = gbaes.ctr_xcrypt(k, iv, x, kind=kind)
    ks = host(c.view(-1, 16)[ti]) ^ xb
    ctrs = np.frombuffer(b"".join(oracle.counter_block(iv, int(i), kind) for i in idx), np.uint8)
    assert np.array_equal(ks.reshape(-1), oracle.ecb(key, bits, ctrs))
    assert torch.equal(gbaes.ctr_xcrypt(k, iv, c, kind=kind), x)
    del c
    if kind == oracle.CTR_BE128:
        d = gbaes.cbc_decrypt(k, iv, x)
        prev_idx = torch.from_numpy(np.maximum(idx - 1, 0)).cuda()
        prev = host(x.view(-1, 16)[prev_idx])
        prev[idx == 0] = np.frombuffer(iv, np.uint8)
        want = oracle.ecb(key, bits, xb.reshape(-1), decrypt=True).reshape(-1, 16) ^ prev
        assert np.array_equal(host(d.view(-1, 16)[ti]), want)
        del d
    del x
    torch.cuda.empty_cache()


@pytest.mark.parametrize("gib", (4, 16))
def test_sweep_top_sizes_sampled(gbaes, gib):
    """The largest sweep points (4 and 16 GiB; 2^28 and 2^30 blocks): 64-bit
    block indices.  AES-128 and AES-256 encryption against the oracle on 2^20
    sampled blocks (plus the first and last), and the whole output against the
    bitsliced kernel's, which shares no table, round or indexing code."""
    free, _ = torch.cuda.mem_get_info()
    if free < 3 * gib * workloads.GiB + workloads.GiB:
        pytest.skip("not enough device memory")
    x = workloads.device_bytes(11, gib * workloads.GiB)
    for bits in (128, 256):
        key = workloads.random_key(20 + bits, bits)
        k = gbaes.Key(key)
        c = gbaes.encrypt_ecb(k, x)
        sampled_parity(key, bits, x, c, False, nsample=1 << 20, seed=bits)
        b = gbaes.ecb_ex(k, x, kernel=gbaes.KERNEL_BITSLICED)
        assert torch.equal(b, c)
        del b, c
    del x
    torch.cuda.empty_cache()


@pytest.mark.parametrize("bits", BITS)
def test_bitsliced_kernel_vs_oracle(gbaes, bits):
    """The Boolean-circuit kernel (a lane pair holds 32 blocks as bit planes, split
    by state columns; a warp takes 512 blocks, a CTA 2,048): edge sizes around a
    pair's, a warp's and a CTA's tile, and more than one pass of the full grid
    (152 SMs x 4 CTAs for decryption, x 5 for encryption, x 2,048 blocks) with a
    ragged tail."""
    rng = np.random.default_rng(900 + bits)
    key = rng.integers(0, 256, bits // 8, dtype=np.uint8).tobytes()
    k = gbaes.Key(key)
    for n in (1, 15, 16, 17, 31, 33, 511, 512, 513, 2047, 2049, 4097, sms() * 5 * 2048 + 2048 * 3 + 5):
        data = rng.integers(0, 256, 16 * n, dtype=np.uint8)
        for decrypt in (False, True):
            out = gbaes.ecb_ex(k, dev(data), decrypt=decrypt, kernel=gbaes.KERNEL_BITSLICED)
            assert np.array_equal(host(out), oracle.ecb(key, bits, data, decrypt=decrypt)), (n, decrypt)


def test_bitsliced_equals_table_kernel_large(gbaes):
    x = workloads.device_bytes(77, 256 << 20)
    for bits in BITS:
        k = gbaes.Key(workloads.random_key(70 + bits, bits))
        for decrypt in (False, True):
            a = gbaes.ecb_ex(k, x, decrypt=decrypt, kernel=gbaes.KERNEL_TABLE)
            b = gbaes.ecb_ex(k, x, decrypt=decrypt, kernel=gbaes.KERNEL_BITSLICED)
            assert torch.equal(a, b)


def test_ctr_counter_index_limit(gbaes):
    """Block indices are 64-bit: a call whose last index would pass 2^64 - 1 is
    refused on the host; one ending exactly at 2^64 - 1 runs, its counters
    taken as IV + index modulo 2^128 (checked against plain integer arithmetic
    and ECB of those counter blocks)."""
    key = bytes(range(16))
    k = gbaes.Key(key)
    iv = bytes(16)
    x = torch.zeros(16 * 4, dtype=torch.uint8, device="cuda")
    with pytest.raises(gbaes.AesError):
        gbaes.ctr_xcrypt(k, iv, x, first_block=(1 << 64) - 3)
    first = (1 << 64) - 4
    out = host(gbaes.ctr_xcrypt(k, iv, x, first_block=first))
    ctrs = b"".join((first + i).to_bytes(16, "big") for i in range(4))
    assert out.tobytes() == oracle.ecb(key, 128, np.frombuffer(ctrs, np.uint8)).tobytes()


def test_default_kernel_switch(gbaes):
    """aes_set_kernel changes what aes_encrypt_ecb / aes_decrypt_ecb run; the
    result is the same bytes either way."""
    rng = np.random.default_rng(55)
    key = rng.integers(0, 256, 24, dtype=np.uint8).tobytes()
    k = gbaes.Key(key)
    data = rng.integers(0, 256, 16 * 5000, dtype=np.uint8)
    want = oracle.ecb(key, 192, data)
    prev = gbaes.set_kernel(gbaes.KERNEL_BITSLICED)
    try:
        assert np.array_equal(host(gbaes.encrypt_ecb(k, dev(data))), want)
        assert np.array_equal(host(gbaes.decrypt_ecb(k, dev(want))), data)
    finally:
        gbaes.set_kernel(prev)
    assert np.array_equal(host(gbaes.encrypt_ecb(k, dev(data))), want)


@pytest.mark.parametrize("shape", __import__("paper_1201_0398_gb300.autotune", fromlist=["x"]).ECB_CANDIDATES)
def test_one_gib_every_tuner_shape(gbaes, shape):
    """The 1 GiB single-launch workload in every launch shape the autotuner may
    pick for the bench: sampled blocks against the oracle, AES-128 encryption and
    AES-256 decryption (the bench's dominant launch)."""
    threads, bpt = shape
    x = workloads.device_bytes(workloads.SEED_BULK[128], workloads.GiB)
    for bits, dec in ((128, False), (256, True)):
        key = workloads.random_key(workloads.SEED_BULK[bits], bits)
        k = gbaes.Key(key)
        out = gbaes.ecb_ex(k, x, decrypt=dec, threads=threads, blocks_per_thread=bpt)
        sampled_parity(key, bits, x, out, dec, nsample=1 << 13, seed=threads + bpt)
        del out
    del x
    torch.cuda.empty_cache()


def compact_sizes():
    """Sizes around the compact kernel's shapes: one warp, warps spread one per
    SM, 8 warps per CTA, the grid cap (8 CTAs per SM) with a grid-stride tail."""
    w = 32
    return sorted({1, 2, 31, 32, 33, 255, 256, 257, sms() * w - 1, sms() * w, sms() * w + 1,
                   sms() * 8 * w + 3, 8 * sms() * 8 * w - 1, 8 * sms() * 8 * w + 1000})


@pytest.mark.parametrize("bits", BITS)
def test_compact_tables_vs_oracle(gbaes, bits):
    """The compact-table kernel (each table stored once) in every mode."""
    rng = np.random.default_rng(1300 + bits)
    key = rng.integers(0, 256, bits // 8, dtype=np.uint8).tobytes()
    iv = rng.integers(0, 256, 16, dtype=np.uint8).tobytes()
    k = gbaes.Key(key)
    for n in compact_sizes():
        data = rng.integers(0, 256, 16 * n, dtype=np.uint8)
        x = dev(data)
        for decrypt in (False, True):
            out = gbaes.ecb_ex(k, x, decrypt=decrypt, kernel=gbaes.KERNEL_TABLE_COMPACT)
            assert np.array_equal(host(out), oracle.ecb(key, bits, data, decrypt=decrypt)), (n, decrypt)
        if n <= 128 * sms():  # CTR and CBC decryption take the compact tables for calls this small
            for kind in (oracle.CTR_BE128, oracle.CTR_LE32_CARRY):
                assert np.array_equal(host(gbaes.ctr_xcrypt(k, iv, x, kind=kind)),
                                      oracle.ctr(key, bits, iv, data, kind)), (n, kind)
            assert np.array_equal(host(gbaes.cbc_decrypt(k, iv, x)), oracle.cbc_decrypt(key, bits, iv, data)), n
    assert gbaes.device_status() == 0


@pytest.mark.parametrize("decrypt", (False, True))
def test_size_dispatch_and_balanced_shapes_vs_oracle(gbaes, decrypt):
    """AES_KERNEL_TABLE picks compact tables for small calls and the replicated
    tables above; the replicated kernel shrinks its CTAs so that calls of a few
    tiles per SM spread evenly.  Sizes on both sides of the switch and across
    the shrinking range, through the default call and both variants forced."""
    rng = np.random.default_rng(1400 + decrypt)
    s = sms()
    for bits in (128, 256):
        key = rng.integers(0, 256, bits // 8, dtype=np.uint8).tobytes()
        k = gbaes.Key(key)
        for n in (128 * s - 1, 128 * s, 128 * s + 1, 65536, 3 * s * 1024 + 7, 262144, (1 << 20) + 13):
            data = rng.integers(0, 256, 16 * n, dtype=np.uint8)
            want = oracle.ecb(key, bits, data, decrypt=decrypt)
            x = dev(data)
            out = (gbaes.decrypt_ecb if decrypt else gbaes.encrypt_ecb)(k, x)
            assert np.array_equal(host(out), want), n
            for kid in (gbaes.KERNEL_TABLE_REPLICATED, gbaes.KERNEL_TABLE_COMPACT):
                for bpt in (1, 2, 4):
                    out = gbaes.ecb_ex(k, x, decrypt=decrypt, kernel=kid, blocks_per_thread=bpt)
                    assert np.array_equal(host(out), want), (n, kid, bpt)
    assert gbaes.device_status() == 0
