"""Seeded randomised differential test: every public single-buffer call against the oracle.

Each case draws a key size, an operation (ECB encryption or decryption on one
of the four kernel variants with a random launch shape, CTR with either counter
layout and a random first block index, or CBC decryption), a length
log-uniform over 1 .. 65,536 blocks, an offset into a larger device buffer
(any multiple of 16 bytes) and in-place or separate output (CBC decryption
refuses in place, which the test checks).  The output must
equal the oracle's byte for byte and the bytes around the output range must be
untouched; the device status word must stay 0.
"""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = 160
THREADS = (0, 64, 96, 128, 256, 512, 1024)
BPT = (0, 1, 2, 4)


def test_random_calls_match_oracle(gbaes):
    rng = np.random.default_rng(20261203)
    kernels = (gbaes.KERNEL_TABLE, gbaes.KERNEL_TABLE_COMPACT, gbaes.KERNEL_TABLE_REPLICATED,
               gbaes.KERNEL_BITSLICED)
    pad = 64  # bytes of guard on both sides of every output range
    for case in range(CASES):
        bits = int(rng.choice((128, 192, 256)))
        key = rng.integers(0, 256, bits // 8, dtype=np.uint8).tobytes()
        k = gbaes.Key(key)
        n = int(np.exp(rng.uniform(0, np.log(65536))))
        off = 16 * int(rng.integers(0, 64))
        data = rng.integers(0, 256, 16 * n, dtype=np.uint8)
        buf = torch.from_numpy(rng.integers(0, 256, off + 16 * n + pad, dtype=np.uint8)).cuda()
        before = buf.cpu().numpy()
        buf[off:off + 16 * n] = torch.from_numpy(data).cuda()
        x = buf[off:off + 16 * n]
        op = int(rng.integers(0, 4))
        in_place = bool(rng.integers(0, 2))
        if in_place and op == 3:  # CBC decryption reads the ciphertext before each block: never in place
            with pytest.raises(gbaes.AesError):
                gbaes.cbc_decrypt(k, bytes(16), x, x)
            in_place = False
        if in_place:
            out, guard, base = x, buf, off
        else:
            guard = torch.from_numpy(rng.integers(0, 256, 2 * pad + 16 * n, dtype=np.uint8)).cuda()
            out, base = guard[pad:pad + 16 * n], pad
            before = guard.cpu().numpy()
        if op <= 1:  # ECB
            kern = int(rng.choice(kernels))
            th, bpt = int(rng.choice(THREADS)), int(rng.choice(BPT))
            gbaes.ecb_ex(k, x, out, decrypt=bool(op), kernel=kern, threads=th, blocks_per_thread=bpt)
            want = oracle.ecb(key, bits, data, decrypt=bool(op))
            what = (case, "ecb", op, kern, th, bpt, n, off, in_place)
        elif op == 2:  # CTR
            kind = int(rng.choice((oracle.CTR_BE128, oracle.CTR_LE32_CARRY)))
            iv = rng.integers(0, 256, 16, dtype=np.uint8).tobytes()
            first = [0, int(rng.integers(0, 1 << 40)), (1 << 64) - n][int(rng.integers(0, 3))]
            gbaes.ctr_xcrypt(k, iv, x, out, kind=kind, first_block=first)
            want = oracle.ctr(key, bits, oracle.counter_block(iv, first, kind), data, kind)
            what = (case, "ctr", kind, first, n, off, in_place)
        else:  # CBC decryption
            iv = rng.integers(0, 256, 16, dtype=np.uint8).tobytes()
            gbaes.cbc_decrypt(k, iv, x, out)
            want = oracle.cbc_decrypt(key, bits, iv, data)
            what = (case, "cbc", n, off, in_place)
        torch.cuda.synchronize()
        got_all = guard.cpu().numpy()
        assert np.array_equal(got_all[base:base + 16 * n], want), what
        assert np.array_equal(got_all[:base], before[:base]), ("wrote before the range",) + what
        assert np.array_equal(got_all[base + 16 * n:], before[base + 16 * n:]), ("wrote past the range",) + what
    assert gbaes.device_status() == 0
