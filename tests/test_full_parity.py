"""Full-buffer parity at the measured sizes: every output byte against the CPU oracle.

The bench's workloads are large ECB buffers (Section 3.1, Fig. 4: 1 GiB per key
size here, one launch per operation), the CTR and CBC-decryption modes of
Section 3 (Eq. 2) on the same 1 GiB buffers, and the batched workload (10,000
messages, each with its own key).  These tests run those exact inputs through
the C ABI, copy every output to the host and compare it byte for byte with the
oracle run on all host cores -- no sampling.  AES is a permutation per key, so
the tolerance is zero.  They take a few minutes (the oracle enciphers ~13 GB).
"""
import os

import numpy as np
import pytest

import oracle
from paper_1201_0398_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

CORES = os.cpu_count() or 1


def host(t) -> np.ndarray:
    torch.cuda.synchronize()
    return t.cpu().numpy()


def first_difference(got: np.ndarray, want: np.ndarray) -> str:
    bad = np.flatnonzero(got != want)
    return f"{bad.size} bytes differ, first at byte {bad[0]} (block {bad[0] // 16})" if bad.size else ""


@pytest.mark.parametrize("bits", (128, 192, 256))
def test_one_gib_ecb_every_byte(gbaes, bits):
    """The bench's buffer for this key size (seeded as the bench seeds it), one
    encryption launch and one decryption launch of the ciphertext."""
    key = workloads.random_key(workloads.SEED_BULK[bits], bits)
    k = gbaes.Key(key)
    x = workloads.device_bytes(workloads.SEED_BULK[bits], workloads.GiB)
    c = gbaes.encrypt_ecb(k, x)
    p = gbaes.decrypt_ecb(k, c)
    xh, ch, ph = host(x), host(c), host(p)
    del x, c, p
    torch.cuda.empty_cache()
    want_c = oracle.ecb(key, bits, xh, nthreads=CORES)
    assert np.array_equal(ch, want_c), first_difference(ch, want_c)
    want_p = oracle.ecb(key, bits, ch, decrypt=True, nthreads=CORES)
    assert np.array_equal(ph, want_p), first_difference(ph, want_p)
    assert np.array_equal(ph, xh)


@pytest.mark.parametrize("bits", (128, 256))
def test_one_gib_ctr_and_cbc_every_byte(gbaes, bits):
    """CTR (both counter layouts) and CBC decryption on the bench's 1 GiB buffer
    with the bench's IV (bytes 00..0f)."""
    key = workloads.random_key(workloads.SEED_BULK[bits], bits)
    k = gbaes.Key(key)
    iv = bytes(range(16))
    x = workloads.device_bytes(workloads.SEED_BULK[bits], workloads.GiB)
    xh = host(x)
    for kind in (oracle.CTR_BE128, oracle.CTR_LE32_CARRY):
        got = host(gbaes.ctr_xcrypt(k, iv, x, kind=kind))
        want = oracle.ctr(key, bits, iv, xh, kind, nthreads=CORES)
        assert np.array_equal(got, want), (kind, first_difference(got, want))
        del got, want
    got = host(gbaes.cbc_decrypt(k, iv, x))
    del x
    torch.cuda.empty_cache()
    want = oracle.cbc_decrypt(key, bits, iv, xh, nthreads=CORES)
    assert np.array_equal(got, want), first_difference(got, want)


def test_batched_workload_every_message(gbaes):
    """The 10,000-message batch (log-uniform 16 B - 4 MiB, one key each, key
    sizes 2:1:1, mixed directions) in one launch of the plan shape the
    autotuner picks on the GB300 (512 threads x 8 blocks per thread), every
    message against the oracle with its own key and direction."""
    w = workloads.batch_workload()
    ks = [gbaes.Key(k) for k in w.keys]
    off = np.concatenate([[0], np.cumsum(w.lengths)[:-1]])
    d = gbaes.make_descs(off, off, w.lengths // 16, np.arange(len(ks)), w.decrypt)
    x = workloads.device_bytes(workloads.SEED_BATCH, w.total_bytes)
    y = torch.empty_like(x)
    gbaes.BatchPlan(d, ks, 512, 8).launch(x, y)
    xh, yh = host(x), host(y)
    del x, y
    torch.cuda.empty_cache()
    bad = []
    for i in range(len(ks)):
        a, n = int(off[i]), int(w.lengths[i])
        want = oracle.ecb(w.keys[i], int(w.bits[i]), xh[a:a + n], decrypt=bool(w.decrypt[i]), nthreads=CORES)
        if not np.array_equal(yh[a:a + n], want):
            bad.append(i)
    assert not bad, f"{len(bad)} messages differ, first {bad[:5]}"
