"""Seeded synthetic inputs for the benchmarks and tests (no cipher arithmetic here).

The paper measures on data of "different input data size" with no named dataset
(Section 3.1, Fig. 4); these generators stand in for it.  Keys and payload bytes
are uniform random, drawn from numpy's PCG64 (``default_rng(seed)``) on the host
or from torch's CUDA generator for device-resident buffers of a GiB and more.
Both the GPU path and the CPU oracle consume what these functions return.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

MiB = 1 << 20
GiB = 1 << 30

# Seeds per workload: the small end-to-end check, then one per key size of the
# 1 GiB single-launch workload, then the batched and the serving workloads.
SEED_SMALL = 0
SEED_BULK = {128: 1, 192: 2, 256: 3}
SEED_BATCH = 4
SEED_SERVE = 5


def random_key(seed: int, bits: int) -> bytes:
    """bits/8 uniform random key bytes."""
    return np.random.default_rng(seed).integers(0, 256, bits // 8, dtype=np.uint8).tobytes()


def host_bytes(seed: int, nbytes: int) -> np.ndarray:
    """nbytes uniform random bytes on the host."""
    return np.random.default_rng(seed).integers(0, 256, nbytes, dtype=np.uint8)


def small_workload():
    """AES-128 key + 1 MiB (65,536 blocks) plaintext, both from seed 0."""
    rng = np.random.default_rng(SEED_SMALL)
    key = rng.integers(0, 256, 16, dtype=np.uint8).tobytes()
    data = rng.integers(0, 256, MiB, dtype=np.uint8)
    return key, data


def device_bytes(seed: int, nbytes: int, device="cuda"):
    """nbytes uniform random bytes generated directly on a CUDA device."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed)
    return torch.randint(0, 256, (nbytes,), dtype=torch.uint8, device=device, generator=g)


@dataclass
class BatchWorkload:
    """Messages for the batched launch.

    lengths: bytes per message (multiples of 16); bits: key size per message;
    decrypt: direction per message; keys: one key per message.
    """

    lengths: np.ndarray
    bits: np.ndarray
    decrypt: np.ndarray
    keys: list

    @property
    def total_bytes(self) -> int:
        return int(self.lengths.sum())


def batch_workload(n: int = 10_000, seed: int = SEED_BATCH, min_len: int = 16, max_len: int = 4 * MiB) -> BatchWorkload:
    """n messages, lengths log-uniform in [min_len, max_len] rounded to 16 B, key
    sizes 128/192/256 in ratio 2:1:1 (fixed counts, shuffled), direction a fair coin."""
    rng = np.random.default_rng(seed)
    raw = np.exp(rng.uniform(np.log(min_len), np.log(max_len), n))
    lengths = np.maximum(16, np.round(raw / 16).astype(np.int64) * 16)
    n128 = n // 2
    n192 = (n - n128) // 2
    bits = np.array([128] * n128 + [192] * n192 + [256] * (n - n128 - n192), dtype=np.int64)
    rng.shuffle(bits)
    decrypt = rng.integers(0, 2, n).astype(bool)
    keys = [rng.integers(0, 256, b // 8, dtype=np.uint8).tobytes() for b in bits]
    return BatchWorkload(lengths=lengths, bits=bits, decrypt=decrypt, keys=keys)


@dataclass
class ServeWorkload:
    """Open-loop request stream for the server.

    arrival_s: scheduled arrival time of each request (seconds from start);
    lengths: bytes; key_index: index into the resident key set; decrypt: direction;
    keys/key_bits: the resident key set.
    """

    arrival_s: np.ndarray
    lengths: np.ndarray
    key_index: np.ndarray
    decrypt: np.ndarray
    keys: list
    key_bits: np.ndarray


def serve_workload(rate: float = 200_000.0, duration_s: float = 10.0, nkeys: int = 1024, seed: int = SEED_SERVE,
                   min_len: int = 64, max_len: int = MiB) -> ServeWorkload:
    """Poisson arrivals (exponential gaps of mean 1/rate) over duration_s, sizes
    log-uniform in [min_len, max_len] rounded to 16 B, keys uniform over nkeys
    resident keys of all three sizes, encrypt/decrypt 50/50."""
    rng = np.random.default_rng(seed)
    expected = int(rate * duration_s * 1.1) + 16
    gaps = rng.exponential(1.0 / rate, expected)
    t = np.cumsum(gaps)
    t = t[t < duration_s]
    n = t.size
    raw = np.exp(rng.uniform(np.log(min_len), np.log(max_len), n))
    lengths = np.maximum(16, np.round(raw / 16).astype(np.int64) * 16)
    key_bits = np.array([(128, 192, 256)[i % 3] for i in range(nkeys)], dtype=np.int64)
    keys = [rng.integers(0, 256, b // 8, dtype=np.uint8).tobytes() for b in key_bits]
    key_index = rng.integers(0, nkeys, n)
    decrypt = rng.integers(0, 2, n).astype(bool)
    return ServeWorkload(arrival_s=t, lengths=lengths, key_index=key_index, decrypt=decrypt, keys=keys,
                         key_bits=key_bits)
