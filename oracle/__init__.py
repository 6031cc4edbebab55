"""CPU oracle for bulk AES -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` import this package.  The product
path (``paper_1201_0398_gb300``) never imports it and shares no code with it.

The arithmetic lives in ``aes_oracle.c`` (plain byte-oriented FIPS-197 AES, the
cipher that Section 2.1 of the paper builds on); this module only compiles it
with gcc and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import build_oracle

__all__ = [
    "CTR_BE128",
    "CTR_LE32_CARRY",
    "sbox",
    "gf_mul",
    "key_expansion",
    "ecb",
    "ctr",
    "cbc_decrypt",
    "counter_block",
    "nrounds",
]

CTR_BE128 = 0
CTR_LE32_CARRY = 1

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = build_oracle()
        lib = ctypes.CDLL(path)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        lib.oracle_gf_mul.restype = ctypes.c_uint8
        lib.oracle_gf_mul.argtypes = [ctypes.c_uint8, ctypes.c_uint8]
        lib.oracle_sbox.restype = None
        lib.oracle_sbox.argtypes = [u8p, u8p]
        lib.oracle_key_expansion.restype = ctypes.c_int
        lib.oracle_key_expansion.argtypes = [u8p, ctypes.c_int, u8p]
        lib.oracle_ecb.restype = ctypes.c_int
        lib.oracle_ecb.argtypes = [u8p, ctypes.c_int, ctypes.c_int, u8p, u8p, ctypes.c_uint64, ctypes.c_int]
        lib.oracle_ctr.restype = ctypes.c_int
        lib.oracle_ctr.argtypes = [u8p, ctypes.c_int, u8p, ctypes.c_int, u8p, u8p, ctypes.c_uint64, ctypes.c_int]
        lib.oracle_cbc_decrypt.restype = ctypes.c_int
        lib.oracle_cbc_decrypt.argtypes = [u8p, ctypes.c_int, u8p, u8p, u8p, ctypes.c_uint64, ctypes.c_int]
        lib.oracle_counter_block.restype = None
        lib.oracle_counter_block.argtypes = [u8p, ctypes.c_int, ctypes.c_uint64, u8p]
        _lib = lib
    return _lib


def _u8(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def _bytes_arr(x, n=None) -> np.ndarray:
    a = np.ascontiguousarray(np.frombuffer(bytes(x), dtype=np.uint8) if isinstance(x, (bytes, bytearray)) else x,
                             dtype=np.uint8)
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} bytes, got {a.size}")
    return a


def _threads(nthreads):
    return int(nthreads) if nthreads else (os.cpu_count() or 1)


def _check(rc: int):
    if rc != 0:
        raise ValueError(f"oracle error {rc}")


def nrounds(bits: int) -> int:
    """Rounds per key size (Section 2.1: 10, 12 or 14)."""
    return {128: 10, 192: 12, 256: 14}[bits]


def gf_mul(a: int, b: int) -> int:
    """Product in GF(2^8) (Section 2.1's field, modulus x^8+x^4+x^3+x+1)."""
    return int(_load().oracle_gf_mul(a, b))


def sbox() -> tuple[np.ndarray, np.ndarray]:
    """(S, S^-1): the S-box of Section 2.1 computed from the GF inverse + affine map."""
    s = np.zeros(256, np.uint8)
    si = np.zeros(256, np.uint8)
    _load().oracle_sbox(_u8(s), _u8(si))
    return s, si


def key_expansion(key, bits: int) -> np.ndarray:
    """Round keys K of Eq. 1: (Nr+1) x 16 bytes (FIPS-197 KeyExpansion)."""
    k = _bytes_arr(key, bits // 8)
    w = np.zeros(16 * (nrounds(bits) + 1), np.uint8)
    _check(_load().oracle_key_expansion(_u8(k), bits, _u8(w)))
    return w.reshape(-1, 16)


def ecb(key, bits: int, data, decrypt: bool = False, nthreads: int | None = None) -> np.ndarray:
    """ECB encryption/decryption of independent 16-byte blocks (Section 3)."""
    k = _bytes_arr(key, bits // 8)
    d = _bytes_arr(data)
    if d.size % 16:
        raise ValueError("data length must be a multiple of 16")
    out = np.empty_like(d)
    _check(_load().oracle_ecb(_u8(k), bits, int(bool(decrypt)), _u8(d), _u8(out), d.size // 16,
                              _threads(nthreads)))
    return out


def ctr(key, bits: int, iv, data, kind: int = CTR_BE128, nthreads: int | None = None) -> np.ndarray:
    """CTR mode (Section 3): data XOR E_K(IV + i)."""
    k = _bytes_arr(key, bits // 8)
    v = _bytes_arr(iv, 16)
    d = _bytes_arr(data)
    if d.size % 16:
        raise ValueError("data length must be a multiple of 16")
    out = np.empty_like(d)
    _check(_load().oracle_ctr(_u8(k), bits, _u8(v), int(kind), _u8(d), _u8(out), d.size // 16,
                              _threads(nthreads)))
    return out


def cbc_decrypt(key, bits: int, iv, data, nthreads: int | None = None) -> np.ndarray:
    """CBC decryption (Section 3, Eq. 2)."""
    k = _bytes_arr(key, bits // 8)
    v = _bytes_arr(iv, 16)
    d = _bytes_arr(data)
    if d.size % 16:
        raise ValueError("data length must be a multiple of 16")
    out = np.empty_like(d)
    _check(_load().oracle_cbc_decrypt(_u8(k), bits, _u8(v), _u8(d), _u8(out), d.size // 16,
                                      _threads(nthreads)))
    return out


def counter_block(iv, i: int, kind: int = CTR_BE128) -> bytes:
    """The counter block the oracle encrypts for block index i."""
    v = _bytes_arr(iv, 16)
    out = np.zeros(16, np.uint8)
    _load().oracle_counter_block(_u8(v), int(kind), int(i), _u8(out))
    return out.tobytes()
