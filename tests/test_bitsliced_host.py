"""The bitsliced cipher (csrc/bitsliced.h) compiled for the CPU by a test
harness and compared with the oracle: the state split between two halves as in
the kernel (each half on its own host thread, the lane shuffle replaced by a
read of the other thread's plane), the byte-permute transposes, the S-box
circuit, ShiftRows across the halves, MixColumns / InvMixColumns and the key
planes with the affine constant and InvMixColumns folded in."""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1201_0398_gb300", "csrc")


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    exe = str(tmp_path_factory.mktemp("bs") / "bitsliced_check")
    subprocess.run(["g++", "-std=c++17", "-O1", "-pthread", "-Wno-unknown-pragmas", "-I", CSRC,
                    os.path.join(HERE, "bitsliced_check.cpp"), "-o", exe], check=True)
    return exe


@pytest.mark.parametrize("bits", (128, 192, 256))
def test_bitsliced_circuit_matches_oracle(gbaes, harness, bits):
    rng = np.random.default_rng(bits)
    for trial in range(6):
        key = rng.integers(0, 256, bits // 8, dtype=np.uint8).tobytes()
        if trial == 0:
            key = bytes(bits // 8)
        enc_rk, _ = gbaes.key_schedule(key, bits)
        data = rng.integers(0, 256, 512, dtype=np.uint8)
        for decrypt in (0, 1):
            payload = (np.array([bits, decrypt], "<i4").tobytes() + enc_rk.astype("<u4").tobytes()
                       + data.tobytes())
            out = subprocess.run([harness], input=payload, capture_output=True, check=True).stdout
            assert out == oracle.ecb(key, bits, data, decrypt=bool(decrypt)).tobytes()
