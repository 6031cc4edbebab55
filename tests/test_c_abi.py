"""A plain C program (tests/c_abi_check.c) drives the C ABI directly: device
buffers from cudaMalloc, encrypt/decrypt round trips, error codes for bad
arguments; its ciphertexts are compared with the oracle."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_c_program_compiles_against_the_header(tmp_path):
    """The header is valid C and declares every call the program uses."""
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    obj = tmp_path / "c_abi_check.o"
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-c", "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(cuda, "include"), os.path.join(HERE, "c_abi_check.c"), "-o", str(obj)],
                   check=True)


@pytest.mark.gpu
def test_c_program_round_trip_and_oracle(gbaes, tmp_path):
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    lib = gbaes.library_path()
    exe = tmp_path / "c_abi_check"
    subprocess.run(["gcc", "-std=c11", "-O1", "-I", os.path.join(ROOT, "include"), "-I", os.path.join(cuda, "include"),
                    os.path.join(HERE, "c_abi_check.c"), lib, "-L", os.path.join(cuda, "lib64"), "-lcudart",
                    f"-Wl,-rpath,{os.path.dirname(lib)}", f"-Wl,-rpath,{os.path.join(cuda, 'lib64')}",
                    "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    lines = out.stdout.split("\n")
    assert "c abi ok" in out.stdout
    pt = np.array([(i * 131 + 7) & 0xFF for i in range(16)], np.uint8)
    for t, bits in enumerate((128, 192, 256)):
        key = bytes((i + 16 * t) & 0xFF for i in range(32))[: bits // 8]
        got = [l for l in lines if l.startswith(f"{bits} ")][0].split()[1]
        assert got == oracle.ecb(key, bits, pt).tobytes().hex()
