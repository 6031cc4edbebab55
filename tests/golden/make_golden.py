"""Writes ecb_kat.json: known-answer vectors for AES-ECB computed by the oracle only.

Each vector is one (key, 4-block plaintext, ciphertext) triple.  The values come
from the CPU oracle (FIPS-197 AES, Section 2.1) on seeded inputs; the not-gpu test
``test_golden_kat_file_matches_library_and_oracle`` re-derives every ciphertext
with the installed ``cryptography`` package, so the stored values are pinned to a
source outside this repository.  The GPU tests use the file on machines that have
no ``cryptography`` package.

Run: python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
import oracle  # noqa: E402


def main():
    rng = np.random.default_rng(20120102)
    vectors = []
    for bits in (128, 192, 256):
        keys = [bytes(bits // 8), bytes([0xFF]) * (bits // 8), bytes(range(bits // 8))]
        keys += [rng.integers(0, 256, bits // 8, dtype=np.uint8).tobytes() for _ in range(3)]
        for i, key in enumerate(keys):
            pt = bytes(64) if i == 0 else rng.integers(0, 256, 64, dtype=np.uint8).tobytes()
            ct = oracle.ecb(key, bits, pt).tobytes()
            vectors.append({"bits": bits, "key": key.hex(), "plaintext": pt.hex(), "ciphertext": ct.hex()})
    out = {
        "what": "AES-ECB known answers (FIPS-197 cipher; Section 2.1), written by tests/golden/make_golden.py "
                "from the CPU oracle; checked against the cryptography package by tests/test_oracle.py",
        "vectors": vectors,
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "ecb_kat.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(f"wrote {len(vectors)} vectors to {path}")


if __name__ == "__main__":
    main()
