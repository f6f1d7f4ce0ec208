"""Write bitmap_digests.txt: prime count and SHA-256 of the oracle's dense
prime bitmap and of its (mask, value) list, for seeded functions too large
for the oracle to run beside a GPU test (Algorithm 3, Section 4.1, in the
oracle's bit-per-cube mode; the list in ascending rho as uint32 pairs, mask
then value, little-endian).

Calls only the oracle and the seeded input generator.  The packed state's
words, read as bytes in little-endian order, are the dense LSB-first bitmap
(cube rho at bit rho % 8 of byte rho // 8; bits past 3^n stay 0), so the
digest is taken over its first ceil(3^n / 8) bytes without a copy.

    python tests/golden/make_digests.py [n ...]     (default: 22 23 24)
"""
import hashlib
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2302_10083_gb300 import synth  # noqa: E402

OUT = os.path.join(HERE, "bitmap_digests.txt")

# (n, seed, p_on, p_dc): n = 22, 23 as the sampled GPU cases of those sizes;
# n = 24 the benchmark workload (ON ~ Bernoulli(0.85), seed 1, no don't-cares)
CASES = {22: (22, 2, 0.8, 0.05), 23: (23, 2, 0.8, 0.05), 24: (24, 1, 0.85, 0.0)}

POP = np.array([bin(i).count("1") for i in range(256)], dtype=np.uint8)


def digest(n, seed, p_on, p_dc):
    on, dc = synth.random_function(n, seed, p_on, p_dc)
    S = oracle.sweep_packed(n, on, dc if p_dc > 0 else None)
    A = (3 ** n + 7) // 8
    b = S.view(np.uint8)[:A]
    count = sum(int(POP[b[i: i + (1 << 26)]].sum(dtype=np.uint64)) for i in range(0, A, 1 << 26))
    h = hashlib.sha256(memoryview(b)).hexdigest()
    pairs = oracle.packed_pairs(n, S)
    assert len(pairs) == count
    return h, count, hashlib.sha256(memoryview(np.ascontiguousarray(pairs, dtype="<u4"))).hexdigest()


def main(ns):
    rows = {}
    if os.path.exists(OUT):
        for line in open(OUT):
            if line.strip() and not line.startswith("#"):
                rows[int(line.split()[0])] = line.rstrip("\n")
    for n in ns:
        n_, seed, p_on, p_dc = CASES[n]
        t0 = time.time()
        h, count, hl = digest(n_, seed, p_on, p_dc)
        rows[n] = f"{n_} {seed} {p_on} {p_dc} {count} {h} {hl}"
        print(f"n={n}: {count} primes, {h} {hl} ({time.time() - t0:.0f} s, {oracle.max_threads()} threads)",
              flush=True)
    with open(OUT, "w") as f:
        f.write("# Prime count, SHA-256 of the dense prime bitmap (ceil(3^n/8) bytes, bit rho\n"
                "# LSB-first) and SHA-256 of the (mask, value) list (uint32 pairs in ascending\n"
                "# rho, little-endian) of seeded functions, from the oracle's bit-per-cube sweep\n"
                "# (Algorithm 3, Section 4.1); written by make_digests.py in this folder.\n"
                "# Function: synth.random_function(n, seed, p_on, p_dc); p_dc = 0 means no DC table.\n"
                "# Columns: n seed p_on p_dc count bitmap_sha256 list_sha256\n")
        for n in sorted(rows):
            f.write(rows[n] + "\n")


if __name__ == "__main__":
    main([int(a) for a in sys.argv[1:]] or sorted(CASES))
