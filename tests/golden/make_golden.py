"""Writes the stored oracle fixtures in this folder.  Calls only ``oracle`` (and ``workloads`` for
the seeded inputs); nothing here comes from the CUDA library.

    python tests/golden/make_golden.py

Fixture ``bernoulli64_dmax16.txt``: the dense 64^3 Bernoulli(0.02) grids of seeds 0..4 with
dmax = 16 (clamp 256), transformed by the oracle's Eq. 1 brute force.  One line per seed:
seed, obstacle count, sha256 of the int32 little-endian field, and the count of each distinct
value.  The test beside it recomputes the field on whatever machine runs the suite, so the x86 and
Arm builds of the oracle and the generators are held to the same bytes.
"""
import hashlib
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
import workloads as W  # noqa: E402


def field_line(seed):
    occ = W.bernoulli_grid(seed, (64, 64, 64), 0.02)
    D = O.edt_naive(occ, 16)
    vals, counts = np.unique(D, return_counts=True)
    digest = hashlib.sha256(D.astype("<i4").tobytes()).hexdigest()
    hist = " ".join(f"{v}:{c}" for v, c in zip(vals.tolist(), counts.tolist()))
    return f"{seed} {int(occ.sum())} {digest} {hist}"


def main():
    lines = ["# seed obstacles sha256(int32 LE field) value:count ...  (Eq. 1, dmax 16, 64^3, p 0.02)"]
    lines += [field_line(s) for s in range(5)]
    with open(os.path.join(HERE, "bernoulli64_dmax16.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
