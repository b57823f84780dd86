"""Writes tests/golden/lotkin_*.txt using only the oracle (oracle/).

The workload is Section 3's: the n x n Lotkin matrix (first row all ones,
a_ij = 1/(i+j-1) below it), with s % of its entries set to zero and dropped
from the sparse storage, entries rounded to p bits; b = A [1 2 ... n]^T in
multiple precision; then y = A b.  The zero pattern uses the shared seeded
generator (paper_1411_2377_gb300.synth), drawn once per (i, j).

Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1411_2377_gb300 import synth  # noqa: E402

CASES = ((128, 8, 40.0, 7), (256, 6, 25.0, 8))


def lotkin_sparse(n, s_percent, seed):
    """Pattern and the (numerator, denominator) of each stored entry."""
    return synth.lotkin_pattern(n, s_percent, seed)


def hexrec(rec):
    return " ".join(f"{int(w):016x}" for w in rec)


def write_case(p, n, s, seed):
    rowptr, colidx, num, den = lotkin_sparse(n, s, seed)
    vals, st = oracle.ewise(p, oracle.OP_DIV, oracle.from_f64(p, num), oracle.from_f64(p, den))
    assert st == oracle.OK
    xv = oracle.from_f64(p, np.arange(1, n + 1, dtype=np.float64))
    b, st = oracle.spmv(p, oracle.EXACT, rowptr, colidx, vals, xv)
    assert st == oracle.OK
    y_ord, _ = oracle.spmv(p, oracle.ORDERED, rowptr, colidx, vals, b)
    y_ex, _ = oracle.spmv(p, oracle.EXACT, rowptr, colidx, vals, b)
    path = os.path.join(HERE, f"lotkin_p{p}_n{n}.txt")
    with open(path, "w") as f:
        f.write(f"# Section 3 workload: sparse Lotkin matrix, p={p} bits, n={n}, s={s}% zeros "
                f"(seed {seed}).\n")
        f.write("# Written by tests/golden/make_golden.py from the oracle; records are\n")
        f.write("# [exp*2+sign, limb0 .. limbL-1] in hex.\n")
        f.write(f"p {p}\nn {n}\ns {s}\nseed {seed}\n")
        f.write("rowptr " + " ".join(map(str, rowptr)) + "\n")
        f.write("colidx " + " ".join(map(str, colidx)) + "\n")
        for k in range(len(colidx)):
            f.write("a " + hexrec(vals[k]) + "\n")
        for name, vec in (("b", b), ("y_ordered", y_ord), ("y_exact", y_ex)):
            for i in range(n):
                f.write(f"{name} " + hexrec(vec[i]) + "\n")
    return path


if __name__ == "__main__":
    for case in CASES:
        print(write_case(*case))
