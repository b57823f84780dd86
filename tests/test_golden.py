"""Golden fixtures of the paper's SpMV workload (Section 3: a Lotkin matrix
with s % random zeros, b = A [1 .. n]^T, then y = A b), stored by
tests/golden/make_golden.py from the oracle and checked here both against
the oracle (regression) and against exact rational arithmetic (the pin)."""
import glob
import os
from fractions import Fraction

import numpy as np
import pytest

import exact
import oracle

GOLDEN = sorted(glob.glob(os.path.join(os.path.dirname(__file__), "golden", "lotkin_*.txt")))


def load(path):
    d = {"a": [], "b": [], "y_ordered": [], "y_exact": []}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        key, *rest = line.split()
        if key in ("p", "n", "seed"):
            d[key] = int(rest[0])
        elif key == "s":
            d[key] = float(rest[0])
        elif key == "rowptr":
            d[key] = np.array(rest, np.int64)
        elif key == "colidx":
            d[key] = np.array(rest, np.int32)
        else:
            d[key].append(np.array([int(w, 16) for w in rest], np.uint64))
    for k in ("a", "b", "y_ordered", "y_exact"):
        d[k] = np.stack(d[k])
    return d


def test_golden_present():
    assert len(GOLDEN) >= 2


@pytest.mark.parametrize("path", GOLDEN, ids=os.path.basename)
def test_lotkin_golden(path):
    g = load(path)
    p, n = g["p"], g["n"]
    rowptr, colidx = g["rowptr"], g["colidx"]
    # entries are RN(1/(i+j-1)) (1-based), first row ones
    for i in range(n):
        for k in range(rowptr[i], rowptr[i + 1]):
            j = int(colidx[k])
            want = Fraction(1) if i == 0 else exact.round_rne(Fraction(1, i + j + 1), p)
            assert exact.decode(g["a"][k], p).q == want
    A = exact.vec_decode(g["a"], p)
    # b = A [1..n]^T, exact sum rounded once
    for i in range(n):
        terms = [A[k].q * (int(colidx[k]) + 1) for k in range(rowptr[i], rowptr[i + 1])]
        assert exact.decode(g["b"][i], p).q == exact.round_rne(sum(terms, Fraction(0)), p)
    B = exact.vec_decode(g["b"], p)
    for i in range(n):
        y = exact.Val(Fraction(0))
        for k in range(rowptr[i], rowptr[i + 1]):
            y = exact.radd(y, exact.rmul(A[k], B[colidx[k]], p), p)
        assert exact.same(y, exact.decode(g["y_ordered"][i], p))
        terms = [A[k].q * B[colidx[k]].q for k in range(rowptr[i], rowptr[i + 1])]
        assert exact.same(exact.exact_sum(terms, p), exact.decode(g["y_exact"][i], p))
    # the oracle reproduces the stored vectors bit for bit
    y1, _ = oracle.spmv(p, oracle.ORDERED, rowptr, colidx, g["a"], g["b"])
    y2, _ = oracle.spmv(p, oracle.EXACT, rowptr, colidx, g["a"], g["b"])
    assert np.array_equal(y1, g["y_ordered"]) and np.array_equal(y2, g["y_exact"])
