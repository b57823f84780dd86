"""Pins for the oracle's CSR SpMV (ORDERED and EXACT), transpose, exact dot,
axpy and residual.  Expectations come from exact rational arithmetic
(tests/exact.py), dense-matrix brute force and invariants of the
definitions, never from the oracle itself."""
from fractions import Fraction

import numpy as np
import pytest

import exact
import oracle
from paper_1411_2377_gb300 import synth


def rand_recs(n, p, seed, zero_frac=0.1, emin=-4, emax=4):
    return synth.planes_to_records(synth.random_values(n, p, seed, zero_frac=zero_frac,
                                                       emin=emin, emax=emax))


def ordered_row(vals, cols, x, p):
    """Section 3's CSR row loop, step by step in exact arithmetic: y <- +0;
    skip zero factors; y <- RN(y + RN(a*x))."""
    y = exact.Val(Fraction(0))
    for a, c in zip(vals, cols):
        if a.q == 0 or x[c].q == 0:
            continue
        y = exact.radd(y, exact.rmul(a, x[c], p), p)
    return y


def exact_row(vals, cols, x, p):
    return exact.exact_sum([a.q * x[c].q for a, c in zip(vals, cols)], p)


CASES = [(128, 7, 0.5), (128, 9, 0.3), (256, 8, 0.4), (512, 6, 0.6), (1024, 5, 0.7),
         (2048, 6, 0.5), (4096, 5, 0.5), (8192, 4, 0.7)]


@pytest.mark.parametrize("p,n,density", CASES)
@pytest.mark.parametrize("seed", (1, 2))
def test_spmv_vs_fraction_brute_force(p, n, density, seed):
    rowptr, colidx = synth.small_random_csr(n, seed, density, empty_rows=1)
    nnz = int(rowptr[-1])
    vals = rand_recs(nnz, p, 10 + seed)
    x = rand_recs(n, p, 20 + seed)
    V, X = exact.vec_decode(vals, p), exact.vec_decode(x, p)
    for mode, fn in ((oracle.ORDERED, ordered_row), (oracle.EXACT, exact_row)):
        y, st = oracle.spmv(p, mode, rowptr, colidx, vals, x)
        assert st == oracle.OK
        for i in range(n):
            s, e = rowptr[i], rowptr[i + 1]
            want = fn(V[s:e], colidx[s:e], X, p)
            assert exact.same(want, exact.decode(y[i], p)), (mode, i)


@pytest.mark.parametrize("p", (128, 512))
def test_integer_matrix_closed_form(p):
    """Small integers: every partial sum is exact, so ORDERED = EXACT = the
    integer product A x, and b = A*ones is the row sum."""
    n = 12
    rowptr, colidx = synth.small_random_csr(n, 3, 0.5, diag=True)
    nnz = int(rowptr[-1])
    ivals = (synth.u64(3, 77, np.arange(nnz)) % np.uint64(41)).astype(np.int64) - 20
    ix = (synth.u64(3, 78, np.arange(n)) % np.uint64(31)).astype(np.int64) - 15
    vals = oracle.from_f64(p, ivals.astype(np.float64))
    x = oracle.from_f64(p, ix.astype(np.float64))
    dense = np.zeros((n, n), dtype=object)
    for i in range(n):
        for k in range(rowptr[i], rowptr[i + 1]):
            dense[i, colidx[k]] = int(ivals[k])
    want = dense.dot(np.array([int(v) for v in ix], dtype=object))
    ones = oracle.from_f64(p, np.ones(n))
    for mode in (oracle.ORDERED, oracle.EXACT):
        y, st = oracle.spmv(p, mode, rowptr, colidx, vals, x)
        assert [exact.decode(r, p).q for r in y] == list(want)
        b, _ = oracle.spmv(p, mode, rowptr, colidx, vals, ones)
        assert [exact.decode(r, p).q for r in b] == list(dense.sum(axis=1))


@pytest.mark.parametrize("p", (128, 256))
def test_explicit_zeros_are_skipped_exactly(p):
    """The zero fast path (Section 2): stored zeros change nothing, bitwise."""
    n = 40
    rowptr, colidx = synth.small_random_csr(n, 5, 0.3, empty_rows=2)
    nnz = int(rowptr[-1])
    vals = rand_recs(nnz, p, 31, zero_frac=0.2)
    x = rand_recs(n, p, 32, zero_frac=0.1)
    keep = np.array([exact.decode(v, p).q != 0 for v in vals])
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    rp2 = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rp2, rows[keep] + 1, 1)
    rp2 = np.cumsum(rp2)
    for mode in (oracle.ORDERED, oracle.EXACT):
        y1, _ = oracle.spmv(p, mode, rowptr, colidx, vals, x)
        y2, _ = oracle.spmv(p, mode, rp2, colidx[keep], vals[keep], x)
        assert np.array_equal(y1, y2)
        # empty rows give +0
        assert exact.decode(y1[0], p).key() == (0, False)


def test_empty_matrix():
    p = 128
    y, st = oracle.spmv(p, oracle.ORDERED, np.zeros(1, np.int64), np.zeros(0, np.int32),
                        np.zeros((0, 3), np.uint64), np.zeros((0, 3), np.uint64))
    assert st == oracle.OK and y.shape == (0, 3)


@pytest.mark.parametrize("p", (128, 1024))
def test_transpose_vs_dense(p):
    n = 15
    rowptr, colidx = synth.small_random_csr(n, 7, 0.3, empty_rows=1)
    nnz = int(rowptr[-1])
    vals = rand_recs(nnz, p, 41)
    trp, tci, tv = oracle.transpose(p, rowptr, colidx, vals)
    dense = {}
    for i in range(n):
        for k in range(rowptr[i], rowptr[i + 1]):
            dense[(i, int(colidx[k]))] = k
    k2 = 0
    for j in range(n):
        rows_j = sorted(i for (i, c) in dense if c == j)
        assert list(tci[trp[j]:trp[j + 1]]) == rows_j
        for i in rows_j:
            assert np.array_equal(tv[k2], vals[dense[(i, j)]])
            k2 += 1
    x = rand_recs(n, p, 42)
    V, X = exact.vec_decode(vals, p), exact.vec_decode(x, p)
    for mode, fn in ((oracle.ORDERED, ordered_row), (oracle.EXACT, exact_row)):
        y, _ = oracle.spmv_t(p, mode, rowptr, colidx, vals, x)
        for j in range(n):
            ks = [dense[(i, j)] for i in sorted(i for (i, c) in dense if c == j)]
            cols = [i for i in sorted(i for (i, c) in dense if c == j)]
            want = fn([V[k] for k in ks], cols, X, p)
            assert exact.same(want, exact.decode(y[j], p))


@pytest.mark.parametrize("p", (128, 256, 512, 1024, 2048, 8192))
def test_dot_vs_fractions(p):
    for seed, (emin, emax) in ((1, (-5, 5)), (2, (-300, 300))):
        n = 257
        x = rand_recs(n, p, 50 + seed, emin=emin, emax=emax)
        y = rand_recs(n, p, 60 + seed, emin=emin, emax=emax)
        r, st = oracle.dot(p, x, y)
        assert st == oracle.OK
        X, Y = exact.vec_decode(x, p), exact.vec_decode(y, p)
        want = exact.exact_sum([a.q * b.q for a, b in zip(X, Y)], p)
        assert exact.same(want, exact.decode(r, p))


@pytest.mark.parametrize("p", (128, 256, 8192))
def test_dot_cancellation_and_zeros(p):
    x = rand_recs(50, p, 71, zero_frac=0.0)
    y = rand_recs(50, p, 72, zero_frac=0.0)
    xx = np.concatenate([x, x])
    yneg = y.copy()
    yneg[:, 0] ^= np.uint64(1)  # flip signs
    yy = np.concatenate([y, yneg])
    r, _ = oracle.dot(p, xx, yy)
    assert exact.decode(r, p).key() == (0, False)  # exact zero is +0
    r, _ = oracle.dot(p, oracle.empty(p, 4), x[:4])
    assert exact.decode(r, p).key() == (0, False)
    r, _ = oracle.dot(p, x[:0], y[:0])
    assert exact.decode(r, p).key() == (0, False)
    # a sum that is exact at 2p bits but not at p bits rounds once
    big = exact.encode(exact.Val(Fraction(1)), p)
    tiny = exact.encode(exact.Val(Fraction(3, 2 ** (p + 1))), p)
    one = exact.encode(exact.Val(Fraction(1)), p)
    r, _ = oracle.dot(p, np.stack([big, tiny, tiny]), np.stack([one, one, one]))
    assert exact.decode(r, p).q == exact.round_rne(1 + Fraction(3, 2 ** p), p)


@pytest.mark.parametrize("p", (128, 512, 2048))
def test_span_cap(p):
    """Exponent spans up to the cap are summed exactly; beyond it both
    implementations report a span error (the row becomes +0)."""
    cap = oracle.SPAN_CAP
    one = exact.encode(exact.Val(Fraction(1)), p)
    for span, ok in ((cap - 1, True), (cap, True), (cap + 1, False)):
        small = exact.encode(exact.Val(-Fraction(3, 2) * Fraction(2) ** -span), p)
        x = np.stack([one, small, one])
        y = np.stack([one, one, one])
        r, st = oracle.dot(p, x, y)
        if ok:
            assert st == oracle.OK
            want = exact.round_rne(2 - Fraction(3, 2) * Fraction(2) ** -span, p)
            assert exact.decode(r, p).q == want
        else:
            assert st == oracle.ERR_SPAN and exact.decode(r, p).q == 0
        rowptr = np.array([0, 3, 4, 4], np.int64)
        colidx = np.array([0, 1, 2, 0], np.int32)
        vals = np.stack([one, one, one, one])
        yv, st = oracle.spmv(p, oracle.EXACT, rowptr, colidx, vals, x)
        assert (st == oracle.OK) == ok
        assert exact.decode(yv[1], p).q == 1  # the other row is unaffected


@pytest.mark.parametrize("p", (128, 1024, 4096))
def test_axpy_and_residual(p):
    n = 30
    x = rand_recs(n, p, 81)
    y = rand_recs(n, p, 82)
    alpha = rand_recs(1, p, 83, zero_frac=0.0)
    r, _ = oracle.axpy(p, alpha, x, y)
    A, X, Y = exact.decode(alpha[0], p), exact.vec_decode(x, p), exact.vec_decode(y, p)
    for i in range(n):
        assert exact.same(exact.radd(Y[i], exact.rmul(A, X[i], p), p), exact.decode(r[i], p))
    rowptr, colidx = synth.small_random_csr(n, 9, 0.2, diag=True)
    vals = rand_recs(int(rowptr[-1]), p, 84)
    res, st = oracle.residual(p, rowptr, colidx, vals, y, x)
    V = exact.vec_decode(vals, p)
    for i in range(n):
        s, e = rowptr[i], rowptr[i + 1]
        want = exact.exact_sum([Y[i].q] + [-V[k].q * X[colidx[k]].q for k in range(s, e)], p)
        assert exact.same(want, exact.decode(res[i], p))
    # with x = 0 the residual is b exactly
    res0, _ = oracle.residual(p, rowptr, colidx, vals, y, oracle.empty(p, n))
    for i in range(n):
        assert exact.decode(res0[i], p).q == Y[i].q


@pytest.mark.parametrize("mode", (oracle.ORDERED, oracle.EXACT))
def test_row_ranges_on_threads_match_one_call(mode):
    """Rows are independent: splitting them over host threads that write one
    shared result (the CPU baseline's all-cores form) gives the one-call
    result bit for bit."""
    from concurrent.futures import ThreadPoolExecutor

    p, n = 256, 3000
    rowptr, colidx = synth.spmv_pattern(n, seed=5)
    nnz = int(rowptr[-1])
    vals = rand_recs(nnz, p, 501, zero_frac=0.01, emin=-40, emax=40)
    x = rand_recs(n, p, 502, zero_frac=0.0, emin=-40, emax=40)
    want, st = oracle.spmv(p, mode, rowptr, colidx, vals, x)
    assert st == oracle.OK
    y = oracle.empty(p, n)
    cuts = [0, 1, 700, 701, 1900, n]
    with ThreadPoolExecutor(4) as ex:
        sts = list(ex.map(lambda r: oracle.spmv(p, mode, rowptr, colidx, vals, x, rows=r,
                                                out=y)[1], zip(cuts[:-1], cuts[1:])))
    assert all(s == oracle.OK for s in sts)
    assert np.array_equal(y, want)
    with pytest.raises(ValueError):
        oracle.spmv(p, mode, rowptr, colidx, vals, x, out=np.zeros((n, 3), np.uint64))
