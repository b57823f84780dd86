"""Pins for the oracle's ILU(0) preconditioner and BiCGSTAB+ILU(0)
(Section 4's preconditioned rows; textbook forms).

Expectations come from mathematics: an exact-arithmetic replay of every
rounded step (tests/replay.py), the defining property of ILU(0) that L U
equals A on A's pattern, ILU(0) = LU where no fill is dropped (tridiagonal
and full patterns) so that M^{-1} solves A, one-iteration convergence of the
preconditioned solver when M = A, the known solution x = ones, and the
residual invariant.
"""
from fractions import Fraction

import numpy as np
import pytest

import exact
import oracle
import replay
from paper_1411_2377_gb300 import synth
from test_oracle_solvers import rand_system, rows_of, to_frac


def lu_product_rows(lu_rows, n):
    """(L U)_ij over all (i, j) as exact fractions (L unit lower)."""
    L = [[Fraction(0)] * n for _ in range(n)]
    U = [[Fraction(0)] * n for _ in range(n)]
    for i, row in enumerate(lu_rows):
        L[i][i] = Fraction(1)
        for c, v in row:
            if c < i:
                L[i][c] = v.q
            else:
                U[i][c] = v.q
    return [[sum(L[i][k] * U[k][j] for k in range(n)) for j in range(n)] for i in range(n)]


def decode_rows(rowptr, colidx, recs, p):
    V = exact.vec_decode(recs, p)
    return [[(int(colidx[k]), V[k]) for k in range(rowptr[i], rowptr[i + 1])]
            for i in range(len(rowptr) - 1)]


def tridiag(n, p):
    rows, cols, vals = [], [], []
    for i in range(n):
        for j, v in ((i - 1, -1.0 - 0.1 * i), (i, 4.0 + 0.25 * i), (i + 1, -1.5)):
            if 0 <= j < n:
                rows.append(i)
                cols.append(j)
                vals.append(v)
    rowptr = np.zeros(n + 1, np.int64)
    np.add.at(rowptr, np.array(rows) + 1, 1)
    return np.cumsum(rowptr), np.array(cols, np.int32), oracle.from_f64(p, np.array(vals))


@pytest.mark.parametrize("p", (128, 512))
def test_ilu0_and_apply_replay_bitwise(p):
    rowptr, colidx, vals, b = rand_system(7, p, 4, density=0.5)
    lu, st = oracle.ilu0(p, rowptr, colidx, vals)
    assert st == oracle.OK
    want = replay.ilu0(rows_of(rowptr, colidx, vals, p), p)
    got = decode_rows(rowptr, colidx, lu, p)
    assert [[(c, v.key()) for c, v in r] for r in got] == [[(c, v.key()) for c, v in r] for r in want]
    w, st = oracle.ilu0_apply(p, rowptr, colidx, lu, b)
    assert st == oracle.OK
    wr = replay.ilu0_apply(want, exact.vec_decode(b, p), p)
    assert [v.key() for v in wr] == [exact.decode(x, p).key() for x in w]


def test_ilu0_matches_a_on_its_pattern():
    """The defining property: (L U)_ij = a_ij for every stored (i, j), here
    to 2^-1000 relative at 1024 bits on the 2-D stencil (whose ILU(0) drops
    fill, so L U differs from A off the pattern)."""
    p = 1024
    rowptr, colidx, v64 = synth.stencil2d(5, seed=3)
    vals = oracle.from_f64(p, v64)
    n = len(rowptr) - 1
    lu, st = oracle.ilu0(p, rowptr, colidx, vals)
    assert st == oracle.OK
    P = lu_product_rows(decode_rows(rowptr, colidx, lu, p), n)
    A = decode_rows(rowptr, colidx, vals, p)
    off_pattern = 0
    for i in range(n):
        stored = {c for c, _ in A[i]}
        for c, v in A[i]:
            assert abs(P[i][c] - v.q) <= abs(v.q) / 2 ** 1000 + Fraction(1, 2 ** 1000)
        off_pattern += sum(1 for j in range(n) if j not in stored and P[i][j] != 0)
    assert off_pattern > 0  # fill was dropped


@pytest.mark.parametrize("kind", ("tridiagonal", "full"))
def test_ilu0_is_lu_without_fill(kind):
    """Where no fill is dropped ILU(0) is the LU factorization: M^{-1} r
    solves A w = r to 2^-1000 at 1024 bits."""
    p = 1024
    n = 9
    if kind == "tridiagonal":
        rowptr, colidx, vals = tridiag(n, p)
    else:
        rowptr = np.arange(0, n * n + 1, n, dtype=np.int64)
        colidx = np.tile(np.arange(n, dtype=np.int32), n)
        d = np.array([[(5.0 * n if i == j else 1.0 / (1 + i + 2 * j)) for j in range(n)]
                      for i in range(n)]).ravel()
        vals = oracle.from_f64(p, d)
    lu, st = oracle.ilu0(p, rowptr, colidx, vals)
    assert st == oracle.OK
    r = oracle.from_f64(p, np.arange(1.0, n + 1))
    w, st = oracle.ilu0_apply(p, rowptr, colidx, lu, r)
    A = decode_rows(rowptr, colidx, vals, p)
    W = to_frac(w, p)
    for i in range(n):
        Aw = sum(v.q * W[c] for c, v in A[i])
        assert abs(Aw - (i + 1)) < Fraction(1, 2 ** 1000) * (i + 1) * 10


def test_zero_pivot_is_reported():
    p = 128
    rowptr = np.array([0, 2, 4], np.int64)
    colidx = np.array([0, 1, 0, 1], np.int32)
    vals = oracle.from_f64(p, np.array([0.0, 1.0, 1.0, 1.0]))
    _, st = oracle.ilu0(p, rowptr, colidx, vals)
    assert st == oracle.ERR_DIVZERO
    b = oracle.from_f64(p, np.array([1.0, 1.0]))
    _, it, st, _ = oracle.bicgstab_ilu0(p, oracle.ORDERED, rowptr, colidx, vals, b,
                                        oracle.empty(p, 2), 1e-30, 0.0, 5)
    assert st == oracle.ERR_DIVZERO and it == 0


@pytest.mark.parametrize("mode", (oracle.ORDERED, oracle.EXACT))
def test_bicgstab_ilu0_replay_bitwise(mode):
    p, n = 128, 6
    rowptr, colidx, vals, b = rand_system(n, p, 8, density=0.5)
    rows = rows_of(rowptr, colidx, vals, p)
    X0 = exact.vec_decode(oracle.empty(p, n), p)
    for maxit in (1, 2, 4):
        x, it, st, hist = oracle.bicgstab_ilu0(p, mode, rowptr, colidx, vals, b,
                                               oracle.empty(p, n), 1e-300, 0.0, maxit)
        xr, itr, str_, hr = replay.bicgstab_ilu0(rows, exact.vec_decode(b, p), X0, p, mode,
                                                 1e-300, maxit)
        assert it == itr
        assert [v.key() for v in xr] == [exact.decode(r, p).key() for r in x]
        assert [v.key() for v in hr] == [exact.decode(r, p).key() for r in hist]


def test_preconditioner_equal_to_a_converges_in_one_step():
    p = 256
    n = 12
    rowptr, colidx, vals = tridiag(n, p)
    ones = oracle.from_f64(p, np.ones(n))
    b, _ = oracle.spmv(p, oracle.EXACT, rowptr, colidx, vals, ones)
    x, it, st, _ = oracle.bicgstab_ilu0(p, oracle.ORDERED, rowptr, colidx, vals, b,
                                        oracle.empty(p, n), 1e-60, 0.0, 10)
    assert st == oracle.OK and it == 1
    assert max(abs(v - 1) for v in to_frac(x, p)) < Fraction(1, 10 ** 70)


@pytest.mark.parametrize("mode", (oracle.ORDERED, oracle.EXACT))
def test_bicgstab_ilu0_known_solution_and_fewer_iterations(mode):
    """x = ones from b = A ones on the 2-D stencil, in fewer iterations than
    the unpreconditioned BiCGSTAB; the recursive r equals b - A x."""
    p = 256
    rowptr, colidx, v64 = synth.stencil2d(8, seed=1)
    vals = oracle.from_f64(p, v64)
    n = len(rowptr) - 1
    b, _ = oracle.spmv(p, oracle.EXACT, rowptr, colidx, vals, oracle.from_f64(p, np.ones(n)))
    x, it, st, hist = oracle.bicgstab_ilu0(p, mode, rowptr, colidx, vals, b, oracle.empty(p, n),
                                           1e-60, 0.0, 300)
    _, it0, st0, _ = oracle.bicgstab(p, mode, rowptr, colidx, vals, b, oracle.empty(p, n),
                                     1e-60, 0.0, 300)
    assert st == oracle.OK and st0 == oracle.OK
    assert it < it0
    assert max(abs(v - 1) for v in to_frac(x, p)) < Fraction(1, 10 ** 55)
    # before the attainable accuracy is reached, the recursive r is b - A x
    for k in (1, 2, 3):
        x, it, st, hist = oracle.bicgstab_ilu0(p, mode, rowptr, colidx, vals, b,
                                               oracle.empty(p, n), 1e-300, 0.0, k)
        res, _ = oracle.residual(p, rowptr, colidx, vals, b, x)
        true_rr = exact.decode(oracle.dot(p, res, res)[0], p).q
        rec_rr = exact.decode(hist[-1], p).q
        assert true_rr > 0
        assert abs(true_rr - rec_rr) / true_rr < Fraction(1, 2 ** 150), k


def test_reaching_maxit_is_noconv():
    """Tables 1-2's "NC": the iteration limit without convergence."""
    p = 512
    rowptr, colidx, v64 = synth.stencil2d(12, seed=6)
    n = len(rowptr) - 1
    vals = oracle.from_f64(p, v64)
    b = oracle.from_f64(p, np.linspace(-1.0, 2.0, n))
    x, it, st, hist = oracle.bicgstab_ilu0(p, oracle.EXACT, rowptr, colidx, vals, b,
                                           oracle.empty(p, n), 1e-200, 0.0, 3)
    assert st == oracle.ERR_NOCONV and it == 3 and len(hist) == 3
    assert exact.decode(hist[-1], p).q > 0
