"""Pins for the oracle's ILU(0) preconditioner and BiCGSTAB+ILU(0)
(Section 4.2: ILU(0) as the left preconditioner K = LU; the right form is
kept as an option and pinned the same way).

Expectations come from mathematics: an exact-arithmetic replay of every
rounded step (tests/replay.py), the defining property of ILU(0) that L U
equals A on A's pattern, ILU(0) = LU where no fill is dropped (tridiagonal
and full patterns) so that K^{-1} solves A, one-iteration convergence of the
preconditioned solver when K = A, the known solution x = ones, the residual
invariants (r^ = K^{-1}(b - A x) for the left form, r = b - A x for the
right), and, for the left form, agreement at 1024 bits with the plain
BiCGSTAB run on the explicitly formed system (K^{-1} A) x = K^{-1} b.
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


@pytest.mark.parametrize("p", (128, 512, 2048, 8192))
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
    for side in ("left", "right"):
        _, it, st, _ = oracle.bicgstab_ilu0(p, oracle.ORDERED, rowptr, colidx, vals, b,
                                            oracle.empty(p, 2), 1e-30, 0.0, 5, side=side)
        assert st == oracle.ERR_DIVZERO and it == 0


@pytest.mark.parametrize("side", ("left", "right"))
@pytest.mark.parametrize("mode", (oracle.ORDERED, oracle.EXACT))
def test_bicgstab_ilu0_replay_bitwise(mode, side):
    p, n = 128, 6
    rowptr, colidx, vals, b = rand_system(n, p, 8, density=0.5)
    rows = rows_of(rowptr, colidx, vals, p)
    X0 = exact.vec_decode(oracle.empty(p, n), p)
    for maxit in (1, 2, 4):
        x, it, st, hist = oracle.bicgstab_ilu0(p, mode, rowptr, colidx, vals, b,
                                               oracle.empty(p, n), 1e-300, 0.0, maxit,
                                               side=side)
        xr, itr, str_, hr = replay.bicgstab_ilu0(rows, exact.vec_decode(b, p), X0, p, mode,
                                                 1e-300, maxit, side=side)
        assert it == itr
        assert [v.key() for v in xr] == [exact.decode(r, p).key() for r in x]
        assert [v.key() for v in hr] == [exact.decode(r, p).key() for r in hist]


@pytest.mark.parametrize("side", ("left", "right"))
def test_wide_build_bicgstab_ilu0_replay_bitwise(side):
    """The wide build (p = 2048) runs the same steps: every iterate of both
    forms equals the exact-arithmetic replay."""
    p, n = 2048, 5
    rowptr, colidx, vals, b = rand_system(n, p, 9, density=0.5)
    rows = rows_of(rowptr, colidx, vals, p)
    X0 = exact.vec_decode(oracle.empty(p, n), p)
    for maxit in (1, 3):
        x, it, st, hist = oracle.bicgstab_ilu0(p, oracle.ORDERED, rowptr, colidx, vals, b,
                                               oracle.empty(p, n), 1e-300, 0.0, maxit,
                                               side=side)
        xr, itr, str_, hr = replay.bicgstab_ilu0(rows, exact.vec_decode(b, p), X0, p,
                                                 oracle.ORDERED, 1e-300, maxit, side=side)
        assert it == itr
        assert [v.key() for v in xr] == [exact.decode(r, p).key() for r in x]
        assert [v.key() for v in hr] == [exact.decode(r, p).key() for r in hist]


@pytest.mark.parametrize("side", ("left", "right"))
def test_preconditioner_equal_to_a_converges_in_one_step(side):
    p = 256
    n = 12
    rowptr, colidx, vals = tridiag(n, p)
    ones = oracle.from_f64(p, np.ones(n))
    b, _ = oracle.spmv(p, oracle.EXACT, rowptr, colidx, vals, ones)
    x, it, st, _ = oracle.bicgstab_ilu0(p, oracle.ORDERED, rowptr, colidx, vals, b,
                                        oracle.empty(p, n), 1e-60, 0.0, 10, side=side)
    assert st == oracle.OK and it == 1
    assert max(abs(v - 1) for v in to_frac(x, p)) < Fraction(1, 10 ** 70)


@pytest.mark.parametrize("side", ("left", "right"))
@pytest.mark.parametrize("mode", (oracle.ORDERED, oracle.EXACT))
def test_bicgstab_ilu0_known_solution_and_fewer_iterations(mode, side):
    """x = ones from b = A ones on the 2-D stencil, in fewer iterations than
    the unpreconditioned BiCGSTAB; the recursive residual equals the one the
    form defines: K^{-1}(b - A x) (left) or b - A x (right)."""
    p = 256
    rowptr, colidx, v64 = synth.stencil2d(8, seed=1)
    vals = oracle.from_f64(p, v64)
    n = len(rowptr) - 1
    b, _ = oracle.spmv(p, oracle.EXACT, rowptr, colidx, vals, oracle.from_f64(p, np.ones(n)))
    x, it, st, hist = oracle.bicgstab_ilu0(p, mode, rowptr, colidx, vals, b, oracle.empty(p, n),
                                           1e-60, 0.0, 300, side=side)
    _, it0, st0, _ = oracle.bicgstab(p, mode, rowptr, colidx, vals, b, oracle.empty(p, n),
                                     1e-60, 0.0, 300)
    assert st == oracle.OK and st0 == oracle.OK
    assert it < it0
    assert max(abs(v - 1) for v in to_frac(x, p)) < Fraction(1, 10 ** 55)
    lu, _ = oracle.ilu0(p, rowptr, colidx, vals)
    # before the attainable accuracy is reached, the recursive residual is the true one
    for k in (1, 2, 3):
        x, it, st, hist = oracle.bicgstab_ilu0(p, mode, rowptr, colidx, vals, b,
                                               oracle.empty(p, n), 1e-300, 0.0, k, side=side)
        res, _ = oracle.residual(p, rowptr, colidx, vals, b, x)
        if side == "left":
            res, _ = oracle.ilu0_apply(p, rowptr, colidx, lu, res)
        true_rr = exact.decode(oracle.dot(p, res, res)[0], p).q
        rec_rr = exact.decode(hist[-1], p).q
        assert true_rr > 0
        assert abs(true_rr - rec_rr) / true_rr < Fraction(1, 2 ** 150), k


def test_left_form_is_bicgstab_on_the_preconditioned_system():
    """Section 4.2's left preconditioning: BiCGSTAB+ILU(0) equals the plain
    BiCGSTAB run on (K^{-1} A) x = K^{-1} b, with K = L U formed from the
    factor in exact rationals and K^{-1} A, K^{-1} b rounded once to 1024
    bits (a dense system).  The two round different operations, so they
    agree to about 2^-900, not bitwise; the right form, whose Krylov space
    is that of A K^{-1}, does not agree."""
    p, n = 1024, 6
    rowptr, colidx, vals, b = rand_system(n, p, 21, density=0.5)
    lu, st = oracle.ilu0(p, rowptr, colidx, vals)
    assert st == oracle.OK
    lu_rows = decode_rows(rowptr, colidx, lu, p)
    A = [[Fraction(0)] * n for _ in range(n)]
    for i, row in enumerate(decode_rows(rowptr, colidx, vals, p)):
        for c, v in row:
            A[i][c] = v.q
    K = lu_product_rows(lu_rows, n)
    Bq = [v.q for v in exact.vec_decode(b, p)]
    # K^{-1} [A | b] by Gauss-Jordan elimination in exact rationals
    M = [K[i][:] + A[i][:] + [Bq[i]] for i in range(n)]
    for c in range(n):
        piv = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[piv] = M[piv], M[c]
        f = M[c][c]
        M[c] = [v / f for v in M[c]]
        for r in range(n):
            if r != c and M[r][c] != 0:
                g = M[r][c]
                M[r] = [a - g * bb for a, bb in zip(M[r], M[c])]
    KA = [row[n:2 * n] for row in M]
    Kb = [row[2 * n] for row in M]
    rp = np.arange(0, n * n + 1, n, dtype=np.int64)
    ci = np.tile(np.arange(n, dtype=np.int32), n)
    enc = lambda q: exact.encode(exact.Val(exact.round_rne(q, p)), p)
    hat_vals = np.array([enc(KA[i][j]) for i in range(n) for j in range(n)], np.uint64)
    hat_b = np.array([enc(q) for q in Kb], np.uint64)
    for k in (1, 2, 3):
        xl, it, st, _ = oracle.bicgstab_ilu0(p, oracle.EXACT, rowptr, colidx, vals, b,
                                             oracle.empty(p, n), 1e-300, 0.0, k, side="left")
        xh, ith, sth, _ = oracle.bicgstab(p, oracle.EXACT, rp, ci, hat_vals, hat_b,
                                          oracle.empty(p, n), 1e-300, 0.0, k)
        xr, _, _, _ = oracle.bicgstab_ilu0(p, oracle.EXACT, rowptr, colidx, vals, b,
                                           oracle.empty(p, n), 1e-300, 0.0, k, side="right")
        assert it == ith == k
        XL, XH, XR = to_frac(xl, p), to_frac(xh, p), to_frac(xr, p)
        scale = max(abs(v) for v in XH)
        assert max(abs(a - c) for a, c in zip(XL, XH)) < scale / 2 ** 900, k
        assert max(abs(a - c) for a, c in zip(XR, XH)) > scale / 2 ** 100, k


@pytest.mark.parametrize("side", ("left", "right"))
def test_reaching_maxit_is_noconv(side):
    """Tables 1-2's "NC": the iteration limit without convergence."""
    p = 512
    rowptr, colidx, v64 = synth.stencil2d(12, seed=6)
    n = len(rowptr) - 1
    vals = oracle.from_f64(p, v64)
    b = oracle.from_f64(p, np.linspace(-1.0, 2.0, n))
    x, it, st, hist = oracle.bicgstab_ilu0(p, oracle.EXACT, rowptr, colidx, vals, b,
                                           oracle.empty(p, n), 1e-200, 0.0, 3, side=side)
    assert st == oracle.ERR_NOCONV and it == 3 and len(hist) == 3
    assert exact.decode(hist[-1], p).q > 0
