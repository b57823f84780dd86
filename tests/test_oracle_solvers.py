"""Pins for the oracle's BiCG and GPBiCG (Fig. 5, K = I), CGS and BiCGSTAB
(Section 4's other product-type methods, textbook forms).

Expectations come from mathematics, not from the oracle: finite termination
of BiCG-type methods in at most n steps in exact arithmetic (approached at
1024 bits), recovery of the known solution x = ones from b = A*ones
(Section 4's construction), one-step convergence on c*I, breakdown on a
system with (r~, A r0) = 0, the invariant that the recursively updated
residual equals b - A x, and an exact-arithmetic replay (tests/replay.py).
"""
from fractions import Fraction

import numpy as np
import pytest

import exact
import oracle
import replay
from paper_1411_2377_gb300 import synth

SOLVERS = {"bicg": oracle.bicg, "gpbicg": oracle.gpbicg, "cgs": oracle.cgs,
           "bicgstab": oracle.bicgstab}


def rand_system(n, p, seed, density=0.5, emin=-2, emax=2):
    """Random nonsymmetric, diagonally dominant n x n system with b = A*ones
    (b formed by the oracle's EXACT SpMV, i.e. correctly rounded)."""
    rowptr, colidx = synth.small_random_csr(n, seed, density, diag=True)
    nnz = int(rowptr[-1])
    vals = synth.planes_to_records(synth.random_values(nnz, p, seed + 1000, zero_frac=0.0,
                                                       emin=emin, emax=emax))
    # strengthen the diagonal: replace it by a value of larger exponent
    for i in range(n):
        for k in range(rowptr[i], rowptr[i + 1]):
            if colidx[k] == i:
                vals[k] = exact.encode(exact.Val(exact.round_rne(Fraction(3 * n + i, 1), p)), p)
    ones = oracle.from_f64(p, np.ones(n))
    b, _ = oracle.spmv(p, oracle.EXACT, rowptr, colidx, vals, ones)
    return rowptr, colidx, vals, b


def rows_of(rowptr, colidx, vals, p):
    V = exact.vec_decode(vals, p)
    return [[(int(colidx[k]), V[k]) for k in range(rowptr[i], rowptr[i + 1])]
            for i in range(len(rowptr) - 1)]


def to_frac(recs, p):
    return [exact.decode(r, p).q for r in recs]


@pytest.mark.parametrize("name", list(SOLVERS))
@pytest.mark.parametrize("mode", (oracle.ORDERED, oracle.EXACT))
def test_replay_every_iterate_bitwise(name, mode):
    p, n = 128, 5
    rowptr, colidx, vals, b = rand_system(n, p, 3)
    rows = rows_of(rowptr, colidx, vals, p)
    x0 = oracle.empty(p, n)
    X0 = exact.vec_decode(x0, p)
    for maxit in (1, 2, 3, 6):
        x, it, st, hist = SOLVERS[name](p, mode, rowptr, colidx, vals, b, x0, 1e-300, 0.0, maxit)
        B = exact.vec_decode(b, p)
        if name in ("gpbicg", "cgs", "bicgstab"):
            xr, itr, str_, hr = getattr(replay, name)(rows, B, X0, p, mode, 1e-300, maxit)
        else:
            trp, tci, tv = oracle.transpose(p, rowptr, colidx, vals)
            rows_t = rows_of(trp, tci, tv, p)
            xr, itr, str_, hr = replay.bicg(rows, rows_t, B, X0, p, mode, 1e-300, maxit)
        assert it == itr
        assert [v.key() for v in xr] == [exact.decode(r, p).key() for r in x]
        assert [v.key() for v in hr] == [exact.decode(r, p).key() for r in hist]


@pytest.mark.parametrize("name", list(SOLVERS))
@pytest.mark.parametrize("n,seed", ((4, 1), (6, 2), (8, 3)))
def test_finite_termination_at_1024_bits(name, n, seed):
    """In exact arithmetic both methods reach r = 0 in at most n steps; at
    1024 bits the residual drops below 1e-150 relative by then."""
    p = 1024
    rowptr, colidx, vals, b = rand_system(n, p, seed)
    x, it, st, _ = SOLVERS[name](p, oracle.ORDERED, rowptr, colidx, vals, b,
                                 oracle.empty(p, n), 1e-150, 0.0, 3 * n)
    assert st == oracle.OK
    assert it <= n
    err = max(abs(v - 1) for v in to_frac(x, p))
    assert err < Fraction(1, 10 ** 140)


@pytest.mark.parametrize("name", list(SOLVERS))
@pytest.mark.parametrize("mode", (oracle.ORDERED, oracle.EXACT))
def test_known_solution_ones(name, mode):
    """Section 4: b = A*ones in multiple precision; the solve recovers ones."""
    p = 256
    rowptr, colidx, vals64 = synth.stencil2d(6, seed=0)
    vals = oracle.from_f64(p, vals64)
    n = len(rowptr) - 1
    b, _ = oracle.spmv(p, oracle.EXACT, rowptr, colidx, vals, oracle.from_f64(p, np.ones(n)))
    x, it, st, hist = SOLVERS[name](p, mode, rowptr, colidx, vals, b, oracle.empty(p, n),
                                    1e-60, 0.0, 500)
    assert st == oracle.OK, (st, it)
    assert len(hist) == it
    err = max(abs(v - 1) for v in to_frac(x, p))
    assert err < Fraction(1, 10 ** 55)


@pytest.mark.parametrize("name", list(SOLVERS))
def test_recursive_residual_matches_true_residual(name):
    """Invariant of both methods: the updated r equals b - A x up to rounding.
    (The Fig. 5 GPBiCG updates as printed, z = zeta r + zeta z - alpha u and
    r = t - eta y - zeta u, violate it already at i = 1.)"""
    p = 256
    rowptr, colidx, vals, b = rand_system(12, p, 5, density=0.4)
    n = 12
    for k in (1, 2, 3, 4):
        x, it, st, hist = SOLVERS[name](p, oracle.EXACT, rowptr, colidx, vals, b,
                                        oracle.empty(p, n), 1e-300, 0.0, k)
        assert it == k
        res, _ = oracle.residual(p, rowptr, colidx, vals, b, x)
        true_rr, _ = oracle.dot(p, res, res)
        rec_rr = exact.decode(hist[-1], p).q
        tr = exact.decode(true_rr, p).q
        assert tr > 0
        assert abs(rec_rr - tr) / tr < Fraction(1, 2 ** 150), k


@pytest.mark.parametrize("name", list(SOLVERS))
@pytest.mark.parametrize("p", (128, 512))
def test_scaled_identity_converges_in_one_step(name, p):
    n = 7
    rowptr = np.arange(n + 1, dtype=np.int64)
    colidx = np.arange(n, dtype=np.int32)
    vals = oracle.from_f64(p, np.full(n, 3.0))
    b = oracle.from_f64(p, np.arange(1, n + 1, dtype=np.float64))
    x, it, st, _ = SOLVERS[name](p, oracle.ORDERED, rowptr, colidx, vals, b,
                                 oracle.empty(p, n), 1e-30, 0.0, 10)
    assert st == oracle.OK and it == 1
    for i, v in enumerate(to_frac(x, p)):
        want = Fraction(i + 1, 3)
        assert abs(v - want) <= 4 * want / 2 ** p


@pytest.mark.parametrize("name", list(SOLVERS))
def test_one_by_one(name):
    p = 128
    rowptr = np.array([0, 1], np.int64)
    colidx = np.array([0], np.int32)
    vals = oracle.from_f64(p, np.array([-7.0]))
    b = oracle.from_f64(p, np.array([2.0]))
    x, it, st, _ = SOLVERS[name](p, oracle.ORDERED, rowptr, colidx, vals, b,
                                 oracle.empty(p, 1), 1e-30, 0.0, 5)
    assert st == oracle.OK and it == 1
    v = to_frac(x, p)[0]
    assert abs(v + Fraction(2, 7)) <= Fraction(2, 7) * 4 / 2 ** p


@pytest.mark.parametrize("name", list(SOLVERS))
def test_breakdown_and_trivial_cases(name):
    p = 128
    solve = SOLVERS[name]
    # A = [[0,1],[1,0]], b = e1: (r~, A r0) = 0, the first divisor vanishes
    rowptr = np.array([0, 1, 2], np.int64)
    colidx = np.array([1, 0], np.int32)
    vals = oracle.from_f64(p, np.array([1.0, 1.0]))
    b = oracle.from_f64(p, np.array([1.0, 0.0]))
    x, it, st, _ = solve(p, oracle.ORDERED, rowptr, colidx, vals, b, oracle.empty(p, 2),
                         1e-30, 0.0, 10)
    assert st == oracle.ERR_BREAKDOWN and it == 0
    assert all(v == 0 for v in to_frac(x, p))
    # b = 0: (r0, r0) = 0 meets the stopping rule before any iteration
    x, it, st, _ = solve(p, oracle.ORDERED, rowptr, colidx, vals, oracle.empty(p, 2),
                         oracle.empty(p, 2), 1e-30, 0.0, 10)
    assert st == oracle.OK and it == 0
    # not enough iterations: NC, x is the last iterate
    rowptr, colidx, vals, b = rand_system(10, p, 9)
    x, it, st, hist = solve(p, oracle.ORDERED, rowptr, colidx, vals, b, oracle.empty(p, 10),
                            1e-30, 0.0, 2)
    assert st == oracle.ERR_NOCONV and it == 2 and len(hist) == 2


def test_printed_gpbicg_updates_break_the_residual_invariant():
    """Documents the reading of Fig. 5's GPBiCG: with the updates exactly as
    printed, the recursive r departs from b - A x at the first iteration,
    while with z = zeta r + eta z - alpha u and r = t - eta y - zeta A t it
    does not (plain float64, independent of the oracle)."""
    rowptr, colidx, v64 = synth.stencil2d(4, seed=1)
    n = len(rowptr) - 1
    A = np.zeros((n, n))
    for i in range(n):
        A[i, colidx[rowptr[i]:rowptr[i + 1]]] = v64[rowptr[i]:rowptr[i + 1]]
    b = A @ np.ones(n)

    def run(printed, iters=3):
        x = np.zeros(n)
        r = b.copy()
        rt = r.copy()
        u = np.zeros(n); z = np.zeros(n); s = np.zeros(n)
        beta = eta = 0.0
        rho = rt @ r
        gaps = []
        for i in range(1, iters + 1):
            if i == 1:
                p_ = r.copy(); q = A @ p_; alpha = rho / (rt @ q)
                t = r - alpha * q; v = A @ t; y = alpha * q - r
                zeta = (v @ t) / (v @ v); eta = 0.0
            else:
                beta = (rho / rho_prev) * (alpha / zeta)
                w = v + beta * q; p_ = r + beta * (p_ - u); q = A @ p_
                alpha = rho / (rt @ q); s = t - r; t = r - alpha * q; v = A @ t
                y = s - alpha * (w - q)
                m1, m2, m3, m4, m5 = y @ y, v @ t, y @ t, v @ y, v @ v
                tau = m5 * m1 - m4 * m4
                zeta = (m1 * m2 - m3 * m4) / tau; eta = (m5 * m3 - m4 * m2) / tau
            u = zeta * q + eta * (s + beta * u)
            z = zeta * r + (zeta if printed else eta) * z - alpha * u
            x = x + alpha * p_ + z
            r = t - eta * y - zeta * (u if printed else v)
            rho_prev, rho = rho, rt @ r
            gaps.append(np.linalg.norm(r - (b - A @ x)) / np.linalg.norm(b))
        return gaps

    assert max(run(printed=False)) < 1e-12
    assert run(printed=True)[0] > 1e-3


@pytest.mark.parametrize("name", list(SOLVERS))
def test_wide_build_replay_and_finite_termination(name):
    """The wide build's solvers: the exact-arithmetic replay of every iterate
    at 2048 bits (n = 4, two iterations), and termination in at most n
    steps with the residual below 1e-300 relative at 4096 bits."""
    p, n = 2048, 4
    rowptr, colidx, vals, b = rand_system(n, p, 5)
    rows = rows_of(rowptr, colidx, vals, p)
    x0 = oracle.empty(p, n)
    X0 = exact.vec_decode(x0, p)
    B = exact.vec_decode(b, p)
    x, it, st, hist = SOLVERS[name](p, oracle.ORDERED, rowptr, colidx, vals, b, x0, 1e-300, 0.0,
                                    2)
    if name == "bicg":
        trp, tci, tv = oracle.transpose(p, rowptr, colidx, vals)
        xr, itr, _, hr = replay.bicg(rows, rows_of(trp, tci, tv, p), B, X0, p, oracle.ORDERED,
                                     1e-300, 2)
    else:
        xr, itr, _, hr = getattr(replay, name)(rows, B, X0, p, oracle.ORDERED, 1e-300, 2)
    assert it == itr
    assert [v.key() for v in xr] == [exact.decode(r, p).key() for r in x]
    assert [v.key() for v in hr] == [exact.decode(r, p).key() for r in hist]
    p = 4096
    rowptr, colidx, vals, b = rand_system(n, p, 6)
    x, it, st, _ = SOLVERS[name](p, oracle.ORDERED, rowptr, colidx, vals, b,
                                 oracle.empty(p, n), 1e-300, 0.0, 3 * n)
    assert st == oracle.OK and it <= n
    assert max(abs(v - 1) for v in to_frac(x, p)) < Fraction(1, 10 ** 290)
