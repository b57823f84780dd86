"""Pins for the oracle's correctly rounded p-bit arithmetic (Section 2: MPFR
round-to-nearest).  Every expectation comes from exact rational arithmetic
(tests/exact.py) or from mpmath's independent correctly rounded kernels,
never from the oracle itself."""
from fractions import Fraction

import numpy as np
import pytest

import exact
import oracle
from paper_1411_2377_gb300 import synth

PRECS = (128, 256, 512, 1024)
WIDE = (2048, 4096, 8192)  # the wide build (the paper's solves of Tables 1-2 reach 8192 bits)
OPS = {
    oracle.OP_MUL: exact.rmul,
    oracle.OP_ADD: exact.radd,
    oracle.OP_SUB: exact.rsub,
    oracle.OP_DIV: exact.rdiv,
}


def rec_from_mantissa(p, M, e, neg=False):
    v = Fraction(M) * Fraction(2) ** (e - p)
    return exact.encode(exact.Val(-v if neg else v), p)


def check_ewise(p, op, a, b):
    r, st = oracle.ewise(p, op, a, b)
    bad = []
    for i in range(a.shape[0]):
        A, B = exact.decode(a[i], p), exact.decode(b[i], p)
        if op == oracle.OP_DIV and B.q == 0:
            continue
        E = OPS[op](A, B, p)
        R = exact.decode(r[i], p)
        if not exact.same(E, R):
            bad.append((i, A, B, E, R))
    assert not bad, bad[:3]
    return r, st


@pytest.mark.parametrize("p", PRECS)
@pytest.mark.parametrize("op", list(OPS))
def test_random_pairs_vs_fractions(p, op):
    n = 600
    for seed, (emin, emax) in ((11, (-3, 3)), (12, (-2 * p, 2 * p))):
        a = synth.planes_to_records(synth.random_values(n, p, seed + op, zero_frac=0.05,
                                                        emin=emin, emax=emax))
        b = synth.planes_to_records(synth.random_values(n, p, seed + 100 + op, zero_frac=0.05,
                                                        emin=emin, emax=emax))
        check_ewise(p, op, a, b)


@pytest.mark.parametrize("p", WIDE)
@pytest.mark.parametrize("op", list(OPS))
def test_wide_random_pairs_vs_fractions(p, op):
    """The wide build at 2048-8192 bits against exact rationals."""
    n = 60
    for seed, (emin, emax) in ((31, (-3, 3)), (32, (-2 * p, 2 * p))):
        a = synth.planes_to_records(synth.random_values(n, p, seed + op, zero_frac=0.05,
                                                        emin=emin, emax=emax))
        b = synth.planes_to_records(synth.random_values(n, p, seed + 100 + op, zero_frac=0.05,
                                                        emin=emin, emax=emax))
        check_ewise(p, op, a, b)


def test_narrow_build_rejects_wide_precisions():
    """libmpo.so holds 1024-bit mantissas at most and says so."""
    a = oracle.empty(2048, 1)
    assert oracle._load(0).mpo_dot(2048, 1, oracle._p(a, oracle._u64p), oracle._p(a, oracle._u64p),
                                   oracle._p(a, oracle._u64p)) == oracle.ERR_PREC


@pytest.mark.parametrize("p", PRECS + (2048,))
def test_random_pairs_vs_mpmath(p):
    libmp = pytest.importorskip("mpmath.libmp")
    n = 3000 if p <= 1024 else 500
    a = synth.planes_to_records(synth.random_values(n, p, 21, zero_frac=0.0, emin=-70, emax=70))
    b = synth.planes_to_records(synth.random_values(n, p, 22, zero_frac=0.0, emin=-70, emax=70))

    def to_mpf(rec):
        v = exact.decode(rec, p).q
        return libmp.from_rational(v.numerator, v.denominator, p + 64, "n")

    fns = {oracle.OP_MUL: libmp.mpf_mul, oracle.OP_ADD: libmp.mpf_add,
           oracle.OP_SUB: libmp.mpf_sub, oracle.OP_DIV: libmp.mpf_div}
    A = [to_mpf(r) for r in a]
    B = [to_mpf(r) for r in b]
    for op, fn in fns.items():
        r, _ = oracle.ewise(p, op, a, b)
        for i in range(n):
            want = fn(A[i], B[i], p, "n")
            got = exact.decode(r[i], p).q
            sign, man, ex, _ = want
            assert (-1) ** sign * Fraction(man) * Fraction(2) ** ex == got, (op, i)


@pytest.mark.parametrize("p", PRECS + WIDE)
def test_product_ties_both_parities(p):
    """Products whose exact value lies exactly halfway between two p-bit
    numbers: Ma = 2^(p-1) + k (k odd and even) times Mb = 3 * 2^(p-2)."""
    h = 1 << (p - 1)
    a, b, ties = [], [], 0
    for k in range(1, 41):
        a.append(rec_from_mantissa(p, h + k, 1))
        b.append(rec_from_mantissa(p, 3 << (p - 2), 1, neg=(k % 3 == 0)))
        exact_prod = Fraction(h + k) * (3 << (p - 2))
        # the scaled product has p-1 dropped bits; a tie leaves exactly 2^(p-2)
        if exact_prod.numerator % (1 << (p - 1)) == (1 << (p - 2)):
            ties += 1
    assert ties >= 20
    check_ewise(p, oracle.OP_MUL, np.stack(a), np.stack(b))


@pytest.mark.parametrize("p", PRECS + WIDE)
def test_sum_ties_carry_and_binade_edges(p):
    """x + y where y sits at or just below half an ulp of x, including the
    power-of-two x whose lower neighbour is only half an ulp away, and sums
    that carry out of the top bit after rounding."""
    h = 1 << (p - 1)
    full = (1 << p) - 1
    cases = []
    for d in (p - 1, p, p + 1, p + 2, p + 3, 2 * p, 50 * p):
        for Mx in (h, h + 1, full):
            for My in (h, h + 1, 3 << (p - 2), full):
                for neg in (False, True):
                    cases.append((rec_from_mantissa(p, Mx, 7), rec_from_mantissa(p, My, 7 - d, neg)))
    a = np.stack([c[0] for c in cases])
    b = np.stack([c[1] for c in cases])
    check_ewise(p, oracle.OP_ADD, a, b)
    check_ewise(p, oracle.OP_ADD, b, a)
    check_ewise(p, oracle.OP_SUB, a, b)
    # the carry-out case: (2^p - 1) 2^-p + 2^-(p+1) rounds up to exactly 1
    r, _ = oracle.ewise(p, oracle.OP_ADD, rec_from_mantissa(p, full, 0)[None],
                        rec_from_mantissa(p, h, -p)[None])
    assert exact.decode(r[0], p).q == 1


@pytest.mark.parametrize("p", (128, 1024, 8192))
def test_signed_zero_table(p):
    """IEEE/MPFR signed-zero rules in round-to-nearest."""
    pz = exact.encode(exact.Val(Fraction(0)), p)
    nz = exact.encode(exact.Val(Fraction(0), negzero=True), p)
    one = exact.encode(exact.Val(Fraction(1)), p)
    mone = exact.encode(exact.Val(Fraction(-1)), p)
    vals = [pz, nz, one, mone]
    a = np.stack([x for x in vals for _ in vals])
    b = np.stack([y for _ in vals for y in vals])
    for op in (oracle.OP_MUL, oracle.OP_ADD, oracle.OP_SUB):
        check_ewise(p, op, a, b)
    check_ewise(p, oracle.OP_DIV, a, b)
    # exact cancellation is +0, (-0)+(-0) is -0
    r, _ = oracle.ewise(p, oracle.OP_ADD, np.stack([one, nz]), np.stack([mone, nz]))
    assert exact.decode(r[0], p).key() == (0, False)
    assert exact.decode(r[1], p).key() == (0, True)


@pytest.mark.parametrize("p", PRECS + WIDE)
def test_division_exact_quotients_and_zero_divisor(p):
    ints = [1, 2, 3, 5, 6, 7, 10, 12, 48, 96, 1 << 40, 3 << 60]
    a = np.stack([exact.encode(exact.Val(Fraction(x * y)), p) for x in ints for y in ints])
    b = np.stack([exact.encode(exact.Val(Fraction(y)), p) for x in ints for y in ints])
    r, st = check_ewise(p, oracle.OP_DIV, a, b)
    assert st == oracle.OK
    for i, x in enumerate(x for x in ints for _ in ints):
        assert exact.decode(r[i], p).q == x
    # x / 0 is reported, never silently rounded
    _, st = oracle.ewise(p, oracle.OP_DIV, a[:1], oracle.empty(p, 1))
    assert st == oracle.ERR_DIVZERO


@pytest.mark.parametrize("p", PRECS + WIDE)
def test_compare(p):
    vals = [Fraction(-3), Fraction(-1, 3), Fraction(0), Fraction(1, 7), Fraction(2), Fraction(1 << 200)]
    recs = [exact.encode(exact.Val(exact.round_rne(v, p)), p) for v in vals]
    for i, x in enumerate(recs):
        for j, y in enumerate(recs):
            assert oracle.cmp(p, x, y) == (i > j) - (i < j)
    nz = exact.encode(exact.Val(Fraction(0), negzero=True), p)
    assert oracle.cmp(p, nz, recs[2]) == 0


@pytest.mark.parametrize("p", PRECS + WIDE)
def test_from_f64_is_exact(p):
    d = np.array([0.0, -0.0, 1.0, -1.5, 0.1, 1e300, -1e-300, 5e-324, -2.2250738585072014e-308,
                  np.nextafter(1.0, 2.0), 2.0 ** 1023 * 1.9999999999999998, 123456.789])
    r = oracle.from_f64(p, d)
    for i, x in enumerate(d):
        v = exact.decode(r[i], p)
        assert v.q == Fraction(float(x))
        assert v.negzero == (x == 0 and np.signbit(x))
    back = oracle.to_f64(p, r)
    assert np.array_equal(back.view(np.uint64), d.view(np.uint64))
