"""Exact rational model of p-bit round-to-nearest-even arithmetic.

Used only to pin the oracle: values are ``fractions.Fraction`` objects, every
operation is computed exactly and then rounded by :func:`round_rne`, which is
written from the definition of round-to-nearest, ties-to-even (MPFR's RN,
Section 2 of the paper) using rational comparisons, independently of the
oracle's bit-level C code.  Records use the interchange layout of the test
harness: ``[exp*2 + sign, limb_0, ..., limb_{L-1}]`` with value
``(-1)^sign * M * 2^(exp-p)``, ``2^(p-1) <= M < 2^p``, zero flagged by
``exp == EXP_ZERO``.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

EXP_ZERO = -(1 << 61)
MASK64 = (1 << 64) - 1


class Val:
    """A signed p-bit value: exact rational ``q`` plus the sign of zero."""

    __slots__ = ("q", "negzero")

    def __init__(self, q: Fraction, negzero: bool = False):
        self.q = Fraction(q)
        self.negzero = bool(negzero) and self.q == 0

    def __repr__(self):
        return f"Val({self.q}{', -0' if self.negzero else ''})"

    def key(self):
        return (self.q, self.negzero)


def decode(rec, p: int) -> Val:
    L = p // 64
    head = int(rec[0])
    if head >= 1 << 63:
        head -= 1 << 64
    sign = head & 1
    e = (head - sign) // 2
    M = 0
    for k in range(L):
        M |= int(rec[1 + k]) << (64 * k)
    if e == EXP_ZERO:
        assert M == 0
        return Val(Fraction(0), negzero=bool(sign))
    assert M >> (p - 1) == 1, "unnormalised record"
    q = Fraction(M) * Fraction(2) ** (e - p)
    return Val(-q if sign else q)


def encode(v: Val, p: int):
    """Record of a value that is exactly representable with p bits."""
    L = p // 64
    rec = np.zeros(L + 1, dtype=np.uint64)
    if v.q == 0:
        rec[0] = np.uint64((EXP_ZERO * 2 + (1 if v.negzero else 0)) & MASK64)
        return rec
    sign = 1 if v.q < 0 else 0
    a = abs(v.q)
    e = _exponent(a)
    M = a * Fraction(2) ** (p - e)
    assert M.denominator == 1 and (1 << (p - 1)) <= M.numerator < (1 << p), "not representable"
    M = M.numerator
    rec[0] = np.uint64((e * 2 + sign) & MASK64)
    for k in range(L):
        rec[1 + k] = np.uint64((M >> (64 * k)) & MASK64)
    return rec


def _exponent(a: Fraction) -> int:
    """The e with 2^(e-1) <= a < 2^e, for a > 0."""
    e = a.numerator.bit_length() - a.denominator.bit_length()
    while Fraction(2) ** (e - 1) > a:
        e -= 1
    while Fraction(2) ** e <= a:
        e += 1
    return e


def round_rne(q: Fraction, p: int) -> Fraction:
    """Nearest p-bit binary value to q; on a tie, the one with an even mantissa."""
    if q == 0:
        return Fraction(0)
    a = abs(q)
    e = _exponent(a)
    scaled = a * Fraction(2) ** (p - e)  # in [2^(p-1), 2^p)
    lo = scaled.numerator // scaled.denominator
    frac = scaled - lo
    if frac > Fraction(1, 2) or (frac == Fraction(1, 2) and lo % 2 == 1):
        lo += 1
    r = Fraction(lo) * Fraction(2) ** (e - p)
    return -r if q < 0 else r


def rmul(a: Val, b: Val, p: int) -> Val:
    if a.q == 0 or b.q == 0:
        sa = a.negzero if a.q == 0 else a.q < 0
        sb = b.negzero if b.q == 0 else b.q < 0
        return Val(Fraction(0), negzero=(sa != sb))
    return Val(round_rne(a.q * b.q, p))


def radd(a: Val, b: Val, p: int) -> Val:
    if a.q == 0 and b.q == 0:
        return Val(Fraction(0), negzero=a.negzero and b.negzero)
    s = a.q + b.q
    if s == 0:
        return Val(Fraction(0))
    return Val(round_rne(s, p))


def neg(a: Val) -> Val:
    if a.q == 0:
        return Val(Fraction(0), negzero=not a.negzero)
    return Val(-a.q)


def rsub(a: Val, b: Val, p: int) -> Val:
    return radd(a, neg(b), p)


def rdiv(a: Val, b: Val, p: int) -> Val:
    assert b.q != 0
    if a.q == 0:
        sb = b.q < 0
        return Val(Fraction(0), negzero=(a.negzero != sb))
    return Val(round_rne(a.q / b.q, p))


def exact_sum(terms, p: int) -> Val:
    """RN of the exact sum of rationals; an exact zero (or no terms) is +0."""
    s = sum(terms, Fraction(0))
    return Val(round_rne(s, p)) if s != 0 else Val(Fraction(0))


def vec_decode(recs, p):
    return [decode(r, p) for r in np.asarray(recs).reshape(-1, p // 64 + 1)]


def vec_encode(vals, p):
    return np.stack([encode(v, p) for v in vals]) if vals else np.zeros((0, p // 64 + 1), np.uint64)


def same(a: Val, b: Val) -> bool:
    return a.q == b.q and a.negzero == b.negzero
