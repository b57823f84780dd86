"""The windowed EXACT product's rounding rule, on the CPU.

At p >= 512 the default EXACT product keeps digit counters only for the top
p + g bits (g = 80 guard bits) of a row's sum below its largest term: the
radix-2^29 column sums of each term are added from the window's base digit
wb = floor((span + p - g) / 29) up, the columns below it (and the carry out
of the last of them) are dropped.  When a dropped column may be nonzero,
the row is rounded from the truncated sum only if the bits of its magnitude
between eb = 42 + bitlen(len) and the round bit are neither all zeros nor
all ones (and at least 8 of them); otherwise the row goes to the exact
kernel.  This restates those steps with the device's limb cutting, column
order and index arithmetic and checks that a row rounded from the window
always equals the exact sum rounded once, on rows built to need the rule:
wide exponent spans, sums that cancel far below their largest term, and
ties or near-ties made or broken by the dropped parts.  The shared rounding
of the window's integer is modelled as exact rounding to nearest-even; the
device kernel itself is compared with the oracle by the GPU tests."""
import os
import random
import re

import pytest

KR = 29
RMASK = (1 << KR) - 1
GUARD = 80  # the kernel's guard bits (kTopGuard; test_guard_matches_the_kernel)


def shape(W):
    NA = (32 * W + KR - 1) // KR
    NX = (32 * W + KR - 1 + KR - 1) // KR
    return NA, NX, NA + NX - 1


def top_cols(W):
    return (32 * W + 64 + GUARD) // KR + 6


def digits_cols(span, W):
    return (span + 64 * W + 64) // KR + 4


def limbs(m, n):
    return [(m >> (KR * i)) & RMASK for i in range(n)]


def rne(v, p):
    """v != 0 rounded to p bits: (sign, mantissa, exponent), v = m 2^e."""
    s, a = (1, -v) if v < 0 else (0, v)
    nb = a.bit_length()
    if nb <= p:
        return s, a << (p - nb), nb - p
    cut = nb - p
    q, rem, half = a >> cut, a & ((1 << cut) - 1), 1 << (cut - 1)
    if rem > half or (rem == half and q & 1):
        q += 1
        if q >> p:
            q >>= 1
            cut += 1
    return s, q, cut


def windowed_row(terms, W):
    """terms: (ma, ea, mx, ex, negative) with p-bit mantissas (top bit set).
    Returns (the rounded row as rne() gives it, exponents in units of
    2^(emin - 2p), 0 for +0, or None when the row goes to the exact kernel;
    whether a dropped column may have been nonzero)."""
    p = 32 * W
    NA, NX, NC = shape(W)
    emin = min(ea + ex for _, ea, _, ex, _ in terms)
    emax = max(ea + ex for _, ea, _, ex, _ in terms)
    span = emax - emin
    wb = (span + p - GUARD) // KR
    nd = digits_cols(span, W) - wb
    if nd > top_cols(W):
        return None, False
    c = [0] * nd
    errp = False
    for ma, ea, mx, ex, neg in terms:
        off = ea + ex - emin
        q, s = off // KR, off % KR
        qrel = q - wb
        kmin = -qrel if qrel < 0 else 0
        if kmin > NC:  # the whole term lies below the window
            errp = True
            continue
        al, xl = limbs(ma, NA), limbs(mx << s, NX)
        if kmin > 0 and not errp:
            la = next((i for i in range(NA) if al[i]), NA)
            lx = next((j for j in range(NX) if xl[j]), NX)
            errp = kmin > la + lx
        carry = 0
        for k in range(kmin, NC + 1):
            if k < NC:
                acc = sum(al[i] * xl[k - i] for i in range(NA) if 0 <= k - i < NX)
                assert acc < 1 << 64
                dd = (acc & RMASK) + carry
                carry = acc >> KR
            else:
                dd = carry
            assert 0 <= qrel + k < nd
            c[qrel + k] += -dd if neg else dd
    assert all(abs(v) < 1 << 63 for v in c)
    total = sum(v << (KR * d) for d, v in enumerate(c))
    if total == 0:
        return (None if errp else 0), errp
    mag = abs(total)
    if errp:
        eb = 42 + len(terms).bit_length()
        hi = mag.bit_length() - p - 1  # the round bit
        if hi - eb < 8:
            return None, errp
        bits = (mag >> eb) & ((1 << (hi - eb)) - 1)
        if bits == 0 or bits == (1 << (hi - eb)) - 1:
            return None, errp
    s, m, e = rne(total, p)
    return (s, m, e + KR * wb), errp


def exact_row(terms, W):
    emin = min(ea + ex for _, ea, _, ex, _ in terms)
    total = sum((-1 if neg else 1) * (ma * mx << (ea + ex - emin))
                for ma, ea, mx, ex, neg in terms)
    return 0 if total == 0 else rne(total, 32 * W)


def rows(W, seed):
    p = 32 * W
    rnd = random.Random(seed)
    top = 1 << (p - 1)

    def m():
        return top | rnd.getrandbits(p - 1)

    for _ in range(60):  # spans of a few to a few hundred bits, mixed signs
        n = rnd.randrange(1, 12)
        yield [(m(), rnd.randrange(-200, 200), m(), rnd.randrange(-100, 100), rnd.random() < 0.4)
               for _ in range(n)]
    for _ in range(60):  # a large pair that cancels, small terms under the window
        a, x = m(), m()
        d = rnd.randrange(0, 3 * p)
        row = [(a, 0, x, 0, False), (a, 0, x, 0, True),
               (m(), -d, m(), 0, rnd.random() < 0.5), (m(), -d - 40, m(), 0, False)]
        yield row + [(m(), -rnd.randrange(p, 3 * p), m(), 0, rnd.random() < 0.5)
                     for _ in range(rnd.randrange(0, 4))]
    for _ in range(80):  # ties and near-ties of a large term, decided by small terms
        # a * top = a 2^(p-1) has a as its p kept bits (ulp 2^(p-1)); top * top
        # 2^(-p) = 2^(p-2) is half an ulp, a tie; the terms top * top 2^(-k),
        # k >= p - 1, of either sign (one ulp and below, some of them under
        # the window) move the sum off the tie or back onto it
        a = m()
        big = (a, 0, top, 0, False)
        tie = (top, -p, top, 0, False)
        eps = [(top, -k, top, 0, rnd.random() < 0.5) for k in
               rnd.sample(range(p - 1, p + GUARD + 60), rnd.randrange(1, 4))]
        yield [big, tie] + eps
        yield [big] + eps
    for _ in range(40):  # many small terms just under the window, one large term
        a = m()
        row = [(a, 0, m(), 0, False)]
        row += [(m(), -(p + GUARD - 30 + rnd.randrange(0, 60)), m(), 0, rnd.random() < 0.5)
                for _ in range(rnd.randrange(20, 60))]
        yield row


@pytest.mark.parametrize("W", (16, 32))
def test_window_never_rounds_wrongly(W):
    decided = decided_dropping = routed = 0
    for row in rows(W, seed=100 + W):
        want = exact_row(row, W)
        got, dropping = windowed_row(row, W)
        if got is None:
            routed += 1
            continue
        decided += 1
        decided_dropping += dropping
        assert got == want, row
    # every outcome reached: rows rounded from the window with and without
    # dropped nonzero columns, and rows sent to the exact kernel
    assert decided - decided_dropping > 30 and decided_dropping > 30 and routed > 30


def test_dropped_part_is_below_the_error_bound():
    """What the window drops from one term is below 2^36 at the window's
    scale (the last dropped column is below 2^64 = 2^(29 + 35), those under it
    add less than one unit of it), so len terms drop less than
    2^(36 + bitlen(len)) <= 2^(42 + bitlen(len) - 6) = 2^(eb - 6)."""
    for W in (16, 32):
        NA, NX, NC = shape(W)
        col_max = min(NA, NX) * RMASK * RMASK
        assert col_max < 1 << 64
        dropped = sum(col_max << (KR * k) for k in range(NC)) >> (KR * NC)
        assert dropped < 1 << 36


def test_guard_matches_the_kernel():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = open(os.path.join(root, "paper_1411_2377_gb300", "csrc", "spmv.cu")).read()
    m = re.search(r"constexpr int kTopGuard = (\d+);", src)
    assert m and int(m.group(1)) == GUARD
