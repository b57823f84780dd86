"""The short column product's rounding rule, on the CPU.

From p = 512 the products take radix-2^29 column sums of the two mantissas
and skip every column below K0 = min(floor((p - 97)/29), KLO - 3) (KLO: the
first digit that reaches the product's word W - 1).  What is left is a
lower bound T of the exact product P; the bits of T from digit K0 + 3 up to
the round bit (the guard region) decide the rounding unless they are all
ones (the skipped part could carry into the round bit) or all zeros with
the round bit set (the sticky bit is unknown), and then the full column
product is used.  This restates those steps with the device's word sizes
(29-bit digits from 64-bit column sums, 32-bit words, the same index
arithmetic) and checks that the rule never rounds differently from the
exact product rounded to nearest-even, on random operands and on operands
built so that P has long runs of ones or zeros right under the round bit.
The device products themselves are compared with the oracle's by the GPU
tests; this pins the argument they rely on."""
import random

import pytest

KR = 29
RMASK = (1 << KR) - 1
M32 = (1 << 32) - 1


def shape(W):
    NA = (32 * W + KR - 1) // KR
    WLO = W - 1
    KLO = (32 * WLO) // KR
    K0 = min((32 * W - 97) // KR, KLO - 3)
    return NA, 2 * NA, WLO, KLO, 32 * WLO - KR * KLO, K0, K0 + 3


def digits(ma, mb, W, kfrom):
    """Columns k >= kfrom summed into 64-bit accumulators, one carry pass:
    digit k for kfrom <= k < ND - 1 and the final carry as digit ND - 1."""
    NA, ND = shape(W)[:2]
    al = [(ma >> (KR * i)) & RMASK for i in range(NA)]
    bl = [(mb >> (KR * i)) & RMASK for i in range(NA)]
    D, carry = {}, 0
    for k in range(kfrom, ND - 1):
        acc = carry + sum(al[i] * bl[k - i] for i in range(max(0, k - NA + 1), min(k, NA - 1) + 1))
        assert acc < 1 << 64
        carry = acc >> KR
        D[k] = acc & RMASK
    assert carry < 1 << 32
    D[ND - 1] = carry
    return D


def words(D, W):
    """Words W-1 .. 2W-1 of the product reassembled from the digits, with the
    device's 32-bit shifts."""
    ND, WLO = shape(W)[1], shape(W)[2]
    T = []
    for j in range(W + 1):
        bit = 32 * (WLO + j)
        kk, rr = bit // KR, bit % KR
        v = D[kk] >> rr
        if kk + 1 < ND:
            v |= (D[kk + 1] << (KR - rr)) & M32
        if 2 * KR - rr < 32 and kk + 2 < ND:
            v |= (D[kk + 2] << (2 * KR - rr)) & M32
        T.append(v & M32)
    return T


def finish(T, W, rb, sticky, p):
    sh = 1 - (T[W] >> 31)
    m = 0
    for k in range(W):
        w = ((T[k + 1] << sh) | (T[k] >> (32 - sh))) & M32 if sh else T[k + 1]
        m |= w << (32 * k)
    e = -sh
    if rb and (sticky or m & 1):
        m += 1
        if m == 1 << p:
            m, e = 1 << (p - 1), e + 1
    return m, e


def short_product(ma, mb, W):
    """(mantissa, exponent offset) or None when the rule takes the full product."""
    p = 32 * W
    _, _, _, KLO, R0, K0, KG = shape(W)
    D = digits(ma, mb, W, K0)
    T = words(D, W)
    sh = 1 - (T[W] >> 31)
    g = (T[0] << sh) & M32
    rb = g >> 31
    below = (g << 1) & M32
    any_, all_ = below, below | ((1 << (1 + sh)) - 1)
    for k in range(KG, KLO):
        any_ |= D[k]
        all_ &= D[k] | (~RMASK & M32)
    if R0 > 0:
        lowm = (1 << R0) - 1
        any_ |= D[KLO] & lowm
        all_ &= D[KLO] | (~lowm & M32)
    if all_ == M32 or (rb and any_ == 0):
        return None
    return finish(T, W, rb, any_ != 0, p)


def full_product(ma, mb, W):
    """The full column product: every column, the digits below word W-1
    only as the sticky bit."""
    p = 32 * W
    _, _, _, KLO, R0, _, _ = shape(W)
    D = digits(ma, mb, W, 0)
    st = 0
    for k in range(KLO):
        st |= D[k]
    if R0 > 0:
        st |= D[KLO] & ((1 << R0) - 1)
    T = words(D, W)
    sh = 1 - (T[W] >> 31)
    g = (T[0] << sh) & M32
    st |= (g << 1) & M32
    return finish(T, W, g >> 31, st != 0, p)


def exact_rne(ma, mb, p):
    """RN(ma * mb) to p bits: (mantissa, exponent offset) in the same
    convention (offset -1 when the exact product has 2p - 1 bits)."""
    P = ma * mb
    e = 0 if P >> (2 * p - 1) else -1
    cut = p + e
    q, rem, half = P >> cut, P & ((1 << cut) - 1), 1 << (cut - 1)
    if rem > half or (rem == half and q & 1):
        q += 1
        if q == 1 << p:
            q, e = 1 << (p - 1), e + 1
    return q, e


def operands(p, seed):
    rnd = random.Random(seed)
    top = 1 << (p - 1)
    for _ in range(300):
        yield top | rnd.getrandbits(p - 1), top | rnd.getrandbits(p - 1)
    for j in range(0, p - 1, 7):
        # (2^(p-1) + 2^j)(2^(p-1) - 2^j) = 2^(2p-2) - 2^(2j): ones from bit 2j up
        yield top + (1 << j), top - (1 << j)
        yield top + (1 << j), top + (1 << j)
        yield top, top | rnd.getrandbits(p - 1) >> j << j       # exact: zeros below
        yield (1 << p) - 1, top | (rnd.getrandbits(p - 1) >> j << j)  # runs of ones
    for _ in range(100):
        # a product whose bits under the round bit are a tie or one ulp off it
        a = top | rnd.getrandbits(p - 1)
        k = rnd.randrange(1, 40)
        b = top | (rnd.getrandbits(p - 1 - k) << k)
        yield a, b
        yield a | 1, (b >> k) << k | ((1 << k) - 1)


@pytest.mark.parametrize("W", (16, 32))
def test_short_rule_never_rounds_wrongly(W):
    p = 32 * W
    taken = fallback = 0
    for ma, mb in operands(p, seed=W):
        want = exact_rne(ma, mb, p)
        assert full_product(ma, mb, W) == want
        got = short_product(ma, mb, W)
        if got is None:
            fallback += 1
        else:
            taken += 1
            assert got == want, (hex(ma), hex(mb))
    assert taken > 300 and fallback > 0  # both paths reached


def test_skipped_columns_stay_below_the_guard_region():
    """The part the short product drops, the columns k < K0 (each below
    NA 2^58), sums to less than 2^(29 K0 + 64), which is below the guard
    region's lowest bit 29 (K0 + 3) because 3 * 29 > 64; so the dropped part
    reaches the guard region only as a carry.  At least 36 guard bits lie
    under the lowest possible round bit (p - 2) at p = 512 and 1024."""
    for W in (16, 32):
        p = 32 * W
        NA, _, _, KLO, _, K0, KG = shape(W)
        assert K0 > 0 and KG <= KLO
        cmax = NA * RMASK * RMASK
        bound = sum(cmax << (KR * k) for k in range(K0))
        assert bound < 1 << (KR * K0 + 64) <= 1 << (KR * KG)
        round_bit = p - 2  # lowest position of the round bit (a 2p-1-bit product)
        assert round_bit - KR * KG >= 36
