"""The quotient-word estimate of the p-bit division, on the CPU: Moller and
Granlund's 2/1 division by an invariant integer ("Improved division by
invariant integers", IEEE Trans. Computers 60(2), 2011), in the 32-bit
form the device division uses (a reciprocal of the divisor's top word,
one widening multiply, a two-word add, one low multiply, at most two
corrections), must give exactly floor((u1 2^32 + u0) / d) and its
remainder for every normalised d (top bit set) and u1 < d.  The device
results themselves are compared with the oracle's correctly rounded
quotients by the GPU tests; this pins the estimate rule they rely on."""
import random

M32 = (1 << 32) - 1


def reciprocal(d):
    """v = floor((2^64 - 1) / d) - 2^32, a 32-bit word for d >= 2^31."""
    v = ((1 << 64) - 1) // d - (1 << 32)
    assert 0 <= v <= M32
    return v


def div2by1(u1, u0, d, v):
    q = v * u1 + ((u1 << 32) | u0)
    assert q < (1 << 64)  # the sum fits one 64-bit word because u1 < d
    q1 = ((q >> 32) + 1) & M32
    q0 = q & M32
    r = (u0 - q1 * d) & M32
    if r > q0:
        q1 = (q1 - 1) & M32
        r = (r + d) & M32
    if r >= d:
        q1 = (q1 + 1) & M32
        r -= d
    return q1, r


def check(u1, u0, d):
    q, r = div2by1(u1, u0, d, reciprocal(d))
    assert (q, r) == divmod((u1 << 32) | u0, d), (hex(u1), hex(u0), hex(d))


def test_boundaries():
    ds = [1 << 31, (1 << 31) + 1, (1 << 31) | 0x5555, 0xC0000000, M32 - 1, M32]
    for d in ds:
        for u1 in {0, 1, d >> 1, d - 2, d - 1}:
            for u0 in (0, 1, d - 1, d, 1 << 31, M32 - 1, M32):
                check(u1, u0 & M32, d)


def test_random_operands():
    rnd = random.Random(20111)
    for _ in range(200_000):
        d = rnd.randrange(1 << 31, 1 << 32)
        u1 = rnd.randrange(0, d)
        u0 = rnd.getrandbits(32)
        check(u1, u0, d)


def test_quotients_next_to_a_multiple():
    """Dividends one below, at and one above a multiple of d (the cases where
    a too-large first estimate needs both corrections)."""
    rnd = random.Random(7)
    for _ in range(50_000):
        d = rnd.randrange(1 << 31, 1 << 32)
        q = rnd.randrange(0, 1 << 32)
        for n in (q * d - 1, q * d, q * d + 1, q * d + d - 1):
            if 0 <= n < (d << 32):
                check(n >> 32, n & M32, d)
