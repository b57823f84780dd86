"""Device p-bit arithmetic (mul/add/sub/div, conversions) vs the oracle,
bit for bit, through the C ABI (mp_ewise, mp_vec_from_f64)."""
from fractions import Fraction

import numpy as np
import pytest

import exact
import oracle
from gpu_util import assert_bitwise, need_gpu, rand_planes, recs

pytestmark = pytest.mark.gpu
PRECS = (128, 256, 512, 1024)
OPS = {"mul": (0, oracle.OP_MUL), "add": (1, oracle.OP_ADD), "sub": (2, oracle.OP_SUB),
       "div": (3, oracle.OP_DIV)}


@pytest.mark.parametrize("p", PRECS)
@pytest.mark.parametrize("op", list(OPS))
def test_random_pairs(p, op):
    mpk = need_gpu()
    n = 20000
    for seed, (lo, hi) in ((1, (-3, 3)), (2, (-300, 300)), (3, (-4 * p, 4 * p))):
        A = rand_planes(n, p, 100 * seed, zero_frac=0.03, emin=lo, emax=hi)
        B = rand_planes(n, p, 100 * seed + 1, zero_frac=0.03, emin=lo, emax=hi)
        if op == "div":  # no zero divisors here
            Bz = recs(B)
            nz = (Bz[:, 0].view(np.int64) >> 1) == oracle.EXP_ZERO
            B[:, nz] = rand_planes(int(nz.sum()), p, 7, zero_frac=0.0)
        a, b = mpk.Vec.from_planes(A, p), mpk.Vec.from_planes(B, p)
        out = mpk.ewise(OPS[op][0], a, b)
        want, st = oracle.ewise(p, OPS[op][1], recs(A), recs(B))
        assert st == oracle.OK
        assert_bitwise(out.planes(), want, f"{op} p={p} seed={seed}")


def _edge_records(p):
    h = 1 << (p - 1)
    full = (1 << p) - 1
    vals = []
    for M in (h, h + 1, 3 << (p - 2), full, full - 1, h + (1 << (p // 2))):
        for e in (0, 1, -1, p, -p, p + 1, p + 2, 2 * p + 5, 37):
            for neg in (False, True):
                v = Fraction(M) * Fraction(2) ** (e - p)
                vals.append(exact.encode(exact.Val(-v if neg else v), p))
    vals.append(exact.encode(exact.Val(Fraction(0)), p))
    vals.append(exact.encode(exact.Val(Fraction(0), negzero=True), p))
    return np.stack(vals)


@pytest.mark.parametrize("p", PRECS)
def test_all_pairs_of_edge_values(p):
    """Ties, carries out of the top, power-of-two binade edges, exponent gaps
    around p+1 and p+2, exact cancellation and signed zeros: every pair."""
    mpk = need_gpu()
    E = _edge_records(p)
    m = E.shape[0]
    A = np.repeat(E, m, axis=0)
    B = np.tile(E, (m, 1))
    a = mpk.Vec.from_planes(A.T, p)
    b = mpk.Vec.from_planes(B.T, p)
    for name, (code, ocode) in OPS.items():
        if name == "div":
            keep = (B[:, 0].view(np.int64) >> 1) != oracle.EXP_ZERO
            a2 = mpk.Vec.from_planes(A[keep].T, p)
            b2 = mpk.Vec.from_planes(B[keep].T, p)
            out = mpk.ewise(code, a2, b2)
            want, _ = oracle.ewise(p, ocode, A[keep], B[keep])
        else:
            out = mpk.ewise(code, a, b)
            want, _ = oracle.ewise(p, ocode, A, B)
        assert_bitwise(out.planes(), want, f"{name} edges p={p}")


@pytest.mark.parametrize("p", PRECS)
def test_cancellation_depths(p):
    """Differences of operands one binade apart or in the same binade whose
    leading bits cancel to every depth from 0 to p - 1 bits (the leading one
    landing in every bit of the top words and below them), with and without
    nonzero bits under the difference's leading one, and the same pairs
    added with opposite signs: add and sub against the oracle."""
    mpk = need_gpu()
    rng = np.random.default_rng(p + 17)
    h = 1 << (p - 1)
    A, B = [], []
    for j in range(p - 1):  # |M1 - M2| has its leading one at bit j
        for rep in range(2):
            low = int(rng.integers(0, 1 << min(j, 62))) if (rep and j) else 0
            diff = (1 << j) + (low % (1 << j) if j else 0)
            M2 = h + int(rng.integers(0, 1 << min(p - 2, 62)))
            M1 = M2 + diff
            if M1 >= 2 * h:
                M2 -= diff
                M1 = M2 + diff
            for e2 in (0, -1):  # same binade, or b one binade lower (d = 1)
                a = Fraction(M1) * Fraction(2) ** (3 - p)
                b = Fraction(M2) * Fraction(2) ** (3 + e2 - p)
                A.append(exact.encode(exact.Val(a), p))
                B.append(exact.encode(exact.Val(b), p))
                A.append(exact.encode(exact.Val(-a), p))
                B.append(exact.encode(exact.Val(-b), p))
    A, B = np.stack(A), np.stack(B)
    a = mpk.Vec.from_planes(A.T.copy(), p)
    b = mpk.Vec.from_planes(B.T.copy(), p)
    for name in ("sub", "add"):
        code, ocode = OPS[name]
        want, st = oracle.ewise(p, ocode, A, B)
        assert st == oracle.OK
        assert_bitwise(mpk.ewise(code, a, b).planes(), want, f"{name} cancellation p={p}")


def test_division_by_zero_is_reported():
    mpk = need_gpu()
    p = 256
    A = rand_planes(4, p, 3, zero_frac=0.0)
    B = oracle.empty(p, 4).T.copy()
    out = mpk.ewise(3, mpk.Vec.from_planes(A, p), mpk.Vec.from_planes(B, p), sync=False)
    with pytest.raises(mpk.MPError) as e:
        mpk.check()
    assert e.value.status == 9
    assert np.all((out.records()[:, 0].view(np.int64) >> 1) == oracle.EXP_ZERO)
    mpk.check()  # the status word was cleared


@pytest.mark.parametrize("p", PRECS)
def test_from_f64_exact(p):
    mpk = need_gpu()
    import torch

    d = np.concatenate([np.array([0.0, -0.0, 1.0, -2.5, 5e-324, -2.2250738585072014e-308,
                                  1.7976931348623157e308, 0.1]),
                        np.random.default_rng(0).standard_normal(5000) *
                        10.0 ** np.random.default_rng(1).integers(-300, 300, 5000)])
    v = mpk.Vec.from_f64(torch.from_numpy(d), p)
    assert_bitwise(v.planes(), oracle.from_f64(p, d), f"from_f64 p={p}")
    back = v.to_f64().cpu().numpy()
    assert np.array_equal(back.view(np.uint64), d.view(np.uint64))
