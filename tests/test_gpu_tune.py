"""Launch configurations and the autotuner: every configuration of a
matrix's products (threads per block; ORDERED operand staging; EXACT word
digits or radix-2^29 column sums) gives the oracle's result bit for bit, the
tuner keeps one of them, and the on-disk cache reproduces it without timing
again."""
import json

import numpy as np
import pytest

import oracle
from gpu_util import assert_bitwise, need_gpu, rand_planes, random_csr, recs

pytestmark = pytest.mark.gpu
MODES = (("ordered", oracle.ORDERED), ("exact", oracle.EXACT))


@pytest.mark.parametrize("p", (128, 256, 512, 1024))
def test_every_configuration_matches_the_oracle(p):
    mpk = need_gpu()
    n = 2113 if p <= 256 else 803
    rowptr, colidx = random_csr(n, seed=p + 1, mean_len=9, max_len=120, empty_every=13)
    V = rand_planes(len(colidx), p, 31, zero_frac=0.05, emin=-30, emax=30)
    X = rand_planes(n, p, 32, zero_frac=0.05, emin=-30, emax=30)
    A = mpk.CSR(rowptr, colidx, V, p, transpose=True)
    x = mpk.Vec.from_planes(X, p)
    for name, m in MODES:
        want, st = oracle.spmv(p, m, rowptr, colidx, recs(V), recs(X))
        want_t, _ = oracle.spmv_t(p, m, rowptr, colidx, recs(V), recs(X))
        for tpb, carve in ((32, -1), (64, 25), (128, 50), (256, 75), (-1, -1)):
            for v in (0, 1, 2, 3, 6, 7, 9, 11, 15, 18, 19, 27, -1):
                A.set_config(name, tpb, v, carve)
                got = A.get_config(name)
                if tpb > 0:
                    assert got["threads_per_block"] == tpb
                if carve > 0:
                    assert got["carveout"] == carve
                if v >= 0:
                    assert got["variant"] & 2 == v & 2  # the product form asked for
                    if name == "ordered":
                        capped = 4 if (v & 4 and (tpb if tpb > 0 else 128) <= 128) else 0
                        assert got["variant"] == (v & 3 if p <= 512 else v & 2) | capped | (v & 8)
                    elif v & 2:
                        assert got["variant"] == (v if p >= 512 else v & ~16)
                what = f"{name} p={p} tpb={tpb} variant={v} carveout={carve}"
                assert_bitwise(mpk.spmv(A, x, mode=name).planes(), want, what)
                assert_bitwise(mpk.spmv_t(A, x, mode=name).planes(), want_t, "T " + what)


def test_bad_configuration_is_rejected():
    mpk = need_gpu()
    rowptr, colidx = random_csr(64, seed=2)
    A = mpk.CSR(rowptr, colidx, np.ones(len(colidx)), 128)
    for args in (("ordered", 96, -1, -1), ("ordered", 128, 32, -1), ("exact", 512, -1, -1),
                 ("exact", 64, -2, -1), ("exact", 64, 0, 101)):
        with pytest.raises(mpk.MPError):
            A.set_config(*args)
    assert A.get_config("ordered") == {"threads_per_block": 128, "variant": 5, "carveout": -1}
    assert A.get_config("exact") == {"threads_per_block": 128, "variant": 1, "carveout": 50}


@pytest.mark.parametrize("p", (128, 1024))
def test_tuner_and_cache(p, tmp_path):
    mpk = need_gpu()
    from paper_1411_2377_gb300 import tune

    n = 20000
    rowptr, colidx = random_csr(n, seed=7, mean_len=8, max_len=64, band=300)
    V = rand_planes(len(colidx), p, 41, emin=-10, emax=10)
    X = rand_planes(n, p, 42, emin=-10, emax=10)
    A = mpk.CSR(rowptr, colidx, V, p)
    x = mpk.Vec.from_planes(X, p)
    cache = str(tmp_path / "tune.json")
    first = tune.autotune(A, reps=2, cache=cache)
    for name, m in MODES:
        r = first[name]
        assert not r["cached"] and r["ms"] > 0
        assert r["threads_per_block"] in (32, 64, 128, 256)
        assert A.get_config(name)["threads_per_block"] == r["threads_per_block"]
        base = {"ordered": ((0, 1, 2, 3, 5, 7) if p <= 512 else (0, 2, 6)),
                "exact": (0, 1, 2, 3, 6, 7) + ((18, 19, 22, 23) if p >= 512 else ())}[name]
        assert r["variant"] in set(base) | {v | 8 for v in base}
        want, _ = oracle.spmv(p, m, rowptr, colidx, recs(V), recs(X))
        assert_bitwise(mpk.spmv(A, x, mode=name).planes(), want, f"tuned {name} p={p}")
    assert len(json.load(open(cache))) == 2
    B = mpk.CSR(rowptr, colidx, V, p)
    again = tune.autotune(B, reps=2, cache=cache)
    for name, _ in MODES:
        assert again[name]["cached"]
        assert B.get_config(name) == A.get_config(name)


@pytest.mark.parametrize("p", (128, 256, 512, 1024))
@pytest.mark.parametrize("variant", (0, 2, 3, 6, 7, 19, 23, 27))
def test_exact_variants_on_hard_rows(p, variant):
    """Both EXACT product forms, and the windowed form (bit 4, p >= 512), on
    rows whose spans sit around the per-thread window (in it, just beyond it:
    the warp-per-row path), beyond the span cap, with exact cancellation (the
    windowed form then hands the row to the exact path), and in the residual
    with its b term."""
    mpk = need_gpu()
    from paper_1411_2377_gb300 import synth

    n = 300
    rowptr, colidx = random_csr(n, seed=p + variant, mean_len=12, max_len=40)
    V = rand_planes(len(colidx), p, 51, zero_frac=0.02, emin=-3, emax=3)
    X = rand_planes(n, p, 52, zero_frac=0.02, emin=-3, emax=3)
    Vr, Xr = recs(V), recs(X)
    # push one entry of some rows down by s bits: spans s + O(10)
    zero_head = np.uint64((oracle.EXP_ZERO * 2) & ((1 << 64) - 1))

    def nonzeros(r):
        return [k for k in range(rowptr[r], rowptr[r + 1])
                if (Vr[k, 0] >> np.uint64(1)) != zero_head >> np.uint64(1)]

    rows = [r for r in range(n) if len(nonzeros(r)) >= 3][:8]
    assert len(rows) == 8
    # push one entry of a row down by s bits: spans s + O(10) around the
    # per-thread window (512 bits), and one beyond the span cap
    for r, shift in zip(rows, (400, 490, 505, 530, 700, 2000, oracle.SPAN_CAP + 50)):
        k = nonzeros(r)[0]
        Vr[k, 0] = np.int64(Vr[k, 0].view(np.int64) - 2 * shift).view(np.uint64)
    # last row: a, -a against equal x values, the rest stored zeros -> +0
    r = rows[7]
    k = rowptr[r]
    Xr[colidx[k + 1]] = Xr[colidx[k]]
    Vr[k] = Vr[nonzeros(r)[0]]
    Vr[k + 1] = Vr[k]
    Vr[k + 1, 0] ^= np.uint64(1)
    Vr[k + 2:rowptr[r + 1]] = 0
    Vr[k + 2:rowptr[r + 1], 0] = zero_head
    A = mpk.CSR(rowptr, colidx, synth.records_to_planes(Vr), p, transpose=True)
    A.set_config("exact", 128, variant, 50)
    x = mpk.Vec.from_planes(synth.records_to_planes(Xr), p)
    want, st = oracle.spmv(p, oracle.EXACT, rowptr, colidx, Vr, Xr)
    assert st == oracle.ERR_SPAN
    y = mpk.spmv(A, x, mode="exact", sync=False)
    with pytest.raises(mpk.MPError):
        mpk.check()
    assert_bitwise(y.planes(), want, f"exact variant={variant} p={p}")
    B = rand_planes(n, p, 53, zero_frac=0.1, emin=-300, emax=3)
    r = mpk.residual(A, mpk.Vec.from_planes(B, p), x, sync=False)
    with pytest.raises(mpk.MPError):
        mpk.check()
    want_r, _ = oracle.residual(p, rowptr, colidx, Vr, recs(B), Xr)
    assert_bitwise(r.planes(), want_r, f"residual variant={variant} p={p}")


def _mantissa_planes(ms, p, exps, signs):
    """Planes of values (-1)^s * M * 2^(e-p) from integer mantissas M."""
    L = p // 64
    out = np.zeros((L + 1, len(ms)), np.uint64)
    for k, (m, e, sg) in enumerate(zip(ms, exps, signs)):
        out[0, k] = np.uint64((2 * e + sg) & ((1 << 64) - 1))
        for l in range(L):
            out[1 + l, k] = np.uint64((m >> (64 * l)) & ((1 << 64) - 1))
    return out


@pytest.mark.parametrize("p", (128, 256, 512, 1024))
def test_ordered_products_round_ties_to_even(p):
    """y_i = RN(a_i x_i) on a diagonal matrix whose products are exact ties
    (M_a = 2^(p-1) + 2^i, M_x = 2^(p-1) + 2^(p-2-i): the dropped bits are
    exactly one half) and near-ties, in both product forms."""
    mpk = need_gpu()
    ia = [0, 1, 2, 5, 31, 32, 33, p // 2 - 1, p // 2, p - 3]
    ma, mx = [], []
    for i in ia:
        a, x = (1 << (p - 1)) + (1 << i), (1 << (p - 1)) + (1 << (p - 2 - i))
        ma += [a, a, a + 1]
        mx += [x, x + (1 << 0), x]
    n = len(ma)
    rowptr = np.arange(n + 1, dtype=np.int64)
    colidx = np.arange(n, dtype=np.int32)
    V = _mantissa_planes(ma, p, [3] * n, [k % 2 for k in range(n)])
    X = _mantissa_planes(mx, p, [-7] * n, [0] * n)
    A = mpk.CSR(rowptr, colidx, V, p)
    x = mpk.Vec.from_planes(X, p)
    want, _ = oracle.spmv(p, oracle.ORDERED, rowptr, colidx, recs(V), recs(X))
    for v in (0, 2):
        A.set_config("ordered", 128, v, -1)
        assert_bitwise(mpk.spmv(A, x, mode="ordered").planes(), want, f"ties variant={v} p={p}")


@pytest.mark.parametrize("p", (512, 1024))
def test_windowed_exact_on_cancelling_and_integer_rows(p):
    """The windowed EXACT form against the oracle where its window cannot
    decide alone: near and exact cancellation of the largest terms, and
    integer-valued rows whose skipped columns are provably zero."""
    mpk = need_gpu()
    from paper_1411_2377_gb300 import synth

    n = 400
    rowptr, colidx = random_csr(n, seed=p + 77, mean_len=10, max_len=30)
    V = rand_planes(len(colidx), p, 71, zero_frac=0.0, emin=-40, emax=40)
    X = rand_planes(n, p, 72, zero_frac=0.0, emin=-40, emax=40)
    Vr, Xr = recs(V), recs(X)
    # rows 0..99: the second entry cancels the first (same x, negated a) or
    # nearly (a with its last bit flipped)
    for r in range(100):
        k0, k1 = rowptr[r], rowptr[r + 1]
        if k1 - k0 < 2:
            continue
        Xr[colidx[k0 + 1]] = Xr[colidx[k0]]
        Vr[k0 + 1] = Vr[k0]
        Vr[k0 + 1, 0] ^= np.uint64(1)
        if r % 2:
            Vr[k0 + 1, 1] ^= np.uint64(1)
    A = mpk.CSR(rowptr, colidx, synth.records_to_planes(Vr), p)
    x = mpk.Vec.from_planes(synth.records_to_planes(Xr), p)
    want, _ = oracle.spmv(p, oracle.EXACT, rowptr, colidx, Vr, Xr)
    for v in (18, 19, 26, 27):
        A.set_config("exact", 128, v, -1)
        assert_bitwise(mpk.spmv(A, x, mode="exact").planes(), want, f"windowed v={v} p={p}")
    # integers: a_ij in 1..9, x_j in 1..99 (exact products, skipped columns zero)
    ai = 1.0 + (np.arange(len(colidx)) % 9)
    xi = 1.0 + (np.arange(n) % 99)
    B = mpk.CSR(rowptr, colidx, ai, p)
    xb = mpk.Vec.from_f64(xi, p)
    wi, _ = oracle.spmv(p, oracle.EXACT, rowptr, colidx, oracle.from_f64(p, ai),
                        oracle.from_f64(p, xi))
    for v in (18, 27):
        B.set_config("exact", 128, v, -1)
        assert_bitwise(mpk.spmv(B, xb, mode="exact").planes(), wi, f"integers v={v} p={p}")
