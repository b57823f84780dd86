"""p-bit CSR SpMV (ORDERED / EXACT), A^T products and residuals on the GPU
vs the oracle, bit for bit, through the C ABI."""
import numpy as np
import pytest

import oracle
from gpu_util import (assert_bitwise, need_gpu, oracle_spmv_threads, rand_planes, random_csr,
                      recs)
from paper_1411_2377_gb300 import synth

pytestmark = pytest.mark.gpu
PRECS = (128, 256, 512, 1024)
MODES = (("ordered", oracle.ORDERED), ("exact", oracle.EXACT))


@pytest.mark.parametrize("p", PRECS)
def test_spmv_random_ragged(p):
    """Several 32-row chunks and sigma windows, a ragged tail (n not a
    multiple of 32), empty rows, long rows, 5% explicit zeros."""
    mpk = need_gpu()
    n = 4099 if p <= 256 else 1187
    rowptr, colidx = random_csr(n, seed=p, mean_len=10, max_len=150, empty_every=17)
    V = rand_planes(len(colidx), p, 11, zero_frac=0.05, emin=-20, emax=20)
    X = rand_planes(n, p, 12, zero_frac=0.05, emin=-20, emax=20)
    A = mpk.CSR(rowptr, colidx, V, p, transpose=True)
    x = mpk.Vec.from_planes(X, p)
    for name, m in MODES:
        y = mpk.spmv(A, x, mode=name)
        want, st = oracle.spmv(p, m, rowptr, colidx, recs(V), recs(X))
        assert st == oracle.OK
        assert_bitwise(y.planes(), want, f"spmv {name} p={p}")
        yt = mpk.spmv_t(A, x, mode=name)
        want_t, _ = oracle.spmv_t(p, m, rowptr, colidx, recs(V), recs(X))
        assert_bitwise(yt.planes(), want_t, f"spmv_t {name} p={p}")


@pytest.mark.parametrize("p", (128, 512))
def test_unsorted_columns_and_explicit_zeros(p):
    """Columns given out of order are summed in ascending column order; stored
    zeros change nothing (Section 2's zero fast path)."""
    mpk = need_gpu()
    n = 300
    rowptr, colidx = random_csr(n, seed=5, mean_len=8, max_len=40)
    V = rand_planes(len(colidx), p, 21, zero_frac=0.1)
    X = rand_planes(n, p, 22, zero_frac=0.0)
    # reverse each row's entries
    perm = np.concatenate([np.arange(rowptr[i + 1] - 1, rowptr[i] - 1, -1) for i in range(n)])
    A1 = mpk.CSR(rowptr, colidx, V, p)
    A2 = mpk.CSR(rowptr, colidx[perm], V[:, perm], p)
    keep = (recs(V)[:, 0].view(np.int64) >> 1) != oracle.EXP_ZERO
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    rp3 = np.zeros(n + 1, np.int64)
    np.add.at(rp3, rows[keep] + 1, 1)
    A3 = mpk.CSR(np.cumsum(rp3), colidx[keep], V[:, keep], p)
    x = mpk.Vec.from_planes(X, p)
    for name, m in MODES:
        want, _ = oracle.spmv(p, m, rowptr, colidx, recs(V), recs(X))
        for A in (A1, A2, A3):
            assert_bitwise(mpk.spmv(A, x, mode=name).planes(), want, f"{name} p={p}")


@pytest.mark.parametrize("p", (128, 1024))
def test_exact_wide_rows_and_span_cap(p):
    """EXACT rows whose exponent span exceeds the per-thread window take the
    wide path; spans beyond the cap are reported and give +0."""
    mpk = need_gpu()
    n = 64
    rowptr, colidx = random_csr(n, seed=9, mean_len=20, max_len=60)
    V = rand_planes(len(colidx), p, 31, zero_frac=0.0, emin=-2, emax=2)
    X = rand_planes(n, p, 32, zero_frac=0.0, emin=-2, emax=2)
    Vr = recs(V)
    # rows 3 and 40: one entry pushed 3000 bits down (wide path); row 7: beyond the cap
    for r, shift in ((3, 3000), (40, 9000), (7, oracle.SPAN_CAP + 100)):
        k = rowptr[r]
        h = Vr[k, 0].view(np.int64)
        Vr[k, 0] = np.int64(h - 2 * shift).view(np.uint64)
    V2 = synth.records_to_planes(Vr)
    A = mpk.CSR(rowptr, colidx, V2, p)
    x = mpk.Vec.from_planes(X, p)
    y = mpk.spmv(A, x, mode="exact", sync=False)
    with pytest.raises(mpk.MPError) as e:
        mpk.check()
    assert e.value.status == 5
    want, st = oracle.spmv(p, oracle.EXACT, rowptr, colidx, Vr, recs(X))
    assert st == oracle.ERR_SPAN
    assert_bitwise(y.planes(), want, f"exact wide p={p}")
    # ORDERED has no span limit
    yo = mpk.spmv(A, x, mode="ordered")
    want_o, _ = oracle.spmv(p, oracle.ORDERED, rowptr, colidx, Vr, recs(X))
    assert_bitwise(yo.planes(), want_o, f"ordered wide p={p}")


@pytest.mark.parametrize("p", (128, 256))
def test_residual(p):
    mpk = need_gpu()
    n = 777
    rowptr, colidx = random_csr(n, seed=13, mean_len=7, max_len=30, empty_every=11)
    V = rand_planes(len(colidx), p, 41, zero_frac=0.02, emin=-5, emax=5)
    X = rand_planes(n, p, 42, zero_frac=0.1, emin=-5, emax=5)
    B = rand_planes(n, p, 43, zero_frac=0.1, emin=-5, emax=5)
    A = mpk.CSR(rowptr, colidx, V, p)
    r = mpk.residual(A, mpk.Vec.from_planes(B, p), mpk.Vec.from_planes(X, p))
    want, _ = oracle.residual(p, rowptr, colidx, recs(V), recs(B), recs(X))
    assert_bitwise(r.planes(), want, f"residual p={p}")


@pytest.mark.parametrize("p", (128, 256, 1024))
def test_stencil_f64_matrices(p):
    """Double-valued matrices (the 2-D and 3-D stencils) converted exactly."""
    mpk = need_gpu()
    for rowptr, colidx, v64 in (synth.stencil2d(24, 0), synth.stencil3d(8, 2)):
        n = len(rowptr) - 1
        A = mpk.CSR(rowptr, colidx, v64, p, transpose=True)
        X = rand_planes(n, p, 51, zero_frac=0.0, emin=-3, emax=3)
        vals = oracle.from_f64(p, v64)
        x = mpk.Vec.from_planes(X, p)
        for name, m in MODES:
            want, _ = oracle.spmv(p, m, rowptr, colidx, vals, recs(X))
            assert_bitwise(mpk.spmv(A, x, mode=name).planes(), want, f"stencil {name} p={p}")


def test_bad_inputs_are_rejected():
    mpk = need_gpu()
    p = 128
    rowptr = np.array([0, 2, 3], np.int64)
    V = rand_planes(3, p, 1, zero_frac=0.0)
    with pytest.raises(mpk.MPError):  # column out of range
        mpk.CSR(rowptr, np.array([0, 5, 1], np.int32), V, p)
    with pytest.raises(mpk.MPError):  # repeated column
        mpk.CSR(rowptr, np.array([1, 1, 0], np.int32), V, p)
    bad = V.copy()
    bad[p // 64, 1] = 0  # unnormalised mantissa
    with pytest.raises(mpk.MPError):
        mpk.CSR(rowptr, np.array([0, 1, 1], np.int32), bad, p)
    with pytest.raises(mpk.MPError):  # NaN
        mpk.CSR(rowptr, np.array([0, 1, 1], np.int32), np.array([1.0, np.nan, 2.0]), p)
    with pytest.raises(mpk.MPError):  # unsupported precision
        mpk.CSR(rowptr, np.array([0, 1, 1], np.int32), np.array([1.0, 3.0, 2.0]), 192)
    A = mpk.CSR(rowptr, np.array([0, 1, 1], np.int32), V, p)
    with pytest.raises(mpk.MPError):  # no transpose built
        mpk.spmv_t(A, mpk.Vec.zeros(2, p))
    with pytest.raises(mpk.MPError):  # wrong length
        mpk.spmv(A, mpk.Vec.zeros(3, p))
    empty = mpk.CSR(np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros((3, 0), np.uint64), p)
    y = mpk.spmv(empty, mpk.Vec.zeros(0, p))
    assert y.n == 0


_PATTERN = {}


@pytest.mark.parametrize("p", PRECS)
def test_full_size_every_row(p):
    """The throughput workload at full size (n = 10^6, lognormal rows, band
    +-5000, 10% far columns, 1% zeros): every row of y = A x, both modes,
    bit-identical to the oracle (run over the host's cores) in the launch
    configuration the benchmark times (autotuned as it does), in the
    library's default one, and in every variant code 0-31 of the launch
    configuration (whatever the tuner could pick)."""
    mpk = need_gpu()
    from paper_1411_2377_gb300 import tune

    if "p" not in _PATTERN:
        _PATTERN["p"] = synth.spmv_pattern()
    rowptr, colidx = _PATTERN["p"]
    n = len(rowptr) - 1
    V, X = synth.spmv_values(p, len(colidx), n)
    Vr, Xr = recs(V), recs(X)
    A = mpk.CSR(rowptr, colidx, V, p)
    del V
    x = mpk.Vec.from_planes(X, p)
    y = mpk.Vec.empty(n, p)
    tuned = tune.autotune(A, reps=3, cache=None)
    for name, mode in MODES:
        want = oracle_spmv_threads(oracle, p, mode, rowptr, colidx, Vr, Xr).T

        def check(what):
            mpk.spmv(A, x, y, mode=name)
            got = y.planes()
            bad = np.nonzero(np.any(got != want, axis=0))[0]
            assert bad.size == 0, f"{name} p={p} {what}: {bad.size} rows differ, first {bad[:5]}"

        t = tuned[name]
        A.set_config(name, t["threads_per_block"], t["variant"], t["carveout"])
        check(f"tuned {t}")
        carve = 50 if name == "exact" else -1
        for v in range(-1, 32):
            A.set_config(name, 128, v, carve)
            check(f"variant {v}")
        del want
    A.close()


@pytest.mark.parametrize("p", (128, 256))
def test_device_transpose_with_a_long_column_and_unsorted_rows(p):
    """A and A^T laid out on the device: column 3 holds 600 entries (its row of
    A^T is longer than one thread sorts, so the host sorts it) and every input
    row lists its columns in reverse (the host sorts those rows); A x and A^T x
    bit-identical to the oracle in both modes."""
    mpk = need_gpu()
    n = 700
    rowptr, colidx = random_csr(n, seed=41, mean_len=5, max_len=20)
    rows = [set(colidx[rowptr[i]:rowptr[i + 1]].tolist()) for i in range(n)]
    for i in range(600):
        rows[i].add(3)
    cols = [sorted(r) for r in rows]
    rowptr = np.zeros(n + 1, np.int64)
    rowptr[1:] = np.cumsum([len(c) for c in cols])
    colidx = np.array([c for r in cols for c in r], np.int32)
    V = rand_planes(len(colidx), p, 51, zero_frac=0.05)
    X = rand_planes(n, p, 52, zero_frac=0.0)
    perm = np.concatenate([np.arange(rowptr[i + 1] - 1, rowptr[i] - 1, -1) for i in range(n)])
    A = mpk.CSR(rowptr, colidx[perm], V[:, perm], p, transpose=True)
    x = mpk.Vec.from_planes(X, p)
    for name, m in MODES:
        want, _ = oracle.spmv(p, m, rowptr, colidx, recs(V), recs(X))
        want_t, _ = oracle.spmv_t(p, m, rowptr, colidx, recs(V), recs(X))
        assert_bitwise(mpk.spmv(A, x, mode=name).planes(), want, f"{name} p={p}")
        assert_bitwise(mpk.spmv_t(A, x, mode=name).planes(), want_t, f"T {name} p={p}")


def test_products_with_a_and_its_transpose_at_the_same_time():
    """y = A x and z = A^T w on two streams at once (as BiCG runs them), EXACT
    at p = 256 on a scattered pattern with n >= 65536, so that both products
    gather x from a record copy, and with exponents spread over +-300, so that
    rows overflow to the exact warp-per-row kernel: the two layouts have their
    own record buffers and overflow lists, and both results equal the
    oracle's, in three rounds with different vectors."""
    mpk = need_gpu()
    import torch

    p, n = 256, 70_000
    rowptr, colidx = random_csr(n, seed=71, mean_len=4, max_len=40)
    V = rand_planes(len(colidx), p, 72, zero_frac=0.02, emin=-300, emax=300)
    A = mpk.CSR(rowptr, colidx, V, p, transpose=True)
    Vr = recs(V)
    rt, ct, vt = oracle.transpose(p, rowptr, colidx, Vr)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    for k in range(3):
        X = rand_planes(n, p, 73 + 2 * k, zero_frac=0.02, emin=-40, emax=40)
        Wv = rand_planes(n, p, 74 + 2 * k, zero_frac=0.02, emin=-40, emax=40)
        x, w = mpk.Vec.from_planes(X, p), mpk.Vec.from_planes(Wv, p)
        y, z = mpk.Vec.empty(n, p), mpk.Vec.empty(n, p)
        torch.cuda.synchronize()
        mpk.spmv(A, x, y, mode="exact", stream=s1, sync=False)
        mpk.spmv_t(A, w, z, mode="exact", stream=s2, sync=False)
        torch.cuda.synchronize()
        want_y = oracle_spmv_threads(oracle, p, oracle.EXACT, rowptr, colidx, Vr, recs(X))
        want_z = oracle_spmv_threads(oracle, p, oracle.EXACT, rt, ct, vt, recs(Wv))
        assert_bitwise(y.planes(), want_y, f"A x beside A^T w, round {k}")
        assert_bitwise(z.planes(), want_z, f"A^T w beside A x, round {k}")
    A.close()
