"""p = 2048, 4096, 8192 (the warp-per-value form): SpMV in both modes and
its transpose, exact dots and axpy on the GPU vs the oracle's wide build, bit
for bit, through the C ABI; calls outside that set refuse the precision."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_bitwise, need_gpu, rand_planes, random_csr, recs

pytestmark = pytest.mark.gpu
WIDE = (2048, 4096, 8192)
MODES = (("ordered", oracle.ORDERED), ("exact", oracle.EXACT))


@pytest.mark.parametrize("p", WIDE)
def test_spmv_and_transpose(p):
    """Ragged rows (empty, long), 5% explicit zeros, n not a multiple of 32,
    exponents over +-40 (ORDERED rounds every product and sum)."""
    mpk = need_gpu()
    n = {2048: 301, 4096: 133, 8192: 70}[p]
    rowptr, colidx = random_csr(n, seed=p + 1, mean_len=8, max_len=60, empty_every=13)
    V = rand_planes(len(colidx), p, 31, zero_frac=0.05, emin=-40, emax=40)
    X = rand_planes(n, p, 32, zero_frac=0.05, emin=-40, emax=40)
    A = mpk.CSR(rowptr, colidx, V, p, transpose=True)
    x = mpk.Vec.from_planes(X, p)
    for name, m in MODES:
        want, st = oracle.spmv(p, m, rowptr, colidx, recs(V), recs(X))
        assert st == oracle.OK
        assert_bitwise(mpk.spmv(A, x, mode=name).planes(), want, f"spmv {name} p={p}")
        want_t, st = oracle.spmv_t(p, m, rowptr, colidx, recs(V), recs(X))
        assert st == oracle.OK
        assert_bitwise(mpk.spmv_t(A, x, mode=name).planes(), want_t, f"spmv_t {name} p={p}")


@pytest.mark.parametrize("p", (2048, 8192))
def test_exact_rows_cancelling_wide_and_over_the_cap(p):
    """EXACT rows whose products cancel to +0 or to a few low bits, a row
    spanning thousands of bits, and a row past the span cap (+0 and
    MP_ERR_SPAN); ORDERED on the same rows."""
    mpk = need_gpu()
    n = 6
    X = rand_planes(n, p, 41, zero_frac=0.0, emin=-3, emax=3)
    V0 = rand_planes(n, p, 42, zero_frac=0.0, emin=-3, emax=3)
    Xr, Vr = recs(X), recs(V0)
    rows = []
    # row 1: a x0 + (-a) x0 = 0 exactly; row 2: the same with one low bit changed
    neg = Vr[0].copy()
    neg[0] ^= np.uint64(1)
    tweak = neg.copy()
    tweak[1] ^= np.uint64(1)
    rows.append([(0, Vr[0]), (1, Vr[1]), (2, Vr[2])])
    rows.append([(0, Vr[0]), (3, neg)])
    rows.append([(0, Vr[0]), (3, tweak)])
    far = Vr[4].copy()
    far[0] = np.uint64((int(far[0].view(np.int64)) + 2 * 5000) & ((1 << 64) - 1))
    rows.append([(1, Vr[1]), (4, far), (5, Vr[5])])
    over = Vr[4].copy()
    over[0] = np.uint64((int(over[0].view(np.int64)) + 2 * (oracle.SPAN_CAP + 100)) & ((1 << 64) - 1))
    rows.append([(2, Vr[2]), (4, over)])
    rows.append([])
    # duplicate x0 into column 3 so that rows 1-2 cancel a x0 against itself
    Xr[3] = Xr[0]
    rowptr = np.zeros(n + 1, np.int64)
    cols, vals = [], []
    for i, r in enumerate(rows):
        rowptr[i + 1] = rowptr[i] + len(r)
        for c, v in r:
            cols.append(c)
            vals.append(v)
    colidx = np.array(cols, np.int32)
    vrec = np.stack(vals)
    A = mpk.CSR(rowptr, colidx, np.ascontiguousarray(vrec.T), p)
    x = mpk.Vec.from_planes(np.ascontiguousarray(Xr.T), p)
    want, st = oracle.spmv(p, oracle.EXACT, rowptr, colidx, vrec, Xr)
    assert st == oracle.ERR_SPAN
    y = mpk.spmv(A, x, mode="exact", sync=False)
    with pytest.raises(mpk.MPError) as e:
        mpk.check()
    assert e.value.status == 5
    assert_bitwise(y.planes(), want, f"exact p={p}")
    assert (want[1, 0].view(np.int64) >> 1) == oracle.EXP_ZERO and want[1, 0] & 1 == 0
    want, st = oracle.spmv(p, oracle.ORDERED, rowptr, colidx, vrec, Xr)
    assert st == oracle.OK
    assert_bitwise(mpk.spmv(A, x, mode="ordered").planes(), want, f"ordered p={p}")


@pytest.mark.parametrize("p", WIDE)
@pytest.mark.parametrize("n,lo,hi", [(1, -3, 3), (257, -40, 40), (1000, -1500, 1500)])
def test_dot(p, n, lo, hi):
    mpk = need_gpu()
    X = rand_planes(n, p, 51 + n, zero_frac=0.02, emin=lo, emax=hi)
    Y = rand_planes(n, p, 52 + n, zero_frac=0.02, emin=lo, emax=hi)
    got = mpk.dot(mpk.Vec.from_planes(X, p), mpk.Vec.from_planes(Y, p))
    want, st = oracle.dot(p, recs(X), recs(Y))
    assert st == oracle.OK
    assert_bitwise(got.planes(), want[None], f"dot p={p} n={n}")


@pytest.mark.parametrize("p", (2048, 8192))
def test_dot_cancellation_empty_and_span_error(p):
    mpk = need_gpu()
    n = 300
    X = rand_planes(n, p, 61, zero_frac=0.0)
    Y = rand_planes(n, p, 62, zero_frac=0.0)
    Yn = Y.copy()
    Yn[0] ^= np.uint64(1)
    x2 = mpk.Vec.from_planes(np.concatenate([X, X], axis=1), p)
    got = mpk.dot(x2, mpk.Vec.from_planes(np.concatenate([Y, Yn], axis=1), p)).records()[0]
    assert (got[0].view(np.int64) >> 1) == oracle.EXP_ZERO and got[0] & 1 == 0
    got = mpk.dot(mpk.Vec.zeros(0, p), mpk.Vec.zeros(0, p)).records()[0]
    assert (got[0].view(np.int64) >> 1) == oracle.EXP_ZERO
    Xr = recs(X)
    Xr[5, 0] = np.int64(Xr[5, 0].view(np.int64) - 2 * (oracle.SPAN_CAP + 500)).view(np.uint64)
    out = mpk.dot(mpk.Vec.from_planes(Xr.T.copy(), p), mpk.Vec.from_planes(Y, p), sync=False)
    with pytest.raises(mpk.MPError) as e:
        mpk.check()
    assert e.value.status == 5
    want, st = oracle.dot(p, Xr, recs(Y))
    assert st == oracle.ERR_SPAN
    assert_bitwise(out.planes(), want[None], "dot span error")
    # the span slots were reset: the next dot is exact again
    got = mpk.dot(mpk.Vec.from_planes(X, p), mpk.Vec.from_planes(Y, p))
    want, st = oracle.dot(p, recs(X), recs(Y))
    assert_bitwise(got.planes(), want[None], "dot after the span error")


@pytest.mark.parametrize("p", WIDE)
def test_axpy_with_signed_zeros(p):
    mpk = need_gpu()
    n = 200
    X = rand_planes(n, p, 71, zero_frac=0.1, emin=-60, emax=60)
    Y = rand_planes(n, p, 72, zero_frac=0.1, emin=-60, emax=60)
    Yr = recs(Y)
    Yr[::7, 0] |= np.uint64(1)  # some -0 (and some negated values)
    Y = np.ascontiguousarray(Yr.T)
    al = rand_planes(1, p, 73, zero_frac=0.0)
    for alpha, arec in ((mpk.Vec.from_planes(al, p), recs(al)),
                        (mpk.Vec.zeros(1, p), oracle.empty(p, 1))):
        y = mpk.Vec.from_planes(Y, p)
        mpk.axpy(alpha, mpk.Vec.from_planes(X, p), y)
        want, _ = oracle.axpy(p, arec, recs(X), recs(Y))
        assert_bitwise(y.planes(), want, f"axpy p={p}")


@pytest.mark.parametrize("p", (2048, 8192))
def test_f64_matrix_and_residual(p):
    """mp_csr_create_f64 at the wide precisions is exact, the residual is
    exact."""
    mpk = need_gpu()
    n = 50
    rowptr, colidx = random_csr(n, seed=7, mean_len=4, max_len=10)
    v64 = np.linspace(-3.5, 7.25, len(colidx))
    v64[::9] = 0.0
    A = mpk.CSR(rowptr, colidx, v64, p)
    X = rand_planes(n, p, 81, zero_frac=0.0, emin=-5, emax=5)
    vrec = oracle.from_f64(p, v64)
    for name, m in MODES:
        want, _ = oracle.spmv(p, m, rowptr, colidx, vrec, recs(X))
        assert_bitwise(mpk.spmv(A, mpk.Vec.from_planes(X, p), mode=name).planes(), want,
                       f"f64 matrix {name} p={p}")
    b = mpk.Vec.from_planes(X, p)
    # the residual b - A x is one exact row sum at these precisions too
    xv = mpk.Vec.from_planes(rand_planes(n, p, 82, zero_frac=0.1, emin=-5, emax=5), p)
    want, _ = oracle.residual(p, rowptr, colidx, vrec, recs(X), xv.records())
    assert_bitwise(mpk.residual(A, b, xv).planes(), want, f"residual p={p}")


def _dominant_system(p, n, seed):
    rowptr, colidx = random_csr(n, seed=seed, mean_len=5, max_len=14)
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    key = np.unique(np.concatenate([rows, np.arange(n)]) * n +
                    np.concatenate([colidx, np.arange(n)]))
    rowptr = np.zeros(n + 1, np.int64)
    np.add.at(rowptr, key // n + 1, 1)
    rowptr = np.cumsum(rowptr)
    colidx = (key % n).astype(np.int32)
    Vr = recs(rand_planes(len(colidx), p, seed + 1, zero_frac=0.0, emin=-1, emax=1))
    for i in range(n):
        for k in range(rowptr[i], rowptr[i + 1]):
            if colidx[k] == i:
                Vr[k] = oracle.from_f64(p, [float(10 + i % 7)])[0]
    b, _ = oracle.spmv(p, oracle.EXACT, rowptr, colidx, Vr, oracle.from_f64(p, np.ones(n)))
    return rowptr, colidx, Vr, b


@pytest.mark.parametrize("name", ("bicg", "gpbicg", "cgs", "bicgstab"))
@pytest.mark.parametrize("p,mode,n,rtol", [(2048, "ordered", 120, 1e-200),
                                           (2048, "exact", 120, 1e-200),
                                           (4096, "ordered", 60, 1e-300),
                                           (8192, "ordered", 40, 1e-300)])
def test_solvers_vs_oracle(name, p, mode, n, rtol):
    """The four solvers at the wide precisions: status, iteration count, every
    iterate's (r_i, r_i) and x bit for bit against the oracle's wide build;
    x0 nonzero so that r0 = b - A x0 goes through the exact residual."""
    mpk = need_gpu()
    rowptr, colidx, Vr, b = _dominant_system(p, n, seed=p // 64 + n)
    X0 = rand_planes(n, p, 99, zero_frac=0.2, emin=-2, emax=0)
    A = mpk.CSR(rowptr, colidx, np.ascontiguousarray(Vr.T), p, transpose=True)
    fn = getattr(mpk, name)
    maxit = 40
    x, info = fn(A, mpk.Vec.from_planes(np.ascontiguousarray(b.T), p),
                 x0=mpk.Vec.from_planes(X0, p), rtol=rtol, maxit=maxit, mode=mode, poll_every=3,
                 history=True)
    m = oracle.ORDERED if mode == "ordered" else oracle.EXACT
    xo, it, st, hist = getattr(oracle, name)(p, m, rowptr, colidx, Vr, b, recs(X0), rtol, 0.0,
                                             maxit)
    assert (info["status"], info["iters"]) == (st, it)
    assert it > 3
    assert_bitwise(info["history"].planes(), hist, f"{name} p={p} {mode} history")
    assert_bitwise(x.planes(), xo, f"{name} p={p} {mode} x")


@pytest.mark.parametrize("name", ("bicg", "gpbicg", "cgs", "bicgstab"))
def test_solver_exits_at_the_wide_precisions(name):
    """A diagonal system converges in one step (zeta = 0 / t = 0 paths), a
    zero right-hand side returns at once, maxit = 0 is NC."""
    mpk = need_gpu()
    p, n = 2048, 33
    rowptr = np.arange(n + 1, dtype=np.int64)
    colidx = np.arange(n, dtype=np.int32)
    Vr = oracle.from_f64(p, np.full(n, 4.0))
    A = mpk.CSR(rowptr, colidx, np.ascontiguousarray(Vr.T), p, transpose=True)
    fn = getattr(mpk, name)
    for b in (oracle.from_f64(p, np.linspace(1, 3, n)), oracle.empty(p, n)):
        for maxit in (0, 5):
            x, info = fn(A, mpk.Vec.from_planes(np.ascontiguousarray(b.T), p), rtol=1e-30,
                         maxit=maxit, poll_every=1, history=True)
            xo, it, st, hist = getattr(oracle, name)(p, oracle.ORDERED, rowptr, colidx, Vr, b,
                                                     oracle.empty(p, n), 1e-30, 0.0, maxit)
            assert (info["status"], info["iters"]) == (st, it), (maxit, st, it)
            assert_bitwise(x.planes(), xo, f"{name} exit case x")


@pytest.mark.parametrize("p", WIDE)
def test_f64_conversions(p):
    """Doubles to p bits exactly, p bits to the nearest double (ties to even,
    a sticky bit from every lower limb), as the oracle's wide build."""
    mpk = need_gpu()
    import torch

    d = np.array([0.0, -0.0, 1.0, -1.5, 0.1, 1e300, -1e-300, 5e-324, 123456.789,
                  np.nextafter(1.0, 2.0)])
    v = mpk.Vec.from_f64(torch.as_tensor(d), p)
    assert_bitwise(v.planes(), oracle.from_f64(p, d), f"from_f64 p={p}")
    R = recs(rand_planes(300, p, 91, zero_frac=0.05, emin=-900, emax=900))
    R[:5, p // 64] = np.uint64(1 << 63) | np.uint64((1 << 10))  # exactly half an ulp of a double
    R[:5, 1:p // 64] = 0
    got = mpk.Vec.from_planes(np.ascontiguousarray(R.T), p).to_f64().cpu().numpy()
    want = oracle.to_f64(p, R)
    assert np.array_equal(got.view(np.uint64), want.view(np.uint64))


@pytest.mark.parametrize("name", ("bicg", "gpbicg"))
def test_transposed_solve(name):
    """A^T x = b at 2048 bits (the adjoint solve): the oracle solves the
    explicit transpose (rows of A^T list the original rows ascending, the
    order the device's A^T keeps)."""
    mpk = need_gpu()
    p, n = 2048, 90
    rowptr, colidx, Vr, b = _dominant_system(p, n, seed=5)
    A = mpk.CSR(rowptr, colidx, np.ascontiguousarray(Vr.T), p, transpose=True)
    x, info = getattr(mpk, name)(A, mpk.Vec.from_planes(np.ascontiguousarray(b.T), p),
                                 rtol=1e-150, maxit=30, poll_every=4, history=True,
                                 transpose=True)
    rt, ct, vt = oracle.transpose(p, rowptr, colidx, Vr)
    xo, it, st, hist = getattr(oracle, name)(p, oracle.ORDERED, rt, ct, vt, b, oracle.empty(p, n),
                                             1e-150, 0.0, 30)
    assert (info["status"], info["iters"]) == (st, it)
    assert it > 3
    assert_bitwise(info["history"].planes(), hist, f"{name} transposed history")
    assert_bitwise(x.planes(), xo, f"{name} transposed x")
