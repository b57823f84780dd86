"""ILU(0) on the device vs the oracle, bit for bit: the factors, the
preconditioner application (one-block and one-launch-per-level forms), and
BiCGSTAB preconditioned with it, left (Section 4.2, the paper's form) and
right (every iterate's residual norm, the iteration count, the status and
x)."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_bitwise, need_gpu, rand_planes, random_csr, recs
from paper_1411_2377_gb300 import synth

pytestmark = pytest.mark.gpu


def dominant_system(n, p, seed):
    rowptr, colidx = random_csr(n, seed=seed, mean_len=6, max_len=20)
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    key = np.unique(np.concatenate([rows * n + colidx, np.arange(n) * (n + 1)]))
    rowptr = np.zeros(n + 1, np.int64)
    np.add.at(rowptr, key // n + 1, 1)
    rowptr = np.cumsum(rowptr)
    colidx = (key % n).astype(np.int32)
    Vr = recs(rand_planes(len(colidx), p, seed + 1, zero_frac=0.05, emin=-1, emax=1))
    for i in range(n):
        for k in range(rowptr[i], rowptr[i + 1]):
            if colidx[k] == i:
                Vr[k] = oracle.from_f64(p, [float(10 + i % 7)])[0]
    return rowptr, colidx, Vr


@pytest.mark.parametrize("p", (128, 256, 512, 1024))
def test_factor_and_apply_match_the_oracle(p):
    mpk = need_gpu()
    n = 300
    rowptr, colidx, Vr = dominant_system(n, p, p + 3)
    A = mpk.CSR(rowptr, colidx, synth.records_to_planes(Vr), p)
    M = mpk.ILU0(A)
    lu_o, st = oracle.ilu0(p, rowptr, colidx, Vr)
    assert st == oracle.OK
    assert_bitwise(M.factor().planes(), lu_o, f"ILU(0) factor p={p}")
    R = rand_planes(n, p, 9, zero_frac=0.1, emin=-5, emax=5)
    w = M.apply(mpk.Vec.from_planes(R, p))
    w_o, st = oracle.ilu0_apply(p, rowptr, colidx, lu_o, recs(R))
    assert st == oracle.OK
    assert_bitwise(w.planes(), w_o, f"ILU(0) apply p={p}")
    nl, nu = M.levels()
    assert 1 <= nl <= n and 1 <= nu <= n


@pytest.mark.parametrize("side", ("left", "right"))
@pytest.mark.parametrize("p", (128, 256, 1024))
@pytest.mark.parametrize("mode", ("ordered", "exact"))
def test_preconditioned_bicgstab_matches_the_oracle(p, mode, side):
    mpk = need_gpu()
    rowptr, colidx, v64 = synth.stencil2d(16, seed=2)
    n = len(rowptr) - 1
    vals = oracle.from_f64(p, v64)
    b, _ = oracle.spmv(p, oracle.EXACT, rowptr, colidx, vals, oracle.from_f64(p, np.ones(n)))
    A = mpk.CSR(rowptr, colidx, v64, p)
    M = mpk.ILU0(A)
    x, info = mpk.bicgstab_ilu0(A, M, mpk.Vec.from_planes(synth.records_to_planes(b), p),
                                rtol=1e-30, maxit=300, mode=mode, poll_every=3, history=True,
                                side=side)
    m = oracle.ORDERED if mode == "ordered" else oracle.EXACT
    xo, it, st, hist = oracle.bicgstab_ilu0(p, m, rowptr, colidx, vals, b, oracle.empty(p, n),
                                            1e-30, 0.0, 300, side=side)
    assert st == oracle.OK
    assert (info["iters"], info["status"]) == (it, st)
    assert_bitwise(info["history"].planes(), hist, f"history p={p} {mode} {side}")
    assert_bitwise(x.planes(), xo, f"x p={p} {mode} {side}")
    # fewer iterations than without the preconditioner
    _, plain = mpk.bicgstab(A, mpk.Vec.from_planes(synth.records_to_planes(b), p), rtol=1e-30,
                            maxit=300, mode=mode)
    assert info["iters"] < plain["iters"]


@pytest.mark.parametrize("side", ("left", "right"))
def test_noconv_and_poll_interval(side):
    mpk = need_gpu()
    p = 512
    rowptr, colidx, v64 = synth.stencil2d(12, seed=6)
    n = len(rowptr) - 1
    Vr = oracle.from_f64(p, v64)
    B = rand_planes(n, p, 22, zero_frac=0.0, emin=-2, emax=2)
    A = mpk.CSR(rowptr, colidx, v64, p)
    M = mpk.ILU0(A)
    xo, it, st, hist = oracle.bicgstab_ilu0(p, oracle.EXACT, rowptr, colidx, Vr, recs(B),
                                            oracle.empty(p, n), 1e-200, 0.0, 3, side=side)
    for poll in (1, 7):
        x, info = mpk.bicgstab_ilu0(A, M, mpk.Vec.from_planes(B, p), rtol=1e-200, maxit=3,
                                    mode="exact", poll_every=poll, history=True, side=side)
        assert (info["iters"], info["status"]) == (it, st) == (3, oracle.ERR_NOCONV)
        assert_bitwise(info["history"].planes(), hist, "history")
        assert_bitwise(x.planes(), xo, "x")


def test_zero_pivot_and_missing_diagonal():
    mpk = need_gpu()
    p = 128
    rowptr = np.array([0, 2, 4], np.int64)
    colidx = np.array([0, 1, 0, 1], np.int32)
    A = mpk.CSR(rowptr, colidx, np.array([0.0, 1.0, 1.0, 1.0]), p)
    with pytest.raises(mpk.MPError) as e:
        mpk.ILU0(A)
    assert e.value.status == 9
    B = mpk.CSR(np.array([0, 1, 2], np.int64), np.array([1, 0], np.int32), np.array([1.0, 1.0]), p)
    with pytest.raises(mpk.MPError) as e:
        mpk.ILU0(B)
    assert e.value.status == 9


def test_apply_beyond_one_block_matches_the_oracle():
    """n > 2^18 rows: the solves run one launch per level instead of one
    block looping over the levels (2-D stencil, 2 * 520 - 1 levels each)."""
    mpk = need_gpu()
    p = 128
    rowptr, colidx, v64 = synth.stencil2d(520, seed=4)
    n = len(rowptr) - 1
    assert n > 2 ** 18
    vals = oracle.from_f64(p, v64)
    A = mpk.CSR(rowptr, colidx, v64, p)
    M = mpk.ILU0(A)
    assert M.levels() == (2 * 520 - 1, 2 * 520 - 1)
    lu_o, st = oracle.ilu0(p, rowptr, colidx, vals)
    assert st == oracle.OK
    assert_bitwise(M.factor().planes(), lu_o, "ILU(0) factor n=270400")
    R = rand_planes(n, p, 31, zero_frac=0.02, emin=-4, emax=4)
    w = M.apply(mpk.Vec.from_planes(R, p))
    w_o, st = oracle.ilu0_apply(p, rowptr, colidx, lu_o, recs(R))
    assert st == oracle.OK
    assert_bitwise(w.planes(), w_o, "ILU(0) apply n=270400")


@pytest.mark.parametrize("p,n", [(2048, 150), (4096, 70), (8192, 40)])
def test_wide_factor_and_apply_match_the_oracle(p, n):
    """p = 2048-8192 (the warp-per-row kernels): factors with zero entries
    (5% of the stored values), then (LU)^{-1} r, against the oracle's wide
    build bit for bit."""
    mpk = need_gpu()
    rowptr, colidx, Vr = dominant_system(n, p, p // 64 + 5)
    A = mpk.CSR(rowptr, colidx, synth.records_to_planes(Vr), p)
    M = mpk.ILU0(A)
    lu_o, st = oracle.ilu0(p, rowptr, colidx, Vr)
    assert st == oracle.OK
    assert_bitwise(M.factor().planes(), lu_o, f"ILU(0) factor p={p}")
    R = rand_planes(n, p, 19, zero_frac=0.1, emin=-5, emax=5)
    w = M.apply(mpk.Vec.from_planes(R, p))
    w_o, st = oracle.ilu0_apply(p, rowptr, colidx, lu_o, recs(R))
    assert st == oracle.OK
    assert_bitwise(w.planes(), w_o, f"ILU(0) apply p={p}")


WIDE_CASES = [(2048, "ordered", 8), (2048, "exact", 8), (4096, "ordered", 6),
              (8192, "ordered", 5)]


def _wide_system(p, grid):
    rowptr, colidx, v64 = synth.stencil2d(grid, seed=3)
    n = len(rowptr) - 1
    vals = oracle.from_f64(p, v64)
    b, _ = oracle.spmv(p, oracle.EXACT, rowptr, colidx, vals, oracle.from_f64(p, np.ones(n)))
    return rowptr, colidx, v64, vals, b


@pytest.fixture(scope="module")
def wide_oracle():
    """The oracle's preconditioned and plain solves of every wide case, run
    at once on host threads (the C oracle releases the interpreter lock; its
    correctly rounded division makes one ILU(0) solve take seconds)."""
    import os
    from concurrent.futures import ThreadPoolExecutor

    def run(key):
        p, mode, grid, side = key
        rowptr, colidx, _, vals, b = _wide_system(p, grid)
        n = len(rowptr) - 1
        m = oracle.ORDERED if mode == "ordered" else oracle.EXACT
        if side == "plain":
            return oracle.bicgstab(p, m, rowptr, colidx, vals, b, oracle.empty(p, n), 1e-60, 0.0,
                                   200)
        return oracle.bicgstab_ilu0(p, m, rowptr, colidx, vals, b, oracle.empty(p, n), 1e-60,
                                    0.0, 200, side=side)

    keys = [c + (side,) for c in WIDE_CASES for side in ("left", "right", "plain")]
    with ThreadPoolExecutor(max(1, min(len(keys), os.cpu_count() or 1))) as ex:
        return dict(zip(keys, ex.map(run, keys)))


@pytest.mark.parametrize("side", ("left", "right"))
@pytest.mark.parametrize("p,mode,grid", WIDE_CASES)
def test_wide_preconditioned_bicgstab_matches_the_oracle(p, mode, grid, side, wide_oracle):
    """Table 3's precisions: BiCGSTAB+ILU(0) at 2048-8192 bits on a 2-D
    convection-diffusion stencil, every iterate's residual norm, the count,
    the status and x against the oracle; fewer iterations than plain
    BiCGSTAB on the same system (the oracle's count)."""
    mpk = need_gpu()
    rowptr, colidx, v64, vals, b = _wide_system(p, grid)
    A = mpk.CSR(rowptr, colidx, v64, p)
    M = mpk.ILU0(A)
    x, info = mpk.bicgstab_ilu0(A, M, mpk.Vec.from_planes(synth.records_to_planes(b), p),
                                rtol=1e-60, maxit=200, mode=mode, poll_every=4, history=True,
                                side=side)
    xo, it, st, hist = wide_oracle[(p, mode, grid, side)]
    assert st == oracle.OK
    assert (info["iters"], info["status"]) == (it, st)
    assert_bitwise(info["history"].planes(), hist, f"history p={p} {mode} {side}")
    assert_bitwise(x.planes(), xo, f"x p={p} {mode} {side}")
    assert it < wide_oracle[(p, mode, grid, "plain")][1]


def test_wide_noconv_zero_pivot_and_missing_diagonal():
    """At 2048 bits: maxit = 3 stops NC with the oracle's third iterate; a zero
    pivot and a row without its diagonal entry refuse the factor
    (MP_ERR_DIVZERO)."""
    mpk = need_gpu()
    p = 2048
    rowptr, colidx, v64 = synth.stencil2d(9, seed=6)
    n = len(rowptr) - 1
    Vr = oracle.from_f64(p, v64)
    B = rand_planes(n, p, 23, zero_frac=0.0, emin=-2, emax=2)
    A = mpk.CSR(rowptr, colidx, v64, p)
    M = mpk.ILU0(A)
    for side in ("left", "right"):
        xo, it, st, hist = oracle.bicgstab_ilu0(p, oracle.EXACT, rowptr, colidx, Vr, recs(B),
                                                oracle.empty(p, n), 1e-200, 0.0, 3, side=side)
        x, info = mpk.bicgstab_ilu0(A, M, mpk.Vec.from_planes(B, p), rtol=1e-200, maxit=3,
                                    mode="exact", poll_every=1, history=True, side=side)
        assert (info["iters"], info["status"]) == (it, st) == (3, oracle.ERR_NOCONV)
        assert_bitwise(info["history"].planes(), hist, f"history {side}")
        assert_bitwise(x.planes(), xo, f"x {side}")
    rp = np.array([0, 2, 4], np.int64)
    ci = np.array([0, 1, 0, 1], np.int32)
    with pytest.raises(mpk.MPError) as e:
        mpk.ILU0(mpk.CSR(rp, ci, np.array([0.0, 1.0, 1.0, 1.0]), p))
    assert e.value.status == 9
    with pytest.raises(mpk.MPError) as e:
        mpk.ILU0(mpk.CSR(np.array([0, 1, 2], np.int64), np.array([1, 0], np.int32),
                         np.array([1.0, 1.0]), p))
    assert e.value.status == 9
