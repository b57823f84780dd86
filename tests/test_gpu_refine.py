"""Mixed-precision iterative refinement on row-scaled (kappa ~ 1e20) 3-D
convection-diffusion systems: the refined p-bit x against the exact rational
solution of A x = b (b itself the correctly rounded A*ones)."""
from fractions import Fraction

import numpy as np
import pytest

import exact
import oracle
from gpu_util import need_gpu
from paper_1411_2377_gb300 import synth

pytestmark = pytest.mark.gpu


def exact_solution(rowptr, colidx, vals_recs, b_recs, p):
    """Dense Gaussian elimination over the rationals (small n)."""
    n = len(rowptr) - 1
    A = [[Fraction(0)] * n for _ in range(n)]
    V = exact.vec_decode(vals_recs, p)
    for i in range(n):
        for k in range(rowptr[i], rowptr[i + 1]):
            A[i][colidx[k]] = V[k].q
    b = [v.q for v in exact.vec_decode(b_recs, p)]
    for c in range(n):
        piv = max(range(c, n), key=lambda r: abs(A[r][c]))
        A[c], A[piv] = A[piv], A[c]
        b[c], b[piv] = b[piv], b[c]
        for r in range(c + 1, n):
            if A[r][c] != 0:
                f = A[r][c] / A[c][c]
                for k in range(c, n):
                    A[r][k] -= f * A[c][k]
                b[r] -= f * b[c]
    x = [Fraction(0)] * n
    for r in range(n - 1, -1, -1):
        s = b[r] - sum(A[r][k] * x[k] for k in range(r + 1, n))
        x[r] = s / A[r][r]
    return x


@pytest.mark.parametrize("p,seed", [(256, 2), (128, 5), (512, 2)])
def test_refinement_reaches_1e30_forward_error(p, seed):
    mpk = need_gpu()
    rowptr, colidx, v64 = synth.stencil3d(4, seed=seed)
    n = len(rowptr) - 1
    vals = oracle.from_f64(p, v64)
    b, _ = oracle.spmv(p, oracle.EXACT, rowptr, colidx, vals, oracle.from_f64(p, np.ones(n)))
    xs = exact_solution(rowptr, colidx, vals, b, p)
    A = mpk.CSR(rowptr, colidx, v64, p)
    # stop once a correction is below 256 ulps (x is updated with rounding, so
    # corrections settle at the ulp level and never vanish)
    x, info = mpk.refine(A, mpk.Vec.from_planes(b.T.copy(), p), rtol=2.0 ** (-p + 8),
                         max_outer=40)
    assert info["status"] == 0, info
    X = [v.q for v in exact.vec_decode(x.records(), p)]
    scale = max(abs(v) for v in xs)
    err = max(abs(a - e) for a, e in zip(X, xs)) / scale
    assert err <= Fraction(1, 10 ** 30), (float(err), info)
    # the p-bit residual of the returned x is at rounding level
    assert info["relres"] < 1e-30
    # and x agrees with the exact solution to (almost) the working precision
    assert err <= Fraction(2) ** (-p + 20)


def test_refinement_status_and_options():
    mpk = need_gpu()
    p = 256
    rowptr, colidx, v64 = synth.stencil3d(4, seed=3)
    n = len(rowptr) - 1
    A = mpk.CSR(rowptr, colidx, v64, p)
    b = mpk.spmv(A, mpk.Vec.from_f64(np.ones(n), p), mode="exact")
    x, info = mpk.refine(A, b, max_outer=0)
    assert info["status"] == 7 and info["outer"] == 0  # no correction allowed: NC
    x1, info1 = mpk.refine(A, b, max_outer=1, rtol=1e-60)
    assert info1["outer"] == 1 and info1["inner_iters"] > 0
    # a second call continues from x1 and does not lose accuracy
    x2, info2 = mpk.refine(A, b, x0=x1, rtol=2.0 ** -240, max_outer=30)
    assert info2["status"] == 0
    with pytest.raises(mpk.MPError):
        mpk.refine(A, b, inner_rtol=0.0)


@pytest.mark.parametrize("after", (0, 4, 7))
def test_failed_work_allocation_returns_cuda_status_and_releases_what_it_took(after):
    """A failed stream-ordered allocation of the refinement's work space
    (the first, the fifth or the last of its eight; a fake status from the
    library's host-side fault hook, nothing faults on the GPU) returns
    MP_ERR_CUDA, leaves x as it was and gives back the allocations already
    made; the next refinement is unaffected."""
    import ctypes
    import torch

    mpk = need_gpu()
    lib = mpk._lib.load()
    p = 256
    rowptr, colidx, v64 = synth.stencil3d(4, seed=3)
    n = len(rowptr) - 1
    A = mpk.CSR(rowptr, colidx, v64, p)
    b = mpk.spmv(A, mpk.Vec.from_f64(np.ones(n), p), mode="exact")
    _, info0 = mpk.refine(A, b, rtol=2.0 ** -240, max_outer=30)  # builds the FP64 copy
    assert info0["status"] == 0
    x0 = mpk.Vec.from_f64(np.full(n, 0.5), p)
    torch.cuda.synchronize()
    used = ctypes.c_int64()
    assert lib.mp_debug_pool_used(ctypes.byref(used)) == 0
    before = used.value
    opts = mpk._lib.MpRefineOpts(2.0 ** -240, 30, 1e-10, 20_000, 1, 16)
    info = mpk._lib.MpRefineInfo()
    assert lib.mp_debug_fail(b"work memory", after) == 0
    try:
        st = lib.mp_refine(A.h, b.c(), x0.c(), ctypes.byref(opts), ctypes.byref(info), None)
    finally:
        lib.mp_debug_fail(None, 0)
    assert st == 4  # MP_ERR_CUDA
    assert b"refinement work memory" in lib.mp_last_error()
    torch.cuda.synchronize()
    assert lib.mp_debug_pool_used(ctypes.byref(used)) == 0
    assert used.value == before
    assert np.array_equal(x0.planes(), mpk.Vec.from_f64(np.full(n, 0.5), p).planes())
    _, info1 = mpk.refine(A, b, rtol=2.0 ** -240, max_outer=30)
    assert (info1["status"], info1["outer"]) == (0, info0["outer"])
