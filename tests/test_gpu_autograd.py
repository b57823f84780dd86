"""Differentiated GPBiCG solve: adjoint solve with A^T and the gradient on the
sparsity pattern, against the oracle's adjoint (bit for bit) and against
512-bit central finite differences."""
from fractions import Fraction

import numpy as np
import pytest

import exact
import oracle
from gpu_util import assert_bitwise, need_gpu
from paper_1411_2377_gb300 import synth

pytestmark = pytest.mark.gpu


def _system(m, p, seed=0):
    rowptr, colidx, v64 = synth.stencil2d(m, seed=seed)
    n = len(rowptr) - 1
    vals = oracle.from_f64(p, v64)
    b, _ = oracle.spmv(p, oracle.EXACT, rowptr, colidx, vals, oracle.from_f64(p, np.ones(n)))
    return rowptr, colidx, v64, vals, b


@pytest.mark.parametrize("p", (128, 256))
def test_adjoint_and_pattern_gradient_match_the_oracle(p):
    mpk = need_gpu()
    from paper_1411_2377_gb300 import autograd

    rowptr, colidx, v64, vals, b = _system(12, p, seed=4)
    n = len(rowptr) - 1
    A = mpk.CSR(rowptr, colidx, v64, p, transpose=True)
    x, info = autograd.solve(A, mpk.Vec.from_planes(b.T.copy(), p), rtol=1e-25)
    xo, it, st, _ = oracle.gpbicg(p, oracle.ORDERED, rowptr, colidx, vals, b, oracle.empty(p, n),
                                  1e-25, 0.0, 100_000)
    assert_bitwise(x.planes(), xo, "forward x")
    # L = sum x_i^2  ->  xbar = 2x (exact)
    two = oracle.from_f64(p, np.full(n, 2.0))
    xbar, _ = oracle.ewise(p, oracle.OP_MUL, two, xo)
    lam, g, ainfo = autograd.adjoint(A, x, mpk.Vec.from_planes(xbar.T.copy(), p), rtol=1e-25)
    trp, tci, tv = oracle.transpose(p, rowptr, colidx, vals)
    lo, it2, st2, _ = oracle.gpbicg(p, oracle.ORDERED, trp, tci, tv, xbar, oracle.empty(p, n),
                                    1e-25, 0.0, 100_000)
    assert st2 == oracle.OK and ainfo["iters"] == it2
    assert_bitwise(lam.planes(), lo, "adjoint lambda")
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    neg_lam = lo[rows].copy()
    neg_lam[:, 0] ^= np.uint64(1)
    want, _ = oracle.ewise(p, oracle.OP_MUL, neg_lam, xo[colidx])
    assert_bitwise(g.planes(), want, "pattern gradient")


def _loss(mpk, rowptr, colidx, vals_planes, b_planes, p, rtol):
    A = mpk.CSR(rowptr, colidx, vals_planes, p)
    x, info = mpk.gpbicg(A, mpk.Vec.from_planes(b_planes, p), rtol=rtol, maxit=100_000)
    assert info["status"] == 0
    L = mpk.dot(x, x)
    return exact.decode(L.records()[0], p).q


def test_gradient_vs_512bit_central_differences():
    """32 stored entries and 4 entries of b: (L(a+h) - L(a-h)) / 2h with
    h = 2^-100 at 512 bits, forward solves to 1e-140, against the adjoint
    gradient (L = sum x^2)."""
    mpk = need_gpu()
    from paper_1411_2377_gb300 import autograd

    p = 512
    rowptr, colidx, v64, vals, b = _system(16, p, seed=7)
    n = len(rowptr) - 1
    nnz = len(colidx)
    A = mpk.CSR(rowptr, colidx, v64, p, transpose=True)
    x, _ = autograd.solve(A, mpk.Vec.from_planes(b.T.copy(), p), rtol=1e-140)
    two = mpk.Vec.from_f64(np.full(n, 2.0), p)
    xbar = mpk.ewise(0, two, x)
    lam, g, _ = autograd.adjoint(A, x, xbar, rtol=1e-140)
    G = [exact.decode(r, p).q for r in g.records()]
    LAM = [exact.decode(r, p).q for r in lam.records()]
    h = Fraction(1, 2 ** 100)
    ks = np.unique(synth.u64(9, 1, np.arange(32)) % np.uint64(nnz)).astype(np.int64)
    scale = max(abs(v) for v in G)
    vr = vals.copy()
    for k in ks:
        a = exact.decode(vals[k], p).q
        fd = []
        for sgn in (1, -1):
            vr[k] = exact.encode(exact.Val(a + sgn * h), p)
            fd.append(_loss(mpk, rowptr, colidx, vr.T.copy(), b.T.copy(), p, 1e-140))
        vr[k] = vals[k]
        d = (fd[0] - fd[1]) / (2 * h)
        assert abs(d - G[k]) <= Fraction(1, 10 ** 40) * scale, (k, float(d), float(G[k]))
    br = b.copy()
    for i in (0, n // 3, n // 2, n - 1):
        bi = exact.decode(b[i], p).q
        fd = []
        for sgn in (1, -1):
            br[i] = exact.encode(exact.Val(bi + sgn * h), p)
            fd.append(_loss(mpk, rowptr, colidx, vals.T.copy(), br.T.copy(), p, 1e-140))
        br[i] = b[i]
        d = (fd[0] - fd[1]) / (2 * h)
        assert abs(d - LAM[i]) <= Fraction(1, 10 ** 40) * max(abs(v) for v in LAM), i


def test_p256_gradient_vs_512bit_central_differences():
    """The differentiated solve at the precision it is used at (p = 256, 2-D
    system, L = sum x^2): the adjoint gradient at 32 stored entries and 4
    entries of b against central differences taken at 512 bits (h = 2^-100,
    the perturbed systems solved at 512 bits to 1e-140; the 256-bit values
    and b are exact at 512 bits, so both sides differentiate the same
    function).  The 256-bit gradient carries about kappa * 2^-256 of relative
    error, the differences about h^2: both far below the 1e-40 tolerance."""
    mpk = need_gpu()
    from paper_1411_2377_gb300 import autograd

    p, q = 256, 512
    rowptr, colidx, v64, vals, b = _system(16, p, seed=11)
    n = len(rowptr) - 1
    nnz = len(colidx)
    A = mpk.CSR(rowptr, colidx, v64, p, transpose=True)
    x, _ = autograd.solve(A, mpk.Vec.from_planes(b.T.copy(), p), rtol=1e-70)
    two = mpk.Vec.from_f64(np.full(n, 2.0), p)
    lam, g, _ = autograd.adjoint(A, x, mpk.ewise(0, two, x), rtol=1e-70)
    G = [exact.decode(r, p).q for r in g.records()]
    LAM = [exact.decode(r, p).q for r in lam.records()]
    # the same values and b at 512 bits (exact: they have at most 256 bits)
    vq = np.array([exact.encode(exact.decode(r, p), q) for r in vals], np.uint64)
    bq = np.array([exact.encode(exact.decode(r, p), q) for r in b], np.uint64)
    h = Fraction(1, 2 ** 100)
    ks = np.unique(synth.u64(21, 1, np.arange(32)) % np.uint64(nnz)).astype(np.int64)
    scale = max(abs(v) for v in G)
    vr = vq.copy()
    for k in ks:
        a = exact.decode(vq[k], q).q
        fd = []
        for sgn in (1, -1):
            vr[k] = exact.encode(exact.Val(a + sgn * h), q)
            fd.append(_loss(mpk, rowptr, colidx, vr.T.copy(), bq.T.copy(), q, 1e-140))
        vr[k] = vq[k]
        d = (fd[0] - fd[1]) / (2 * h)
        assert abs(d - G[k]) <= Fraction(1, 10 ** 40) * scale, (k, float(d), float(G[k]))
    br = bq.copy()
    for i in (0, n // 3, n // 2, n - 1):
        bi = exact.decode(bq[i], q).q
        fd = []
        for sgn in (1, -1):
            br[i] = exact.encode(exact.Val(bi + sgn * h), q)
            fd.append(_loss(mpk, rowptr, colidx, vq.T.copy(), br.T.copy(), q, 1e-140))
        br[i] = bq[i]
        d = (fd[0] - fd[1]) / (2 * h)
        assert abs(d - LAM[i]) <= Fraction(1, 10 ** 40) * max(abs(v) for v in LAM), i


def test_torch_autograd_function():
    mpk = need_gpu()
    import torch

    from paper_1411_2377_gb300 import autograd

    p = 256
    rowptr, colidx, v64 = synth.stencil2d(10, seed=2)
    n = len(rowptr) - 1
    values = torch.tensor(v64, dtype=torch.float64, requires_grad=True)
    b = torch.linspace(1.0, 2.0, n, dtype=torch.float64, device="cuda", requires_grad=True)
    x = autograd.MPSolve().apply(values, b, rowptr, colidx, p, 1e-40, 10_000, "ordered")
    loss = (x * x).sum()
    loss.backward()
    # reference at p bits through the adjoint interface
    A = mpk.CSR(rowptr, colidx, v64, p, transpose=True)
    xp, _ = autograd.solve(A, mpk.Vec.from_f64(b.detach(), p), rtol=1e-40)
    xbar = mpk.Vec.from_f64(2.0 * xp.to_f64(), p)
    lam, g, _ = autograd.adjoint(A, xp, xbar, rtol=1e-40)
    assert torch.equal(x.detach(), xp.to_f64())
    assert torch.allclose(b.grad, lam.to_f64(), rtol=1e-14, atol=0)
    assert torch.allclose(values.grad.to("cuda"), g.to_f64(), rtol=1e-14, atol=0)
    # and the float64 gradient agrees with a dense float64 computation
    Ad = torch.zeros(n, n, dtype=torch.float64)
    for i in range(n):
        Ad[i, colidx[rowptr[i]:rowptr[i + 1]]] = torch.tensor(v64[rowptr[i]:rowptr[i + 1]])
    xd = torch.linalg.solve(Ad, b.detach().cpu())
    lamd = torch.linalg.solve(Ad.T, 2 * xd)
    assert torch.allclose(b.grad.cpu(), lamd, rtol=1e-9)
