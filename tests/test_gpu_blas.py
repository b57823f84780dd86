"""Exact dot products and axpy on the GPU vs the oracle, bit for bit."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_bitwise, need_gpu, rand_planes, recs

pytestmark = pytest.mark.gpu
PRECS = (128, 256, 512, 1024)


@pytest.mark.parametrize("p", PRECS)
@pytest.mark.parametrize("n,lo,hi", [(1, -3, 3), (31, -3, 3), (4097, -40, 40),
                                     (2_000, -1500, 1500), (100_003, -200, 200),
                                     (50_000, -1500, 1500)])
def test_dot(p, n, lo, hi):
    """Spans inside the per-thread window and (lo/hi = +-1500) the wide path."""
    mpk = need_gpu()
    X = rand_planes(n, p, 61 + n, zero_frac=0.02, emin=lo, emax=hi)
    Y = rand_planes(n, p, 62 + n, zero_frac=0.02, emin=lo, emax=hi)
    got = mpk.dot(mpk.Vec.from_planes(X, p), mpk.Vec.from_planes(Y, p))
    want, st = oracle.dot(p, recs(X), recs(Y))
    assert st == oracle.OK
    assert_bitwise(got.planes(), want[None], f"dot p={p} n={n}")


@pytest.mark.parametrize("p", (128, 512))
def test_dot_cancellation_zero_and_span_error(p):
    mpk = need_gpu()
    n = 1000
    X = rand_planes(n, p, 71, zero_frac=0.0)
    Y = rand_planes(n, p, 72, zero_frac=0.0)
    Yn = Y.copy()
    Yn[0] ^= np.uint64(1)
    x2 = mpk.Vec.from_planes(np.concatenate([X, X], axis=1), p)
    y2 = mpk.Vec.from_planes(np.concatenate([Y, Yn], axis=1), p)
    got = mpk.dot(x2, y2).records()[0]
    assert (got[0].view(np.int64) >> 1) == oracle.EXP_ZERO and got[0] & 1 == 0  # +0
    # empty vectors
    got = mpk.dot(mpk.Vec.zeros(0, p), mpk.Vec.zeros(0, p)).records()[0]
    assert (got[0].view(np.int64) >> 1) == oracle.EXP_ZERO
    # a span beyond the cap: +0 and MP_ERR_SPAN
    Xr = recs(X)
    Xr[5, 0] = np.int64(Xr[5, 0].view(np.int64) - 2 * (oracle.SPAN_CAP + 500)).view(np.uint64)
    out = mpk.dot(mpk.Vec.from_planes(Xr.T.copy(), p), mpk.Vec.from_planes(Y, p), sync=False)
    with pytest.raises(mpk.MPError) as e:
        mpk.check()
    assert e.value.status == 5
    want, st = oracle.dot(p, Xr, recs(Y))
    assert st == oracle.ERR_SPAN
    assert_bitwise(out.planes(), want[None], "dot span error")


@pytest.mark.parametrize("p", (128, 1024))
@pytest.mark.parametrize("n", (5_000, 70_000))
def test_dot_block_spans_and_cap(p, n):
    """One far product among near ones (the wide path), a low and a high
    outlier in different blocks, and a global span of exactly the cap
    (accepted) or one past it (+0 and MP_ERR_SPAN)."""
    mpk = need_gpu()
    X = rand_planes(n, p, 300 + n, zero_frac=0.01, emin=0, emax=0)
    Y = rand_planes(n, p, 400 + n, zero_frac=0.01, emin=0, emax=0)
    Xr = recs(X)
    Yr = recs(Y)

    def shifted(i, by):
        h = Xr[i, 0].view(np.int64)
        return np.int64(h + 2 * by).view(np.uint64)

    lo_i, hi_i, mid_i = n // 7, n - 3, n // 2
    for i in (lo_i, hi_i, mid_i):  # nonzero at the shifted positions
        assert (Xr[i, 0].view(np.int64) >> 1) != oracle.EXP_ZERO
        assert (Yr[i, 0].view(np.int64) >> 1) != oracle.EXP_ZERO
    cases = (((mid_i, 3000),), ((lo_i, -700), (mid_i, 2500)),
             ((lo_i, -(oracle.SPAN_CAP // 2)), (hi_i, oracle.SPAN_CAP // 2)),
             ((lo_i, -(oracle.SPAN_CAP // 2)), (hi_i, oracle.SPAN_CAP // 2 + 1)))
    for shifts in cases:
        Z = Xr.copy()
        for i, by in shifts:
            Z[i, 0] = shifted(i, by)
        want, st = oracle.dot(p, Z, Yr)
        out = mpk.dot(mpk.Vec.from_planes(Z.T.copy(), p), mpk.Vec.from_planes(Y, p), sync=False)
        if st == oracle.ERR_SPAN:
            with pytest.raises(mpk.MPError) as e:
                mpk.check()
            assert e.value.status == 5
        else:
            assert st == oracle.OK
            mpk.check()
        assert_bitwise(out.planes(), want[None], f"dot p={p} n={n} shifts={shifts}")
    assert st == oracle.ERR_SPAN  # the last case is one past the cap


@pytest.mark.parametrize("p", PRECS)
def test_axpy(p):
    mpk = need_gpu()
    n = 10_001
    X = rand_planes(n, p, 81, zero_frac=0.05, emin=-60, emax=60)
    Y = rand_planes(n, p, 82, zero_frac=0.05, emin=-60, emax=60)
    al = rand_planes(1, p, 83, zero_frac=0.0)
    y = mpk.Vec.from_planes(Y, p)
    mpk.axpy(mpk.Vec.from_planes(al, p), mpk.Vec.from_planes(X, p), y)
    want, _ = oracle.axpy(p, recs(al), recs(X), recs(Y))
    assert_bitwise(y.planes(), want, f"axpy p={p}")


def test_repeated_dots_reuse_scratch():
    """Back-to-back dots of different precisions and lengths (the scratch
    span slots are reset by each dot)."""
    mpk = need_gpu()
    for i, p in enumerate((128, 1024, 256, 128, 512)):
        n = 1000 + 997 * i
        X = rand_planes(n, p, 90 + i, zero_frac=0.01, emin=-10 * i, emax=10 * i + 1)
        Y = rand_planes(n, p, 95 + i, zero_frac=0.01)
        got = mpk.dot(mpk.Vec.from_planes(X, p), mpk.Vec.from_planes(Y, p))
        want, _ = oracle.dot(p, recs(X), recs(Y))
        assert_bitwise(got.planes(), want[None], f"dot #{i}")


@pytest.mark.parametrize("p", (128, 1024))
def test_dot_at_the_benchmark_size(p):
    """The exact dot on the benchmark's vectors (n = 10^6, SpMV-workload
    values, the grid-stride path), through mp_dot and mp_dot_noalloc, equal
    to the oracle's exact dot."""
    mpk = need_gpu()
    from paper_1411_2377_gb300 import synth

    n = 1_000_000
    X = synth.random_values(n, p, seed=11, zero_frac=0.0)
    Y = synth.random_values(n, p, seed=12, zero_frac=0.0)
    x, y = mpk.Vec.from_planes(X, p), mpk.Vec.from_planes(Y, p)
    want, st = oracle.dot(p, recs(X), recs(Y))
    assert st == oracle.OK
    assert_bitwise(mpk.dot(x, y).planes(), want[None], f"dot p={p} n=1e6")
    lib = mpk._lib.load()
    out = mpk.Vec.empty(1, p)
    assert lib.mp_dot_noalloc(x.c(), y.c(), out.c(), mpk._stream(None)) == 0
    mpk.check()
    assert_bitwise(out.planes(), want[None], f"dot_noalloc p={p} n=1e6")


@pytest.mark.parametrize("p", (128, 1024))
def test_dot_right_after_a_kernel_that_writes_its_operand(p):
    """The dot kernels are launched programmatically (they may start while
    the previous kernel in the stream finishes and wait on the device for
    it): a dot issued right after a kernel that writes x, on the same stream
    and without a host sync, sees the written x.  Eight rounds, each writing
    a different x, every result against the oracle."""
    mpk = need_gpu()
    import torch

    n = 200_000
    Y = rand_planes(n, p, 91, zero_frac=0.01, emin=-30, emax=30)
    y = mpk.Vec.from_planes(Y, p)
    src = [mpk.Vec.from_planes(rand_planes(n, p, 92 + k, zero_frac=0.01, emin=-30, emax=30), p)
           for k in range(8)]
    x = mpk.Vec.empty(n, p)
    zero = torch.zeros_like(x.t)
    outs = []
    torch.cuda.synchronize()
    for k in range(8):
        torch.bitwise_xor(src[k].t, zero, out=x.t)  # an elementwise kernel writes x
        outs.append(mpk.dot(x, y, sync=False))
    torch.cuda.synchronize()
    for k in range(8):
        want, st = oracle.dot(p, recs(src[k].planes()), recs(Y))
        assert st == oracle.OK
        assert_bitwise(outs[k].planes(), want[None], f"dot after a producer, round {k}")
