"""Device-resident BiCG, GPBiCG, CGS and BiCGSTAB vs the oracle: iteration
counts, status, every iterate's (r_i, r_i) and the final x, bit for bit."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_bitwise, need_gpu, rand_planes, random_csr, recs
from paper_1411_2377_gb300 import synth

pytestmark = pytest.mark.gpu
SOLVERS = {"gpbicg": oracle.gpbicg, "bicg": oracle.bicg, "cgs": oracle.cgs,
           "bicgstab": oracle.bicgstab}


def run_both(mpk, name, rowptr, colidx, vals_planes, b_planes, p, mode, rtol, maxit,
             poll_every=8, x0=None):
    A = mpk.CSR(rowptr, colidx, vals_planes, p, transpose=True)
    b = mpk.Vec.from_planes(b_planes, p)
    x0v = mpk.Vec.from_planes(x0, p) if x0 is not None else None
    fn = getattr(mpk, name)
    x, info = fn(A, b, x0=x0v, rtol=rtol, maxit=maxit, mode=mode, poll_every=poll_every,
                 history=True)
    m = oracle.ORDERED if mode == "ordered" else oracle.EXACT
    x0r = recs(x0) if x0 is not None else oracle.empty(p, len(rowptr) - 1)
    xo, it, st, hist = SOLVERS[name](p, m, rowptr, colidx, recs(vals_planes), recs(b_planes),
                                     x0r, rtol, 0.0, maxit)
    return x, info, xo, it, st, hist


@pytest.mark.parametrize("name", list(SOLVERS))
def test_stencil_64x64_p128_to_1e30(name):
    """The 2-D convection-diffusion system on a 64x64 grid at 128 bits,
    b = A*ones, stopped at relative residual 1e-30: same iteration count,
    same (r_i, r_i) at every iteration, same x."""
    mpk = need_gpu()
    p = 128
    rowptr, colidx, v64 = synth.stencil2d(64, seed=0)
    n = len(rowptr) - 1
    vals = oracle.from_f64(p, v64)
    b, _ = oracle.spmv(p, oracle.EXACT, rowptr, colidx, vals, oracle.from_f64(p, np.ones(n)))
    x, info, xo, it, st, hist = run_both(mpk, name, rowptr, colidx, vals.T.copy(), b.T.copy(), p,
                                         "ordered", 1e-30, 2000)
    assert st == oracle.OK and info["status"] == 0
    assert info["iters"] == it
    assert_bitwise(info["history"].planes(), hist, f"{name} history")
    assert_bitwise(x.planes(), xo, f"{name} x")
    assert info["relres"] <= 1e-30


@pytest.mark.parametrize("name", list(SOLVERS))
@pytest.mark.parametrize("p", (128, 256, 512, 1024))
@pytest.mark.parametrize("mode", ("ordered", "exact"))
def test_random_systems_every_precision(name, p, mode):
    mpk = need_gpu()
    n = 200
    rowptr, colidx = random_csr(n, seed=p + 7, mean_len=6, max_len=20)
    # add a dominant diagonal
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    allr = np.concatenate([rows, np.arange(n)])
    allc = np.concatenate([colidx, np.arange(n)])
    key = np.unique(allr * n + allc)
    rowptr = np.zeros(n + 1, np.int64)
    np.add.at(rowptr, key // n + 1, 1)
    rowptr = np.cumsum(rowptr)
    colidx = (key % n).astype(np.int32)
    V = rand_planes(len(colidx), p, 3, zero_frac=0.0, emin=-1, emax=1)
    Vr = recs(V)
    for i in range(n):
        for k in range(rowptr[i], rowptr[i + 1]):
            if colidx[k] == i:
                Vr[k] = oracle.from_f64(p, [float(12 + i % 5)])[0]
    V = Vr.T.copy()
    b, _ = oracle.spmv(p, oracle.EXACT, rowptr, colidx, Vr, oracle.from_f64(p, np.ones(n)))
    x, info, xo, it, st, hist = run_both(mpk, name, rowptr, colidx, V, b.T.copy(), p, mode,
                                         1e-25, 300, poll_every=3)
    assert (info["status"], info["iters"]) == (st, it)
    assert_bitwise(info["history"].planes(), hist, f"{name} p={p} {mode} history")
    assert_bitwise(x.planes(), xo, f"{name} p={p} {mode} x")


@pytest.mark.parametrize("name", list(SOLVERS))
def test_nonzero_x0_noconv_and_poll_interval(name):
    """x0 != 0 (exact initial residual), maxit reached ("NC"), and a result
    that does not depend on how often the host polls."""
    mpk = need_gpu()
    p = 256
    rowptr, colidx, v64 = synth.stencil2d(12, seed=3)
    n = len(rowptr) - 1
    vals = oracle.from_f64(p, v64)
    b, _ = oracle.spmv(p, oracle.EXACT, rowptr, colidx, vals, oracle.from_f64(p, np.ones(n)))
    X0 = rand_planes(n, p, 5, zero_frac=0.2, emin=-3, emax=3)
    for poll in (1, 5, 64):
        x, info, xo, it, st, hist = run_both(mpk, name, rowptr, colidx, vals.T.copy(), b.T.copy(),
                                             p, "exact", 1e-60, 7, poll_every=poll, x0=X0)
        assert st == oracle.ERR_NOCONV and info["status"] == st and info["iters"] == it == 7
        assert_bitwise(info["history"].planes(), hist, f"{name} history")
        assert_bitwise(x.planes(), xo, f"{name} x poll={poll}")


@pytest.mark.parametrize("name", list(SOLVERS))
def test_breakdown_and_trivial(name):
    mpk = need_gpu()
    p = 128
    rowptr = np.array([0, 1, 2], np.int64)
    colidx = np.array([1, 0], np.int32)
    vals = oracle.from_f64(p, [1.0, 1.0]).T.copy()
    b = oracle.from_f64(p, [1.0, 0.0]).T.copy()
    x, info, xo, it, st, _ = run_both(mpk, name, rowptr, colidx, vals, b, p, "ordered", 1e-30, 10)
    assert st == oracle.ERR_BREAKDOWN and info["status"] == st and info["iters"] == it == 0
    assert_bitwise(x.planes(), xo, "breakdown x")
    zero_b = oracle.empty(p, 2).T.copy()
    x, info, xo, it, st, _ = run_both(mpk, name, rowptr, colidx, vals, zero_b, p, "ordered",
                                      1e-30, 10)
    assert st == oracle.OK and info["status"] == 0 and info["iters"] == 0
    # scaled identity: one step (GPBiCG takes the zeta = eta = 0 reading)
    n = 9
    rp = np.arange(n + 1, dtype=np.int64)
    ci = np.arange(n, dtype=np.int32)
    v = oracle.from_f64(p, np.full(n, 3.0)).T.copy()
    bb = oracle.from_f64(p, np.arange(1.0, n + 1)).T.copy()
    x, info, xo, it, st, _ = run_both(mpk, name, rp, ci, v, bb, p, "exact", 1e-30, 10)
    assert (info["status"], info["iters"]) == (st, it) == (oracle.OK, 1)
    assert_bitwise(x.planes(), xo, "identity x")


@pytest.mark.parametrize("name", ("cgs", "bicgstab"))
def test_transposed_solve_matches_the_oracle_on_the_transpose(name):
    """opts.transpose: the solve with A^T equals the oracle's solve on the
    explicit transpose."""
    mpk = need_gpu()
    p = 256
    rowptr, colidx, v64 = synth.stencil2d(9, seed=4)
    vals = synth.records_to_planes(oracle.from_f64(p, v64))
    n = len(rowptr) - 1
    trp, tci, tv = oracle.transpose(p, rowptr, colidx, recs(vals))
    b, _ = oracle.spmv(p, oracle.EXACT, trp, tci, tv, oracle.from_f64(p, np.ones(n)))
    A = mpk.CSR(rowptr, colidx, vals, p, transpose=True)
    x, info = getattr(mpk, name)(A, mpk.Vec.from_planes(synth.records_to_planes(b), p),
                                 rtol=1e-40, maxit=300, history=True, transpose=True)
    xo, it, st, hist = SOLVERS[name](p, oracle.ORDERED, trp, tci, tv, b, oracle.empty(p, n),
                                     1e-40, 0.0, 300)
    assert (info["iters"], info["status"]) == (it, st)
    assert_bitwise(x.planes(), xo, f"{name} transpose x")
    assert_bitwise(info["history"].planes(), hist, f"{name} transpose history")


@pytest.mark.parametrize("after", (0, 1))
def test_failed_state_read_returns_cuda_status_and_releases_work_memory(after):
    """A CUDA failure while the host reads the solver's device state (after
    the first iteration, after = 0; after the device-side loop, after = 1;
    made on the host by the library's fault hook: nothing faults on the GPU)
    returns MP_ERR_CUDA and gives back the solve's graph, events, stream and
    work memory; the next solve is unaffected and still matches the oracle."""
    import ctypes
    import torch

    mpk = need_gpu()
    lib = mpk._lib.load()
    p = 256
    rowptr, colidx, v64 = synth.stencil2d(16, seed=0)
    n = len(rowptr) - 1
    vals = oracle.from_f64(p, v64)
    b, _ = oracle.spmv(p, oracle.EXACT, rowptr, colidx, vals, oracle.from_f64(p, np.ones(n)))
    A = mpk.CSR(rowptr, colidx, v64, p)
    bv = mpk.Vec.from_planes(synth.records_to_planes(b), p)
    torch.cuda.synchronize()
    used = ctypes.c_int64()
    assert lib.mp_debug_pool_used(ctypes.byref(used)) == 0
    before = used.value
    assert lib.mp_debug_fail(b"solver poll", after) == 0
    try:
        with pytest.raises(mpk.MPError) as e:
            mpk.gpbicg(A, bv, rtol=1e-40, maxit=200, poll_every=1)
    finally:
        lib.mp_debug_fail(None, 0)
    assert e.value.status == 4  # MP_ERR_CUDA
    assert b"reading the solver state" in lib.mp_last_error()
    torch.cuda.synchronize()
    assert lib.mp_debug_pool_used(ctypes.byref(used)) == 0
    assert used.value == before
    x, info = mpk.gpbicg(A, bv, rtol=1e-40, maxit=200)
    xo, it, st, _ = oracle.gpbicg(p, oracle.ORDERED, rowptr, colidx, vals, b,
                                  oracle.empty(p, n), 1e-40, 0.0, 200)
    assert (info["iters"], info["status"]) == (it, st) == (it, oracle.OK)
    assert_bitwise(x.planes(), xo, "x after the failed solve")


@pytest.mark.parametrize("name,after", [("gpbicg", 0), ("gpbicg", 3), ("bicg", 2)])
def test_failed_work_allocation_returns_cuda_status_and_releases_what_it_took(name, after):
    """A failed stream-ordered allocation of the solver's work space (the
    first one, after = 0, or one after others were made; the failure is a
    fake status from the library's host-side fault hook, nothing faults on
    the GPU) returns MP_ERR_CUDA before any iteration and gives back the
    allocations already made; the next solve still matches the oracle."""
    import ctypes
    import torch

    mpk = need_gpu()
    lib = mpk._lib.load()
    p = 256
    rowptr, colidx, v64 = synth.stencil2d(16, seed=1)
    n = len(rowptr) - 1
    vals = oracle.from_f64(p, v64)
    b, _ = oracle.spmv(p, oracle.EXACT, rowptr, colidx, vals, oracle.from_f64(p, np.ones(n)))
    A = mpk.CSR(rowptr, colidx, v64, p, transpose=True)
    bv = mpk.Vec.from_planes(synth.records_to_planes(b), p)
    fn = getattr(mpk, name)
    torch.cuda.synchronize()
    used = ctypes.c_int64()
    assert lib.mp_debug_pool_used(ctypes.byref(used)) == 0
    before = used.value
    assert lib.mp_debug_fail(b"work memory", after) == 0
    try:
        with pytest.raises(mpk.MPError) as e:
            fn(A, bv, rtol=1e-40, maxit=200)
    finally:
        lib.mp_debug_fail(None, 0)
    assert e.value.status == 4  # MP_ERR_CUDA
    assert b"solver work memory" in lib.mp_last_error()
    torch.cuda.synchronize()
    assert lib.mp_debug_pool_used(ctypes.byref(used)) == 0
    assert used.value == before
    x, info = fn(A, bv, rtol=1e-40, maxit=200)
    xo, it, st, _ = SOLVERS[name](p, oracle.ORDERED, rowptr, colidx, vals, b,
                                  oracle.empty(p, n), 1e-40, 0.0, 200)
    assert (info["iters"], info["status"]) == (it, st)
    assert_bitwise(x.planes(), xo, f"{name} x after the failed allocation")


@pytest.mark.parametrize("name", ("gpbicg", "bicg"))
def test_time_limit_ends_the_device_loop(name):
    """time_limit_ms: the device-side loop ends with MP_ERR_TIMEOUT once an
    iteration finishes past the limit (a 1 ms limit on a solve that needs
    far longer); x holds that iterate, equal to the oracle's after the same
    number of iterations; the next solve without a limit is unaffected."""
    import torch

    mpk = need_gpu()
    p = 1024
    rowptr, colidx, v64 = synth.stencil2d(40, seed=0)
    n = len(rowptr) - 1
    vals = oracle.from_f64(p, v64)
    b, _ = oracle.spmv(p, oracle.EXACT, rowptr, colidx, vals, oracle.from_f64(p, np.ones(n)))
    A = mpk.CSR(rowptr, colidx, v64, p, transpose=True)
    bv = mpk.Vec.from_planes(synth.records_to_planes(b), p)
    fn = getattr(mpk, name)
    x, info = fn(A, bv, rtol=1e-300, maxit=100_000, time_limit_ms=1)
    assert info["status"] == 8  # MP_ERR_TIMEOUT
    it = info["iters"]
    assert 1 <= it < 100_000
    xo, ito, sto, _ = SOLVERS[name](p, oracle.ORDERED, rowptr, colidx, vals, b,
                                    oracle.empty(p, n), 1e-300, 0.0, it)
    assert (ito, sto) == (it, oracle.ERR_NOCONV)
    assert_bitwise(x.planes(), xo, "x at the time limit")
    torch.cuda.synchronize()
    x2, info2 = fn(A, bv, rtol=1e-30, maxit=5000)
    xo2, it2, st2, _ = SOLVERS[name](p, oracle.ORDERED, rowptr, colidx, vals, b,
                                     oracle.empty(p, n), 1e-30, 0.0, 5000)
    assert (info2["iters"], info2["status"]) == (it2, st2)
    assert_bitwise(x2.planes(), xo2, "x after the timed-out solve")
