"""Batched GPBiCG: every instance of a batch must equal the oracle's GPBiCG
on that instance alone, and mp_gpbicg's (iterations, status and x, bit for
bit), including instances that exit at once, break down, or hit the
iteration limit."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_bitwise, need_gpu
from paper_1411_2377_gb300 import synth


def _instances():
    sys = [synth.stencil2d(5, seed=1), synth.stencil2d(9, seed=2), synth.stencil3d(3, seed=3, decades=0.0),
           synth.stencil3d(4, seed=4, decades=20.0),   # row-scaled: slow, may hit maxit
           (np.array([0, 1, 2], np.int64), np.array([1, 0], np.int32), np.array([1.0, 1.0])),
           synth.stencil2d(7, seed=5)]
    # (system index, rhs scale): the [[0,1],[1,0]] system with b = e1 breaks down,
    # scale 0 gives b = 0 (converged before the first iteration)
    plan = [(0, 1.0), (1, 1.0), (1, 2.0), (2, 1.0), (3, 1.0), (4, None), (5, 0.0), (5, 3.0)]
    return sys, plan


pytestmark = pytest.mark.gpu


def _rhs(systems, plan, p):
    """Each instance's b, formed by the oracle: RN(A (scale * ones)) exactly
    rounded, or e1 (the breakdown system)."""
    out = []
    for i, scale in plan:
        rp, ci, va = systems[i]
        n = len(rp) - 1
        if scale is None:
            rhs = np.zeros(n)
            rhs[0] = 1.0
            out.append(oracle.from_f64(p, rhs))
        else:
            b, st = oracle.spmv(p, oracle.EXACT, rp, ci, oracle.from_f64(p, va),
                                oracle.from_f64(p, np.full(n, scale)))
            assert st == oracle.OK
            out.append(b)
    return out


@pytest.mark.parametrize("p", (128, 256))
@pytest.mark.parametrize("mode", ("ordered", "exact"))
def test_batched_matches_the_oracle_and_single_solves(p, mode):
    """Every instance's iterations, status and x equal the oracle's GPBiCG on
    that instance alone, and mp_gpbicg's (bit for bit)."""
    mpk = need_gpu()
    import torch

    systems, plan = _instances()
    inst = [systems[i] for i, _ in plan]
    B = mpk.Batch(inst, p)
    b = mpk.Vec.zeros(B.n, p)
    rhs = _rhs(systems, plan, p)
    for k, bk in enumerate(rhs):
        o0, o1 = int(B.offsets[k]), int(B.offsets[k + 1])
        b.t[:, o0:o1] = torch.from_numpy(np.ascontiguousarray(bk.T).view(np.int64)).to(b.t.device)
    maxit = 300
    om = oracle.ORDERED if mode == "ordered" else oracle.EXACT
    x, infos = mpk.batch_gpbicg(B, b, rtol=1e-25, maxit=maxit, mode=mode, poll_every=5)
    statuses = set()
    for k, ((i, _), bk) in enumerate(zip(plan, rhs)):
        rp, ci, va = systems[i]
        n = len(rp) - 1
        xo, it, st, _ = oracle.gpbicg(p, om, rp, ci, oracle.from_f64(p, va), bk,
                                      oracle.empty(p, n), 1e-25, 0.0, maxit)
        o0, o1 = int(B.offsets[k]), int(B.offsets[k + 1])
        assert (infos[k]["iters"], infos[k]["status"]) == (it, st), k
        assert_bitwise(x.t[:, o0:o1].cpu().numpy().view(np.uint64), xo, f"instance {k}")
        A = mpk.CSR(rp, ci, va, p)
        xs, info = mpk.gpbicg(A, mpk.Vec.from_planes(np.ascontiguousarray(bk.T), p),
                              rtol=1e-25, maxit=maxit, mode=mode)
        assert (info["iters"], info["status"]) == (it, st), k
        assert torch.equal(x.t[:, o0:o1].cpu(), xs.t.cpu()), k
        statuses.add(st)
    assert {oracle.OK, oracle.ERR_BREAKDOWN} <= statuses


def test_batch_matrix_configuration_keeps_results():
    """The batch's block-diagonal matrix takes launch configurations like any
    matrix (the autotuner included); the batched solve's iterates do not
    change with them."""
    mpk = need_gpu()
    import torch

    from paper_1411_2377_gb300 import tune

    systems, plan = _instances()
    inst = [systems[i] for i, _ in plan[:4]]
    p = 256
    B = mpk.Batch(inst, p)
    b = mpk.Vec.zeros(B.n, p)
    for k, (rp, ci, va) in enumerate(inst):
        A = mpk.CSR(rp, ci, va, p)
        n = len(rp) - 1
        bk = mpk.spmv(A, mpk.Vec.from_f64(np.full(n, 1.0 + k), p), mode="exact")
        b.t[:, int(B.offsets[k]):int(B.offsets[k + 1])] = bk.t
    x0, i0 = mpk.batch_gpbicg(B, b, rtol=1e-25, maxit=200, mode="ordered")
    M = B.matrix()
    assert M.info()["n"] == B.n
    for cfg in ((64, 0, -1), (256, 3, 50), (128, 6, -1)):
        M.set_config("ordered", *cfg)
        x1, i1 = mpk.batch_gpbicg(B, b, rtol=1e-25, maxit=200, mode="ordered")
        assert [(a["iters"], a["status"]) for a in i1] == [(a["iters"], a["status"]) for a in i0]
        assert torch.equal(x1.t.cpu(), x0.t.cpu()), cfg
    r = tune.autotune(M, modes=("ordered",), reps=1, cache=None)["ordered"]
    assert M.get_config("ordered")["threads_per_block"] == r["threads_per_block"]
    x2, _ = mpk.batch_gpbicg(B, b, rtol=1e-25, maxit=200, mode="ordered")
    assert torch.equal(x2.t.cpu(), x0.t.cpu())
    M.close()  # a borrowed handle: closing it must not free the batch's matrix
    x3, _ = mpk.batch_gpbicg(B, b, rtol=1e-25, maxit=200, mode="ordered")
    assert torch.equal(x3.t.cpu(), x0.t.cpu())


def test_batch_time_limit_ends_the_device_loop():
    """time_limit_ms on the batched solve: instances still running when an
    iteration ends past the limit stop with MP_ERR_TIMEOUT, each holding the
    iterate the oracle reaches in the same number of iterations (it reports
    NC there); instances that finished before keep their own status."""
    mpk = need_gpu()
    import torch

    p = 512
    systems = [synth.stencil2d(24, seed=11), synth.stencil2d(3, seed=12)]
    plan = [(0, 1.0), (1, 1.0), (0, 2.0)]
    inst = [systems[i] for i, _ in plan]
    B = mpk.Batch(inst, p)
    b = mpk.Vec.zeros(B.n, p)
    rhs = _rhs(systems, plan, p)
    for k, bk in enumerate(rhs):
        o0, o1 = int(B.offsets[k]), int(B.offsets[k + 1])
        b.t[:, o0:o1] = torch.from_numpy(np.ascontiguousarray(bk.T).view(np.int64)).to(b.t.device)
    x, infos = mpk.batch_gpbicg(B, b, rtol=1e-300, maxit=100_000, time_limit_ms=1)
    statuses = [i["status"] for i in infos]
    assert 8 in statuses  # MP_ERR_TIMEOUT
    for k, ((i, _), bk) in enumerate(zip(plan, rhs)):
        rp, ci, va = systems[i]
        n = len(rp) - 1
        it = infos[k]["iters"]
        xo, ito, sto, _ = oracle.gpbicg(p, oracle.ORDERED, rp, ci, oracle.from_f64(p, va), bk,
                                        oracle.empty(p, n), 1e-300, 0.0, max(it, 0))
        if infos[k]["status"] == 8:
            assert it >= 1 and (ito, sto) == (it, oracle.ERR_NOCONV)
        else:
            assert (ito, sto) == (it, infos[k]["status"])
        o0, o1 = int(B.offsets[k]), int(B.offsets[k + 1])
        assert_bitwise(x.t[:, o0:o1].cpu().numpy().view(np.uint64), xo, f"instance {k}")
