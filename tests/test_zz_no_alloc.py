"""mp_dot_noalloc: the exact dot product for callers that cannot let a library
allocate device memory -- processes whose GPU memory belongs to another
allocator or is held to a fixed budget, where a cudaMalloc would fail or break
the budget, and latency-bound callers that must avoid the synchronisation
cudaMalloc/cudaFree can cause.  Its scratch is one fixed device array inside
the library that every call reuses, so its results must equal mp_dot's bit
for bit on consecutive calls, whatever the previous call left in the array.

The length limit is refused on the host before any device work; that check
runs without a GPU in test_abi_cpu.py.  This file is collected last, so a run
that stops at the first failure has already run every other test.  It passes
alone in a fresh process as well: the first mp_dot_noalloc call on the device
does the array's set-up."""

import numpy as np
import pytest

import oracle
from gpu_util import need_gpu, rand_planes, recs

pytestmark = pytest.mark.gpu


def _dot(lib, mpk, name, x, y):
    out = mpk.Vec.empty(1, x.prec)
    st = getattr(lib, name)(x.c(), y.c(), out.c(), mpk._stream(None))
    assert st == 0, (name, st, lib.mp_last_error())
    mpk.check()
    return out.planes().copy()


def test_noalloc_dot_matches_dot_on_two_calls_in_a_row():
    mpk = need_gpu()
    lib = mpk._lib.load()
    # first call: p = 1024 with a span beyond the per-warp window (wide path);
    # second call: p = 128, short span (fast path), smaller grid
    cases = [(1024, 200_003, -1500, 1500, 501), (128, 50_000, -30, 30, 502)]
    vecs, refs = [], []
    for p, n, lo, hi, seed in cases:
        x = mpk.Vec.from_planes(rand_planes(n, p, seed, zero_frac=0.02, emin=lo, emax=hi), p)
        y = mpk.Vec.from_planes(rand_planes(n, p, seed + 7, zero_frac=0.02, emin=lo, emax=hi), p)
        vecs.append((x, y))
        refs.append(_dot(lib, mpk, "mp_dot", x, y))
    got = [_dot(lib, mpk, "mp_dot_noalloc", x, y) for x, y in vecs]  # two calls in a row
    for g, r, case in zip(got, refs, cases):
        assert np.array_equal(g, r), case
    # and once more after the smaller call, to see no state carried over
    again = _dot(lib, mpk, "mp_dot_noalloc", *vecs[0])
    assert np.array_equal(again, refs[0])
    # both entry points against the oracle's exact dot (one rounding)
    for g, (x, y), (p, *_rest) in zip(got, vecs, cases):
        want, st = oracle.dot(p, recs(x.planes()), recs(y.planes()))
        assert st == oracle.OK
        assert np.array_equal(np.ascontiguousarray(g.T)[0], want), p
