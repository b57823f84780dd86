"""Helpers shared by the GPU parity tests (inputs come from the seeded
generators; expectations from the oracle)."""
import numpy as np
import pytest

from paper_1411_2377_gb300 import synth


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("a GPU test ran without a CUDA device")
    import paper_1411_2377_gb300 as mpk
    from paper_1411_2377_gb300 import build

    build.build()
    mpk._lib.load()
    return mpk


def rand_planes(n, p, seed, zero_frac=0.05, emin=-40, emax=40):
    return synth.random_values(n, p, seed, zero_frac=zero_frac, emin=emin, emax=emax)


def recs(planes):
    return synth.planes_to_records(planes)


def assert_bitwise(got_planes, want_records, what=""):
    got = np.ascontiguousarray(np.asarray(got_planes).T)
    want = np.asarray(want_records)
    assert got.shape == want.shape, (got.shape, want.shape)
    bad = np.nonzero(np.any(got != want, axis=1))[0]
    assert bad.size == 0, f"{what}: {bad.size} mismatches, first at {bad[:5]}: " \
                          f"got {got[bad[0]]} want {want[bad[0]]}"


def random_csr(n, seed, mean_len=12, max_len=96, band=None, empty_every=0):
    """A CSR pattern with lognormal row lengths, a few long rows and empty
    rows, columns sorted."""
    i = np.arange(n)
    z = synth.normal(seed, 1, 2, i)
    ln = np.clip(np.rint(np.exp(np.log(mean_len) - 0.5 + z)), 0, min(max_len, n)).astype(np.int64)
    if empty_every:
        ln[::empty_every] = 0
    rowptr = np.zeros(n + 1, np.int64)
    np.cumsum(ln, out=rowptr[1:])
    cols = []
    for r in range(n):
        u = synth.uniform(seed, 3, np.arange(4 * ln[r] + 8) + r * 100003)
        if band is None:
            c = np.unique((u * n).astype(np.int64))
        else:
            lo, hi = max(0, r - band), min(n - 1, r + band)
            c = np.unique(lo + (u * (hi - lo + 1)).astype(np.int64))
        c = c[: ln[r]]
        ln[r] = len(c)
        cols.append(c)
    rowptr = np.zeros(n + 1, np.int64)
    np.cumsum(ln, out=rowptr[1:])
    colidx = np.concatenate(cols).astype(np.int32) if cols else np.zeros(0, np.int32)
    return rowptr, colidx


def oracle_spmv_threads(oracle, p, mode, rowptr, colidx, vals_recs, x_recs, threads=None):
    """The oracle's y = A x over all rows, split into contiguous row ranges of
    about equal nonzeros run on host threads (rows are independent and the C
    oracle releases the interpreter lock, so the result equals one call's)."""
    import os
    from concurrent.futures import ThreadPoolExecutor

    n = len(rowptr) - 1
    threads = threads or max(1, min(32, os.cpu_count() or 1))
    y = oracle.empty(p, n)
    nnz = int(rowptr[-1])
    cuts = np.searchsorted(rowptr, np.linspace(0, nnz, threads + 1))
    cuts = np.clip(cuts, 0, n)
    cuts[0], cuts[-1] = 0, n
    ranges = [(int(u), int(v)) for u, v in zip(cuts[:-1], cuts[1:]) if v > u]
    with ThreadPoolExecutor(max(1, len(ranges))) as ex:
        sts = list(ex.map(lambda r: oracle.spmv(p, mode, rowptr, colidx, vals_recs, x_recs,
                                                rows=r, out=y)[1], ranges))
    assert all(st == oracle.OK for st in sts), sts
    return y
