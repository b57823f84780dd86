"""CPU oracle for the p-bit CSR SpMV / exact dot / BiCG / GPBiCG path.

TEST INFRASTRUCTURE ONLY.  This package wraps ``libmpo.so`` and
``libmpo_wide.so`` (plain C, both built from ``oracle/mpo.c``; the wide build
holds mantissas up to 8192 bits).  Only the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import it; the product package never does.

Values are exchanged as numpy ``uint64`` arrays of shape ``(n, L+1)`` with
``L = p // 64``: column 0 is the head word ``exp*2 + sign``, columns 1..L are
the mantissa limbs, least significant first (see ``mpo.h``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import build_oracle, lib_path

OK, ERR_ARG, ERR_PREC, ERR_SPAN, ERR_BREAKDOWN, ERR_NOCONV, ERR_DIVZERO = 0, 1, 2, 5, 6, 7, 9
ORDERED, EXACT = 0, 1
OP_MUL, OP_ADD, OP_SUB, OP_DIV = 0, 1, 2, 3
EXP_ZERO = -(1 << 61)
SPAN_CAP = 16384

_lib = {}

_u64p = ctypes.POINTER(ctypes.c_uint64)
_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_f64p = ctypes.POINTER(ctypes.c_double)
_i32 = ctypes.c_int
_i64 = ctypes.c_int64


def _load(p=0):
    """The library for precision p: libmpo.so up to 1024 bits, the wide
    build (same source, 256-word mantissas) above."""
    wide = p > 1024
    if _lib.get(wide) is not None:
        return _lib[wide]
    path = lib_path(wide)
    if not os.path.exists(path):
        build_oracle()
    lib = ctypes.CDLL(path)
    sig = {
        "mpo_ewise": [_i32, _i32, _i64, _u64p, _u64p, _u64p],
        "mpo_cmp": [_i32, _u64p, _u64p, ctypes.POINTER(ctypes.c_int)],
        "mpo_from_f64": [_i32, _i64, _f64p, _u64p],
        "mpo_to_f64": [_i32, _i64, _u64p, _f64p],
        "mpo_spmv_rows": [_i32, _i32, _i64, _i64p, _i32p, _u64p, _u64p, _u64p, _i64, _i64],
        "mpo_spmv": [_i32, _i32, _i64, _i64p, _i32p, _u64p, _u64p, _u64p],
        "mpo_spmv_t": [_i32, _i32, _i64, _i64p, _i32p, _u64p, _u64p, _u64p],
        "mpo_transpose": [_i32, _i64, _i64p, _i32p, _u64p, _i64p, _i32p, _u64p],
        "mpo_dot": [_i32, _i64, _u64p, _u64p, _u64p],
        "mpo_axpy": [_i32, _i64, _u64p, _u64p, _u64p],
        "mpo_residual": [_i32, _i64, _i64p, _i32p, _u64p, _u64p, _u64p, _u64p],
        "mpo_bicg": [_i32, _i32, _i64, _i64p, _i32p, _u64p, _u64p, _u64p,
                     ctypes.c_double, ctypes.c_double, _i64, _i64p, _u64p],
        "mpo_gpbicg": [_i32, _i32, _i64, _i64p, _i32p, _u64p, _u64p, _u64p,
                       ctypes.c_double, ctypes.c_double, _i64, _i64p, _u64p],
        "mpo_cgs": [_i32, _i32, _i64, _i64p, _i32p, _u64p, _u64p, _u64p,
                    ctypes.c_double, ctypes.c_double, _i64, _i64p, _u64p],
        "mpo_bicgstab": [_i32, _i32, _i64, _i64p, _i32p, _u64p, _u64p, _u64p,
                         ctypes.c_double, ctypes.c_double, _i64, _i64p, _u64p],
        "mpo_bicgstab_ilu0": [_i32, _i32, _i64, _i64p, _i32p, _u64p, _u64p, _u64p,
                              ctypes.c_double, ctypes.c_double, _i64, _i64p, _u64p],
        "mpo_bicgstab_ilu0_right": [_i32, _i32, _i64, _i64p, _i32p, _u64p, _u64p, _u64p,
                                    ctypes.c_double, ctypes.c_double, _i64, _i64p, _u64p],
        "mpo_ilu0": [_i32, _i64, _i64p, _i32p, _u64p, _u64p],
        "mpo_ilu0_apply": [_i32, _i64, _i64p, _i32p, _u64p, _u64p, _u64p],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    _lib[wide] = lib
    return lib


def _p(a, t):
    return a.ctypes.data_as(t)


def _recs(a, p):
    L = p // 64
    a = np.ascontiguousarray(a, dtype=np.uint64)
    if a.ndim == 1:
        a = a.reshape(-1, L + 1)
    assert a.shape[-1] == L + 1, (a.shape, p)
    return a


def _csr(rowptr, colidx):
    return (np.ascontiguousarray(rowptr, dtype=np.int64),
            np.ascontiguousarray(colidx, dtype=np.int32))


def empty(p, n):
    """n records of +0."""
    r = np.zeros((n, p // 64 + 1), dtype=np.uint64)
    r[:, 0] = np.uint64((EXP_ZERO * 2) & ((1 << 64) - 1))
    return r


def ewise(p, op, a, b):
    a, b = _recs(a, p), _recs(b, p)
    r = np.empty_like(a)
    st = _load(p).mpo_ewise(p, op, a.shape[0], _p(a, _u64p), _p(b, _u64p), _p(r, _u64p))
    return r, st


def cmp(p, a, b):
    a, b = _recs(a, p), _recs(b, p)
    out = ctypes.c_int(0)
    st = _load(p).mpo_cmp(p, _p(a, _u64p), _p(b, _u64p), ctypes.byref(out))
    if st:
        raise ValueError(f"mpo_cmp status {st}")
    return out.value


def from_f64(p, d):
    d = np.ascontiguousarray(d, dtype=np.float64).ravel()
    r = np.empty((d.shape[0], p // 64 + 1), dtype=np.uint64)
    st = _load(p).mpo_from_f64(p, d.shape[0], _p(d, _f64p), _p(r, _u64p))
    if st:
        raise ValueError(f"mpo_from_f64 status {st}")
    return r


def to_f64(p, a):
    a = _recs(a, p)
    d = np.empty(a.shape[0], dtype=np.float64)
    st = _load(p).mpo_to_f64(p, a.shape[0], _p(a, _u64p), _p(d, _f64p))
    if st:
        raise ValueError(f"mpo_to_f64 status {st}")
    return d


def spmv(p, mode, rowptr, colidx, vals, x, rows=None, out=None):
    """y = A x (all rows, or rows[0]:rows[1] with the rest left as +0).
    out: optional (n, p/64 + 1) uint64 C-contiguous record array written in
    place (only the computed rows), so that callers splitting the rows over
    threads share one result."""
    rowptr, colidx = _csr(rowptr, colidx)
    vals, x = _recs(vals, p), _recs(x, p)
    n = rowptr.shape[0] - 1
    if out is None:
        y = empty(p, n)
    else:
        if (out.dtype != np.uint64 or out.shape != (n, p // 64 + 1)
                or not out.flags["C_CONTIGUOUS"]):
            raise ValueError("out must be a C-contiguous (n, p/64 + 1) uint64 array")
        y = out
    r0, r1 = (0, n) if rows is None else rows
    st = _load(p).mpo_spmv_rows(p, mode, n, _p(rowptr, _i64p), _p(colidx, _i32p),
                               _p(vals, _u64p), _p(x, _u64p), _p(y, _u64p), r0, r1)
    return y, st


def spmv_t(p, mode, rowptr, colidx, vals, x):
    rowptr, colidx = _csr(rowptr, colidx)
    vals, x = _recs(vals, p), _recs(x, p)
    n = rowptr.shape[0] - 1
    y = empty(p, n)
    st = _load(p).mpo_spmv_t(p, mode, n, _p(rowptr, _i64p), _p(colidx, _i32p),
                            _p(vals, _u64p), _p(x, _u64p), _p(y, _u64p))
    return y, st


def transpose(p, rowptr, colidx, vals):
    rowptr, colidx = _csr(rowptr, colidx)
    vals = _recs(vals, p)
    n = rowptr.shape[0] - 1
    nnz = int(rowptr[-1])
    trp = np.empty(n + 1, dtype=np.int64)
    tci = np.empty(max(nnz, 1), dtype=np.int32)
    tv = np.empty((max(nnz, 1), p // 64 + 1), dtype=np.uint64)
    st = _load(p).mpo_transpose(p, n, _p(rowptr, _i64p), _p(colidx, _i32p), _p(vals, _u64p),
                               _p(trp, _i64p), _p(tci, _i32p), _p(tv, _u64p))
    if st:
        raise ValueError(f"mpo_transpose status {st}")
    return trp, tci[:nnz], tv[:nnz]


def dot(p, x, y):
    x, y = _recs(x, p), _recs(y, p)
    out = empty(p, 1)
    st = _load(p).mpo_dot(p, x.shape[0], _p(x, _u64p), _p(y, _u64p), _p(out, _u64p))
    return out[0], st


def axpy(p, alpha, x, y):
    alpha, x = _recs(alpha, p), _recs(x, p)
    y = _recs(y, p).copy()
    st = _load(p).mpo_axpy(p, x.shape[0], _p(alpha, _u64p), _p(x, _u64p), _p(y, _u64p))
    return y, st


def residual(p, rowptr, colidx, vals, b, x):
    rowptr, colidx = _csr(rowptr, colidx)
    vals, b, x = _recs(vals, p), _recs(b, p), _recs(x, p)
    r = np.empty_like(b)
    st = _load(p).mpo_residual(p, b.shape[0], _p(rowptr, _i64p), _p(colidx, _i32p),
                              _p(vals, _u64p), _p(b, _u64p), _p(x, _u64p), _p(r, _u64p))
    return r, st


def _solve(fn, p, mode, rowptr, colidx, vals, b, x0, rtol, atol, maxit):
    rowptr, colidx = _csr(rowptr, colidx)
    vals, b = _recs(vals, p), _recs(b, p)
    x = _recs(x0, p).copy()
    hist = np.zeros((max(maxit, 1), p // 64 + 1), dtype=np.uint64)
    iters = ctypes.c_int64(0)
    st = fn(p, mode, b.shape[0], _p(rowptr, _i64p), _p(colidx, _i32p), _p(vals, _u64p),
            _p(b, _u64p), _p(x, _u64p), float(rtol), float(atol), int(maxit),
            ctypes.byref(iters), _p(hist, _u64p))
    return x, iters.value, st, hist[: iters.value]


def bicg(p, mode, rowptr, colidx, vals, b, x0, rtol, atol, maxit):
    """Returns (x, iterations, status, history of (r_i, r_i))."""
    return _solve(_load(p).mpo_bicg, p, mode, rowptr, colidx, vals, b, x0, rtol, atol, maxit)


def gpbicg(p, mode, rowptr, colidx, vals, b, x0, rtol, atol, maxit):
    """Returns (x, iterations, status, history of (r_i, r_i))."""
    return _solve(_load(p).mpo_gpbicg, p, mode, rowptr, colidx, vals, b, x0, rtol, atol, maxit)


def cgs(p, mode, rowptr, colidx, vals, b, x0, rtol, atol, maxit):
    """CGS (textbook form).  Returns (x, iterations, status, history of (r_i, r_i))."""
    return _solve(_load(p).mpo_cgs, p, mode, rowptr, colidx, vals, b, x0, rtol, atol, maxit)


def bicgstab(p, mode, rowptr, colidx, vals, b, x0, rtol, atol, maxit):
    """BiCGSTAB (textbook form).  Returns (x, iterations, status, history of (r_i, r_i))."""
    return _solve(_load(p).mpo_bicgstab, p, mode, rowptr, colidx, vals, b, x0, rtol, atol, maxit)


def ilu0(p, rowptr, colidx, vals):
    """ILU(0) factors in A's CSR order (records).  Returns (lu, status)."""
    rowptr, colidx = _csr(rowptr, colidx)
    vals = _recs(vals, p)
    lu = np.empty_like(vals)
    st = _load(p).mpo_ilu0(p, rowptr.shape[0] - 1, _p(rowptr, _i64p), _p(colidx, _i32p),
                          _p(vals, _u64p), _p(lu, _u64p))
    return lu, st


def ilu0_apply(p, rowptr, colidx, lu, r):
    """w = (LU)^{-1} r.  Returns (w, status)."""
    rowptr, colidx = _csr(rowptr, colidx)
    lu, r = _recs(lu, p), _recs(r, p)
    w = np.empty_like(r)
    st = _load(p).mpo_ilu0_apply(p, rowptr.shape[0] - 1, _p(rowptr, _i64p), _p(colidx, _i32p),
                                _p(lu, _u64p), _p(r, _u64p), _p(w, _u64p))
    return w, st


def bicgstab_ilu0(p, mode, rowptr, colidx, vals, b, x0, rtol, atol, maxit, side="left"):
    """BiCGSTAB preconditioned with ILU(0) K = LU.  side="left" (Section 4.2):
    BiCGSTAB on K^{-1}A x = K^{-1}b, the history holds (r^_i, r^_i) of the
    preconditioned residual r^ = K^{-1}(b - A x); side="right": r stays
    b - A x and the history holds (r_i, r_i).  Returns (x, iterations,
    status, history)."""
    lib = _load(p)
    if side not in ("left", "right"):
        raise ValueError(side)
    fn = lib.mpo_bicgstab_ilu0 if side == "left" else lib.mpo_bicgstab_ilu0_right
    return _solve(fn, p, mode, rowptr, colidx, vals, b, x0, rtol, atol, maxit)
