"""paper_1411_2377_gb300 -- p-bit CSR SpMV, exact dot products and the BiCG /
GPBiCG solvers of Kouya's multiple-precision sparse Krylov paper, on GB300.

The compute path is the native library libmpkrylov.so (hand-written sm_103a
CUDA behind a C ABI, include/mpkrylov.h); this module only marshals
arguments.  PyTorch provides device memory and the current stream.

Surface: :class:`CSR` (with its transpose, launch configuration and tuner),
:class:`Vec`, :func:`spmv` / :func:`spmv_t` (ORDERED or EXACT rows),
:func:`residual`, :func:`dot`, :func:`axpy`, :func:`ewise`; the solvers
:func:`bicg`, :func:`gpbicg`, :func:`cgs`, :func:`bicgstab`,
:func:`bicgstab_ilu0` (with :class:`ILU0`); mixed-precision refinement,
batched solves (:class:`Batch`), the dense MV and the differentiable solve
(``autograd``).  Precisions: 128, 256, 512, 1024 bits everywhere; 2048,
4096, 8192 bits for the products, residual, dot, axpy, conversions and the
four unpreconditioned solvers.

Vectors (:class:`Vec`) hold p-bit values as ``L+1`` planes of 64-bit words
(``L = p // 64``) in a ``torch.int64`` CUDA tensor of shape ``(L+1, n)``:
plane 0 the head words ``exp*2 + sign``, planes 1..L the mantissa limbs,
least significant first.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import (EXP_ZERO, MP_EXACT, MP_OP_ADD, MP_OP_DIV, MP_OP_MUL, MP_OP_SUB,  # noqa: F401
                   MP_ORDERED, SPAN_CAP)

__all__ = ["MPError", "Vec", "CSR", "spmv", "spmv_t", "residual", "dot", "axpy", "ewise",
           "bicg", "gpbicg", "csr_grad", "check", "launch_count", "imad_probe", "MODES"]

MODES = {"ordered": MP_ORDERED, "exact": MP_EXACT, MP_ORDERED: MP_ORDERED, MP_EXACT: MP_EXACT}


class MPError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = _lib.load()
        msg = lib.mp_status_string(status).decode()
        detail = lib.mp_last_error().decode()
        super().__init__(f"{where}: {msg} ({detail})")
        self.status = status


def _torch():
    import torch

    return torch


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ok(status: int, where: str):
    if status != 0:
        raise MPError(status, where)


def check(stream=None):
    """Waits for the stream and raises if a kernel recorded an error."""
    _ok(_lib.load().mp_check(_stream(stream)), "device status")


def launch_count(reset: bool = False) -> int:
    return int(_lib.load().mp_launch_count(1 if reset else 0))


def imad_probe(stream=None) -> float:
    """32x32->64 multiply-adds per second measured on the current GPU."""
    rate = ctypes.c_double(0.0)
    _ok(_lib.load().mp_imad_probe(ctypes.byref(rate), _stream(stream)), "mp_imad_probe")
    return rate.value


def _csr_arrays(rowptr, colidx):
    """rowptr and colidx as the library reads them, contiguous int64 and
    int32; raises ValueError unless colidx holds rowptr[-1] entries (the
    library reads that many host words and checks their contents)."""
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    colidx = np.ascontiguousarray(colidx, dtype=np.int32)
    if rowptr.ndim != 1 or rowptr.shape[0] < 1:
        raise ValueError("rowptr holds n + 1 >= 1 offsets")
    nnz = int(rowptr[-1])
    if colidx.ndim != 1 or colidx.shape[0] != max(nnz, 0):
        raise ValueError(f"colidx holds rowptr[-1] = {nnz} column indices; got "
                         f"shape {colidx.shape}")
    return rowptr, colidx


class Vec:
    """n p-bit values on the GPU (planes of a (L+1, n) int64 tensor)."""

    def __init__(self, tensor, prec: int):
        torch = _torch()
        L = prec // 64
        if tensor.dtype != torch.int64 or tensor.dim() != 2 or tensor.shape[0] != L + 1:
            raise ValueError(f"a {prec}-bit vector is an int64 tensor of shape ({L + 1}, n); got "
                             f"{tuple(tensor.shape)} {tensor.dtype}")
        if not tensor.is_cuda or tensor.stride(1) != 1:
            raise ValueError("a vector's planes are a CUDA tensor with unit stride along n")
        self.t = tensor
        self.prec = prec

    @property
    def n(self) -> int:
        return int(self.t.shape[1])

    def c(self) -> _lib.MpVec:
        ld = self.t.stride(0) if self.n > 0 else max(self.n, 1)
        return _lib.MpVec(self.n, self.prec, max(ld, self.n), self.t.data_ptr())

    @classmethod
    def empty(cls, n: int, prec: int, device="cuda"):
        torch = _torch()
        return cls(torch.empty((prec // 64 + 1, n), dtype=torch.int64, device=device), prec)

    @classmethod
    def zeros(cls, n: int, prec: int, device="cuda"):
        v = cls.empty(n, prec, device)
        v.t.zero_()
        v.t[0].fill_(EXP_ZERO * 2)
        return v

    @classmethod
    def from_planes(cls, planes: np.ndarray, prec: int, device="cuda"):
        torch = _torch()
        a = np.ascontiguousarray(planes, dtype=np.uint64).view(np.int64)
        return cls(torch.from_numpy(a).to(device), prec)

    @classmethod
    def from_f64(cls, d, prec: int, stream=None):
        """Exact conversion of doubles (a CUDA float64 tensor or array)."""
        torch = _torch()
        d = torch.as_tensor(d, dtype=torch.float64).to("cuda").contiguous()
        v = cls.empty(d.numel(), prec)
        _ok(_lib.load().mp_vec_from_f64(ctypes.c_void_p(d.data_ptr()), v.c(), _stream(stream)),
            "mp_vec_from_f64")
        check(stream)
        return v

    def to_f64(self, stream=None):
        torch = _torch()
        d = torch.empty(self.n, dtype=torch.float64, device=self.t.device)
        _ok(_lib.load().mp_vec_to_f64(self.c(), ctypes.c_void_p(d.data_ptr()), _stream(stream)),
            "mp_vec_to_f64")
        return d

    def planes(self) -> np.ndarray:
        """(L+1, n) uint64 planes on the host."""
        return self.t.cpu().numpy().view(np.uint64)

    def records(self) -> np.ndarray:
        """(n, L+1) uint64 records (value-major) on the host."""
        return np.ascontiguousarray(self.planes().T)

    def clone(self):
        return Vec(self.t.clone(), self.prec)


class CSR:
    """A p-bit CSR matrix resident on the GPU (Section 2's sparse storage)."""

    def __init__(self, rowptr, colidx, values, prec: int, transpose: bool = False, stream=None):
        """values: (L+1, nnz) uint64 planes, or float64 values (converted
        exactly to p bits)."""
        lib = _lib.load()
        rowptr, colidx = _csr_arrays(rowptr, colidx)
        n = rowptr.shape[0] - 1
        handle = ctypes.c_void_p()
        flags = _lib.MP_CSR_TRANSPOSE if transpose else 0
        values = np.asarray(values)
        if values.dtype == np.float64:
            vals = np.ascontiguousarray(values)
            if vals.shape != colidx.shape:
                raise ValueError(f"{colidx.shape[0]} double values expected; got shape {vals.shape}")
            st = lib.mp_csr_create_f64(n, rowptr.ctypes.data, colidx.ctypes.data,
                                       vals.ctypes.data, prec, flags, _stream(stream),
                                       ctypes.byref(handle))
        else:
            vals = np.ascontiguousarray(values, dtype=np.uint64)
            if vals.shape != (prec // 64 + 1, colidx.shape[0]):
                raise ValueError(f"values are ({prec // 64 + 1}, {colidx.shape[0]}) planes; got "
                                 f"shape {vals.shape}")
            st = lib.mp_csr_create(n, rowptr.ctypes.data, colidx.ctypes.data, vals.ctypes.data,
                                   prec, flags, _stream(stream), ctypes.byref(handle))
        _ok(st, "mp_csr_create")
        self.h = handle
        self.n = n
        self.nnz = int(rowptr[-1])
        self.prec = prec
        self.transpose = transpose
        lens = np.diff(rowptr)
        # row-length histogram in powers of two (bucket k: lengths in [2^(k-1), 2^k))
        self.row_hist = np.bincount(np.ceil(np.log2(lens + 1)).astype(np.int64)).tolist() \
            if n > 0 else []

    @classmethod
    def _borrowed(cls, handle, n, prec, row_hist, owner):
        """A view of a matrix another object owns (never destroyed here)."""
        A = cls.__new__(cls)
        A.h, A.n, A.prec, A.transpose, A.row_hist = handle, n, prec, False, row_hist
        A._owner = owner
        A.nnz = A.info()["nnz"]
        return A

    def info(self) -> dict:
        n, nnz, slots, nbytes = (ctypes.c_int64() for _ in range(4))
        p = ctypes.c_int32()
        _ok(_lib.load().mp_csr_info(self.h, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(p),
                                    ctypes.byref(slots), ctypes.byref(nbytes)), "mp_csr_info")
        return {"n": n.value, "nnz": nnz.value, "prec": p.value, "slots": slots.value,
                "device_bytes": nbytes.value}

    def set_config(self, mode="ordered", threads_per_block=-1, variant=-1, carveout=-1):
        """SpMV launch configuration for one mode (results do not depend on it).
        variant: bit field, bit 0 = operand staging, bit 1 = products from
        radix-2^29 column sums, bit 2 = EXACT column sums 16 at a time /
        ORDERED register-capped blocks, bit 3 = x gathered from a record copy;
        carveout: shared-memory percent of L1/shared; -1 = library default."""
        _ok(_lib.load().mp_csr_set_config(self.h, MODES[mode], int(threads_per_block),
                                          int(variant), int(carveout)), "mp_csr_set_config")

    def get_config(self, mode="ordered") -> dict:
        t, v, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _ok(_lib.load().mp_csr_get_config(self.h, MODES[mode], ctypes.byref(t), ctypes.byref(v),
                                          ctypes.byref(c)), "mp_csr_get_config")
        return {"threads_per_block": t.value, "variant": v.value, "carveout": c.value}

    def tune(self, mode="ordered", reps=5, stream=None) -> dict:
        """Times every launch configuration of y = A x, keeps the fastest."""
        t, v, c, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
        _ok(_lib.load().mp_csr_tune(self.h, MODES[mode], int(reps), ctypes.byref(t),
                                    ctypes.byref(v), ctypes.byref(c), ctypes.byref(ms),
                                    _stream(stream)), "mp_csr_tune")
        return {"threads_per_block": t.value, "variant": v.value, "carveout": c.value,
                "ms": ms.value}

    def close(self):
        if getattr(self, "_owner", None) is not None:  # borrowed: the owner frees it
            self.h = None
            return
        if getattr(self, "h", None) is not None and self.h.value:
            _lib.load().mp_csr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def spmv(A: CSR, x: Vec, y: Vec | None = None, mode="ordered", stream=None, sync=True) -> Vec:
    """y = A x (Section 3)."""
    y = y if y is not None else Vec.empty(A.n, A.prec)
    _ok(_lib.load().mp_spmv(A.h, x.c(), y.c(), MODES[mode], _stream(stream)), "mp_spmv")
    if sync:
        check(stream)
    return y


def spmv_t(A: CSR, x: Vec, y: Vec | None = None, mode="ordered", stream=None, sync=True) -> Vec:
    """y = A^T x (needs ``transpose=True`` at creation)."""
    y = y if y is not None else Vec.empty(A.n, A.prec)
    _ok(_lib.load().mp_spmv_t(A.h, x.c(), y.c(), MODES[mode], _stream(stream)), "mp_spmv_t")
    if sync:
        check(stream)
    return y


def residual(A: CSR, b: Vec, x: Vec, r: Vec | None = None, stream=None, sync=True) -> Vec:
    """r = RN(b - A x), each row summed exactly."""
    r = r if r is not None else Vec.empty(A.n, A.prec)
    _ok(_lib.load().mp_residual(A.h, b.c(), x.c(), r.c(), _stream(stream)), "mp_residual")
    if sync:
        check(stream)
    return r


def gemv(A: Vec, m: int, n: int, x: Vec, y: Vec | None = None, stream=None,
         sync=True) -> Vec:
    """y = A x for a dense m x n matrix held column-major in the Vec A
    (element (i, j) at j*m + i): Section 3's dense MV, ORDERED row loops."""
    y = y if y is not None else Vec.empty(m, A.prec)
    _ok(_lib.load().mp_gemv(int(m), int(n), A.c(), x.c(), y.c(), _stream(stream)), "mp_gemv")
    if sync:
        check(stream)
    return y


def dot(x: Vec, y: Vec, out: Vec | None = None, stream=None, sync=True) -> Vec:
    """RN(sum x_i y_i), exact sum rounded once; returns a 1-element Vec."""
    out = out if out is not None else Vec.empty(1, x.prec)
    _ok(_lib.load().mp_dot(x.c(), y.c(), out.c(), _stream(stream)), "mp_dot")
    if sync:
        check(stream)
    return out


def axpy(alpha: Vec, x: Vec, y: Vec, stream=None, sync=True) -> Vec:
    """y <- RN(y + RN(alpha x)) in place."""
    _ok(_lib.load().mp_axpy(alpha.c(), x.c(), y.c(), _stream(stream)), "mp_axpy")
    if sync:
        check(stream)
    return y


def ewise(op: int, a: Vec, b: Vec, out: Vec | None = None, stream=None, sync=True) -> Vec:
    out = out if out is not None else Vec.empty(a.n, a.prec)
    _ok(_lib.load().mp_ewise(op, a.c(), b.c(), out.c(), _stream(stream)), "mp_ewise")
    if sync:
        check(stream)
    return out


def _solve(fn, name, A, b, x0, rtol, atol, maxit, mode, poll_every, history, stream,
           transpose=False, time_limit_ms=0):
    x = x0.clone() if x0 is not None else Vec.zeros(A.n, A.prec)
    hist = Vec.empty(max(maxit, 1), A.prec) if history else None
    opts = _lib.MpSolveOpts(float(rtol), float(atol), int(maxit), MODES[mode], int(poll_every),
                            hist.c() if hist is not None else _lib.MpVec(0, A.prec, 1, None),
                            1 if transpose else 0, int(time_limit_ms))
    info = _lib.MpSolveInfo()
    st = fn(A.h, b.c(), x.c(), ctypes.byref(opts), ctypes.byref(info), _stream(stream))
    if st not in (0, _lib.MP_ERR_NOCONV, _lib.MP_ERR_BREAKDOWN, _lib.MP_ERR_TIMEOUT):
        raise MPError(st, name)
    res = {"iters": int(info.iters), "status": int(info.status), "relres": float(info.relres),
           "ms": float(info.ms)}
    if hist is not None:
        res["history"] = Vec(hist.t[:, : max(int(info.iters), 0)].contiguous(), A.prec)
    return x, res


def bicg(A: CSR, b: Vec, x0: Vec | None = None, rtol=1e-30, atol=0.0, maxit=1000,
         mode="ordered", poll_every=8, history=False, stream=None, transpose=False,
         time_limit_ms=0):
    """BiCG (Fig. 5 left, K = I).  Returns (x, info dict).  transpose=True
    solves A^T x = b."""
    return _solve(_lib.load().mp_bicg, "mp_bicg", A, b, x0, rtol, atol, maxit, mode,
                  poll_every, history, stream, transpose, time_limit_ms)


def gpbicg(A: CSR, b: Vec, x0: Vec | None = None, rtol=1e-30, atol=0.0, maxit=1000,
           mode="ordered", poll_every=8, history=False, stream=None, transpose=False,
           time_limit_ms=0):
    """GPBiCG (Fig. 5 right).  Returns (x, info dict).  transpose=True solves
    A^T x = b (an adjoint system)."""
    return _solve(_lib.load().mp_gpbicg, "mp_gpbicg", A, b, x0, rtol, atol, maxit, mode,
                  poll_every, history, stream, transpose, time_limit_ms)


def cgs(A: CSR, b: Vec, x0: Vec | None = None, rtol=1e-30, atol=0.0, maxit=1000,
        mode="ordered", poll_every=8, history=False, stream=None, transpose=False,
        time_limit_ms=0):
    """CGS (Section 4's product-type method, textbook form, K = I).
    Returns (x, info dict)."""
    return _solve(_lib.load().mp_cgs, "mp_cgs", A, b, x0, rtol, atol, maxit, mode,
                  poll_every, history, stream, transpose, time_limit_ms)


def bicgstab(A: CSR, b: Vec, x0: Vec | None = None, rtol=1e-30, atol=0.0, maxit=1000,
             mode="ordered", poll_every=8, history=False, stream=None, transpose=False,
             time_limit_ms=0):
    """BiCGSTAB (Section 4's product-type method, textbook form, K = I).
    Returns (x, info dict)."""
    return _solve(_lib.load().mp_bicgstab, "mp_bicgstab", A, b, x0, rtol, atol, maxit, mode,
                  poll_every, history, stream, transpose, time_limit_ms)


class ILU0:
    """ILU(0) factors of a CSR matrix (Section 4's preconditioner, textbook
    IKJ form), built on the device."""

    def __init__(self, A: CSR, stream=None):
        h = ctypes.c_void_p()
        _ok(_lib.load().mp_ilu0_create(A.h, _stream(stream), ctypes.byref(h)), "mp_ilu0_create")
        self.h = h
        self.n, self.nnz, self.prec = A.n, A.nnz, A.prec

    def levels(self) -> tuple:
        a, b = ctypes.c_int64(), ctypes.c_int64()
        _ok(_lib.load().mp_ilu0_info(self.h, ctypes.byref(a), ctypes.byref(b)), "mp_ilu0_info")
        return a.value, b.value

    def factor(self, stream=None) -> Vec:
        """L and U values in the matrix's CSR order (sorted columns)."""
        lu = Vec.empty(self.nnz, self.prec)
        _ok(_lib.load().mp_ilu0_factor(self.h, lu.c(), _stream(stream)), "mp_ilu0_factor")
        check(stream)
        return lu

    def apply(self, r: Vec, w: Vec | None = None, stream=None, sync=True) -> Vec:
        """w = (LU)^{-1} r."""
        w = w if w is not None else Vec.empty(self.n, self.prec)
        _ok(_lib.load().mp_ilu0_apply(self.h, r.c(), w.c(), _stream(stream)), "mp_ilu0_apply")
        if sync:
            check(stream)
        return w

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            _lib.load().mp_ilu0_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def bicgstab_ilu0(A: CSR, M: ILU0, b: Vec, x0: Vec | None = None, rtol=1e-30, atol=0.0,
                  maxit=1000, mode="ordered", poll_every=8, history=False, stream=None,
                  side="left", time_limit_ms=0):
    """BiCGSTAB preconditioned with ILU(0) K = LU.  side="left" (Section 4.2,
    the paper's form): BiCGSTAB on K^{-1}A x = K^{-1}b, and the stopping rule,
    relres and history take the preconditioned residual K^{-1}(b - A x);
    side="right": r stays b - A x.  Returns (x, info dict)."""
    if side not in ("left", "right"):
        raise ValueError(f"side must be 'left' or 'right', not {side!r}")
    name = "mp_bicgstab_ilu0" if side == "left" else "mp_bicgstab_ilu0_right"
    fn = getattr(_lib.load(), name)

    def call(Ah, bc, xc, opts, info, st):
        return fn(Ah, M.h, bc, xc, opts, info, st)

    return _solve(call, name, A, b, x0, rtol, atol, maxit, mode, poll_every, history, stream,
                  time_limit_ms=time_limit_ms)


class Batch:
    """Independent systems of one precision stacked for batched solves.

    systems: list of (rowptr, colidx, values float64); several right-hand
    sides of one system are passed as repeated entries."""

    def __init__(self, systems, prec: int, stream=None):
        lib = _lib.load()
        self._keep = []
        ns, rps, cis, vas = [], [], [], []
        for rowptr, colidx, values in systems:
            rp, ci = _csr_arrays(rowptr, colidx)
            va = np.ascontiguousarray(values, dtype=np.float64)
            if va.shape != ci.shape:
                raise ValueError(f"{ci.shape[0]} double values expected; got shape {va.shape}")
            self._keep += [rp, ci, va]
            ns.append(rp.shape[0] - 1)
            rps.append(rp.ctypes.data)
            cis.append(ci.ctypes.data)
            vas.append(va.ctypes.data)
        k = len(ns)
        n_arr = np.array(ns, dtype=np.int64)
        ptrs = [np.array(v, dtype=np.uint64) for v in (rps, cis, vas)]
        handle = ctypes.c_void_p()
        st = lib.mp_batch_create_f64(k, n_arr.ctypes.data, ptrs[0].ctypes.data, ptrs[1].ctypes.data,
                                     ptrs[2].ctypes.data, prec, _stream(stream), ctypes.byref(handle))
        _ok(st, "mp_batch_create_f64")
        self._keep = []
        self.h = handle
        self.k = k
        self.prec = prec
        self._row_hist = np.bincount(np.ceil(np.log2(np.concatenate(
            [np.diff(np.asarray(r)) for r, _, _ in systems]) + 1)).astype(np.int64)).tolist()
        off = np.zeros(k + 1, dtype=np.int64)
        total = ctypes.c_int64()
        _ok(lib.mp_batch_info(self.h, None, ctypes.byref(total),
                              off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))), "mp_batch_info")
        self.offsets = off
        self.n = int(total.value)

    def matrix(self) -> "CSR":
        """The batch's block-diagonal matrix (owned by the batch) for
        set_config / tune; its launch configuration is the batched solve's."""
        h = ctypes.c_void_p()
        _ok(_lib.load().mp_batch_matrix(self.h, ctypes.byref(h)), "mp_batch_matrix")
        return CSR._borrowed(h, self.n, self.prec, self._row_hist, owner=self)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            _lib.load().mp_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_gpbicg(B: Batch, b: Vec, x0: Vec | None = None, rtol=1e-30, atol=0.0, maxit=100_000,
                 mode="ordered", poll_every=16, stream=None, time_limit_ms=0):
    """GPBiCG on all instances of a Batch at once.  Returns (x, infos)."""
    x = x0.clone() if x0 is not None else Vec.zeros(B.n, B.prec)
    opts = _lib.MpSolveOpts(float(rtol), float(atol), int(maxit), MODES[mode], int(poll_every),
                            _lib.MpVec(0, B.prec, 1, None), 0, int(time_limit_ms))
    infos = (_lib.MpSolveInfo * B.k)()
    st = _lib.load().mp_batch_gpbicg(B.h, b.c(), x.c(), ctypes.byref(opts), infos,
                                     _stream(stream))
    _ok(st, "mp_batch_gpbicg")
    return x, [{"iters": int(i.iters), "status": int(i.status), "ms": float(i.ms)} for i in infos]


def refine(A: CSR, b: Vec, x0: Vec | None = None, rtol=1e-34, max_outer=20, inner_rtol=1e-10,
           inner_maxit=20_000, equilibrate=True, poll_every=16, stream=None):
    """Mixed-precision iterative refinement (p-bit exact residual, FP64
    GPBiCG correction on a row-equilibrated FP64 copy of A).  Returns
    (x, info dict)."""
    x = x0.clone() if x0 is not None else Vec.zeros(A.n, A.prec)
    opts = _lib.MpRefineOpts(float(rtol), int(max_outer), float(inner_rtol), int(inner_maxit),
                             1 if equilibrate else 0, int(poll_every))
    info = _lib.MpRefineInfo()
    st = _lib.load().mp_refine(A.h, b.c(), x.c(), ctypes.byref(opts), ctypes.byref(info),
                               _stream(stream))
    if st not in (0, _lib.MP_ERR_NOCONV):
        raise MPError(st, "mp_refine")
    return x, {"outer": int(info.outer), "inner_iters": int(info.inner_iters),
               "status": int(info.status), "correction": float(info.correction),
               "relres": float(info.relres), "ms": float(info.ms)}


def csr_grad(A: CSR, lam: Vec, x: Vec, g: Vec | None = None, stream=None, sync=True) -> Vec:
    """dL/da_ij = RN((-lam_i) x_j) for every stored entry, in the caller's CSR
    order (lam solves A^T lam = dL/dx)."""
    g = g if g is not None else Vec.empty(A.nnz, A.prec)
    _ok(_lib.load().mp_csr_grad(A.h, lam.c(), x.c(), g.c(), _stream(stream)), "mp_csr_grad")
    if sync:
        check(stream)
    return g
