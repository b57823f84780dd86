"""Differentiating the GPBiCG solve x = A^{-1} b.

The forward pass is a p-bit GPBiCG solve (Fig. 5 right) on the GPU; only x is
kept for the backward pass.  The backward pass is hand-written: given
xbar = dL/dx it solves the adjoint system A^T lam = xbar with the same p-bit
GPBiCG on the explicit transpose, then dL/db = lam and, on the sparsity
pattern only, dL/da_ij = -lam_i x_j, formed by one fused gather kernel
(mp_csr_grad).  Everything runs in the library's kernels; this module only
marshals arguments.

Two interfaces:

* :func:`adjoint` works on p-bit vectors (:class:`Vec`) throughout, for
  callers that need the gradient at full precision.
* :class:`MPSolve` is a ``torch.autograd.Function`` over float64 tensors: the
  CSR values and b are converted exactly to p bits, x and the gradients are
  returned rounded to float64.
"""
from __future__ import annotations

import numpy as np

from . import CSR, Vec, csr_grad, gpbicg


def solve(A: CSR, b: Vec, rtol=1e-30, maxit=100_000, mode="ordered"):
    """Forward solve; returns (x, info)."""
    x, info = gpbicg(A, b, rtol=rtol, maxit=maxit, mode=mode)
    if info["status"] != 0:
        raise RuntimeError(f"forward GPBiCG did not converge: {info}")
    return x, info


def adjoint(A: CSR, x: Vec, xbar: Vec, rtol=1e-30, maxit=100_000, mode="ordered"):
    """Backward pass at p bits: lam with A^T lam = xbar, and the pattern
    gradient g_k = RN((-lam_i) x_j) in the caller's CSR order.  Returns
    (lam, g, info).  A needs ``transpose=True``."""
    lam, info = gpbicg(A, xbar, rtol=rtol, maxit=maxit, mode=mode, transpose=True)
    if info["status"] != 0:
        raise RuntimeError(f"adjoint GPBiCG did not converge: {info}")
    g = csr_grad(A, lam, x)
    return lam, g, info


def _torch():
    import torch

    return torch


def _make_function():
    torch = _torch()

    class MPSolve(torch.autograd.Function):
        """x = A^{-1} b at p bits with gradients for the CSR values and b.

        apply(values, b, rowptr, colidx, prec, rtol, maxit, mode):
        values (nnz,) and b (n,) are float64 tensors; rowptr/colidx the
        pattern (numpy or CPU tensors).  Returns x as a float64 CUDA tensor."""

        @staticmethod
        def forward(ctx, values, b, rowptr, colidx, prec=256, rtol=1e-30, maxit=100_000,
                    mode="ordered"):
            rp = np.asarray(rowptr.cpu() if hasattr(rowptr, "cpu") else rowptr, dtype=np.int64)
            ci = np.asarray(colidx.cpu() if hasattr(colidx, "cpu") else colidx, dtype=np.int32)
            vals = values.detach().to("cpu", torch.float64).numpy()
            A = CSR(rp, ci, vals, prec, transpose=True)
            x, _ = solve(A, Vec.from_f64(b.detach(), prec), rtol=rtol, maxit=maxit, mode=mode)
            ctx.A, ctx.x, ctx.cfg = A, x, (prec, rtol, maxit, mode)
            ctx.devices = (values.device, b.device)
            return x.to_f64()

        @staticmethod
        def backward(ctx, gx):
            prec, rtol, maxit, mode = ctx.cfg
            xbar = Vec.from_f64(gx.detach().to(torch.float64), prec)
            lam, g, _ = adjoint(ctx.A, ctx.x, xbar, rtol=rtol, maxit=maxit, mode=mode)
            dv, db = ctx.devices
            return (g.to_f64().to(dv), lam.to_f64().to(db), None, None, None, None, None, None)

    return MPSolve


_MPSolve = None


def MPSolve():
    """The torch.autograd.Function class (created on first use, so that
    importing this module does not import torch)."""
    global _MPSolve
    if _MPSolve is None:
        _MPSolve = _make_function()
    return _MPSolve
