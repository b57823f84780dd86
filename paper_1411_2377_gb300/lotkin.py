"""Section 3's SpMV workload on the device: the n x n Lotkin matrix with s %
of its entries set to zero, its entries RN(1/(i+j-1)) at p bits (divided on
the device), stored sparse (zeros dropped) and dense (zeros kept,
column-major for mp_gemv); b = A [1 2 ... n]^T, then y = A b both ways.
"""
from __future__ import annotations

import numpy as np

from . import CSR, MP_OP_DIV, Vec, ewise, synth


def lotkin(n: int, s_percent: float, p: int, seed: int = 7, dense: bool = True):
    """Returns (A sparse CSR, A dense Vec of n*n elements or None)."""
    import torch

    rowptr, colidx, num, den = synth.lotkin_pattern(n, s_percent, seed)
    vals = ewise(MP_OP_DIV, Vec.from_f64(num, p), Vec.from_f64(den, p))
    A = CSR(rowptr, colidx, vals.planes(), p)
    D = None
    if dense:
        D = Vec.zeros(n * n, p)
        rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(rowptr))
        idx = torch.as_tensor(colidx.astype(np.int64) * n + rows, device=D.t.device)
        D.t[:, idx] = vals.t
    return A, D


def rhs(A: CSR, n: int, p: int) -> Vec:
    """b = A [1 2 ... n]^T (ORDERED, as a multiple-precision MV)."""
    from . import spmv

    return spmv(A, Vec.from_f64(np.arange(1, n + 1, dtype=np.float64), p), mode="ordered")
