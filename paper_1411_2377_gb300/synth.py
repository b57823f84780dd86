"""Seeded synthetic workloads (shared by the GPU path's tests and benchmark and
by the oracle's tests as *inputs only*).

No arithmetic of the method lives here: the module draws counter-based
random numbers (splitmix64, Steele/Lea/Flood 2014: state_i = key + (i+1)*G,
output = mix(state_i)) and lays them out as CSR patterns, double-precision
stencil coefficients, or p-bit values encoded bit by bit.

Workloads (the paper's UF matrices cavity04 and epb3 are not available, so
these stand in for its nonsymmetric sparse test problems, Section 4):

* :func:`stencil2d` -- 2-D 5-point convection-diffusion-like matrix on an
  m x m grid (n = m^2): diagonal 4 + U(0, 0.1), each present off-diagonal
  -1 + 0.3 U(-1, 1).  m = 64 gives n = 4096, nnz = 20 224; m = 256 gives
  n = 65 536, nnz = 326 656.
* :func:`stencil3d` -- 3-D 7-point upwind-biased convection-diffusion on an
  m^3 grid, h = 1/(m+1), velocity (1,1,1), Peclet number Pe: diagonal 6,
  upwind neighbours -1 - gamma, downwind -1 + gamma with gamma = Pe h / 2,
  each row scaled by 10^(D U(0,1)) (D = 20 makes kappa ~ 1e20).
* :func:`random_csr_pattern` + :func:`random_values` -- n x n matrix with
  lognormal row lengths (mean 16, clamped to [1, 256]); 90 % of the columns
  of row i uniform in the band [i-5000, i+5000], 10 % uniform in [0, n);
  values with random sign, mantissa 1 + (p-1) random bits in [1, 2) and
  exponent uniform in [-40, 40]; 1 % exact zeros.

p-bit values use the plane-major layout of the library: plane 0 holds the
head words ``exp*2 + sign`` (``exp`` in the 0.1xxx convention, zero flagged by
``EXP_ZERO``), planes 1..L the mantissa limbs, least significant first.
"""
from __future__ import annotations

import math

import numpy as np

EXP_ZERO = -(1 << 61)
_M64 = (1 << 64) - 1
_G = 0x9E3779B97F4A7C15

# draw purposes (streams)
S_ROWLEN_A, S_ROWLEN_B, S_COLPICK, S_COLBAND, S_COLFAR = 1, 2, 3, 4, 5
S_SIGN, S_EXP, S_ZERO, S_LIMB = 10, 11, 12, 100
S_DIAG, S_OFF, S_ROWSCALE = 20, 21, 22
S_MISC = 50


def _mix_int(z: int) -> int:
    z &= _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def u64(seed: int, stream: int, idx) -> np.ndarray:
    """splitmix64 output number ``idx`` of the sequence keyed by (seed, stream)."""
    key = _mix_int(_mix_int(seed * _G + 0x5851F42D4C957F2D) ^ (stream * 0xD1B54A32D192ED03))
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = np.uint64(key) + (idx + np.uint64(1)) * np.uint64(_G)
        return _mix(state)


def uniform(seed: int, stream: int, idx) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits."""
    return (u64(seed, stream, idx) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, stream_a: int, stream_b: int, idx) -> np.ndarray:
    """Standard normal draws (Box-Muller on two independent uniforms)."""
    u1 = 1.0 - uniform(seed, stream_a, idx)  # (0, 1]
    u2 = uniform(seed, stream_b, idx)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def head_words(exp: np.ndarray, sign: np.ndarray) -> np.ndarray:
    """Encode head words exp*2 + sign as uint64 bit patterns."""
    h = exp.astype(np.int64) * 2 + sign.astype(np.int64)
    return h.view(np.uint64)


# ---------------------------------------------------------------------------
# Stencil matrices (double-precision coefficients)
# ---------------------------------------------------------------------------

def _assemble(n, rows, cols, vals):
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    return rowptr, cols.astype(np.int32), vals


def stencil2d(m: int, seed: int = 0):
    """5-point matrix on an m x m grid, node i = gx + m*gy.

    Returns (rowptr int64[n+1], colidx int32[nnz], values float64[nnz])."""
    n = m * m
    idx = np.arange(n, dtype=np.int64)
    gx, gy = idx % m, idx // m
    rows, cols, vals = [idx], [idx], [4.0 + 0.1 * uniform(seed, S_DIAG, idx)]
    for d, (dx, dy) in enumerate(((-1, 0), (1, 0), (0, -1), (0, 1))):
        ok = (gx + dx >= 0) & (gx + dx < m) & (gy + dy >= 0) & (gy + dy < m)
        i = idx[ok]
        j = i + dx + m * dy
        u = uniform(seed, S_OFF + 10 * (d + 1), i)
        rows.append(i)
        cols.append(j)
        vals.append(-1.0 + 0.3 * (2.0 * u - 1.0))
    return _assemble(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def stencil3d(m: int, seed: int = 2, pe: float = 50.0, decades: float = 20.0):
    """7-point convection-diffusion matrix on an m^3 grid, rows scaled by
    10^(decades*U(0,1)).  Node i = gx + m*gy + m^2*gz."""
    n = m * m * m
    h = 1.0 / (m + 1)
    gamma = pe * h / 2.0
    idx = np.arange(n, dtype=np.int64)
    g = (idx % m, (idx // m) % m, idx // (m * m))
    stride = (1, m, m * m)
    scale = 10.0 ** (decades * uniform(seed, S_ROWSCALE, idx))
    rows, cols, vals = [idx], [idx], [6.0 * scale]
    for ax in range(3):
        for step, coef in ((-1, -1.0 - gamma), (1, -1.0 + gamma)):
            ok = (g[ax] + step >= 0) & (g[ax] + step < m)
            i = idx[ok]
            rows.append(i)
            cols.append(i + step * stride[ax])
            vals.append(coef * scale[ok])
    return _assemble(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


# ---------------------------------------------------------------------------
# Random pattern with lognormal row lengths and a band (SpMV throughput)
# ---------------------------------------------------------------------------

def random_csr_pattern(n: int, seed: int = 1, mean_len: float = 16.0, sigma: float = 1.0,
                       max_len: int = 256, band: int = 5000, p_band: float = 0.9):
    """CSR pattern (rowptr int64[n+1], colidx int32[nnz]); columns sorted and
    unique within each row."""
    i = np.arange(n, dtype=np.int64)
    mu = math.log(mean_len) - sigma * sigma / 2.0
    z = normal(seed, S_ROWLEN_A, S_ROWLEN_B, i)
    ln = np.clip(np.rint(np.exp(mu + sigma * z)), 1, min(max_len, n)).astype(np.int64)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(ln, out=rowptr[1:])
    nnz = int(rowptr[-1])
    row = np.repeat(i, ln)
    lo = np.maximum(row - band, 0)
    hi = np.minimum(row + band, n - 1)
    col = np.empty(nnz, dtype=np.int64)
    todo = np.arange(nnz, dtype=np.int64)
    attempt = 0
    while todo.size:
        k = todo.astype(np.uint64) + np.uint64(attempt * nnz)
        pick = uniform(seed, S_COLPICK, k) < p_band
        ub = uniform(seed, S_COLBAND, k)
        uf = uniform(seed, S_COLFAR, k)
        r = row[todo]
        width = hi[todo] - lo[todo] + 1
        cb = lo[todo] + np.minimum((ub * width).astype(np.int64), width - 1)
        cf = np.minimum((uf * n).astype(np.int64), n - 1)
        col[todo] = np.where(pick, cb, cf)
        # the first occurrence (in slot order) of a column in a row is kept,
        # later repeats are drawn again
        key = row * n + col
        order = np.argsort(key, kind="stable")
        ks = key[order]
        dup = np.zeros(nnz, dtype=bool)
        dup[order[1:]] = ks[1:] == ks[:-1]
        todo = np.nonzero(dup)[0]
        attempt += 1
        del r
    key = np.sort(row * n + col)
    colidx = (key - row * n).astype(np.int32)
    return rowptr, colidx


def random_values(count: int, p: int, seed: int, stream0: int = 0, zero_frac: float = 0.01,
                  emin: int = -40, emax: int = 40) -> np.ndarray:
    """(L+1, count) planes of p-bit values: random sign, mantissa in [1, 2)
    with p-1 random bits, exponent uniform in [emin, emax], a fraction
    ``zero_frac`` exact (+0) zeros."""
    L = p // 64
    k = np.arange(count, dtype=np.uint64)
    out = np.empty((L + 1, count), dtype=np.uint64)
    sign = (u64(seed, stream0 + S_SIGN, k) & np.uint64(1)).astype(np.int64)
    span = emax - emin + 1
    e2 = emin + (u64(seed, stream0 + S_EXP, k) % np.uint64(span)).astype(np.int64)
    exp = e2 + 1  # m * 2^e2 with m in [1,2) is 0.1xxx * 2^(e2+1)
    zero = uniform(seed, stream0 + S_ZERO, k) < zero_frac if zero_frac > 0 else np.zeros(count, bool)
    for j in range(L):
        out[1 + j] = u64(seed, stream0 + S_LIMB + j, k)
    out[L] |= np.uint64(1 << 63)
    exp = np.where(zero, EXP_ZERO, exp)
    sign = np.where(zero, 0, sign)
    out[0] = head_words(exp, sign)
    if zero.any():
        out[1:, zero] = 0
    return out


def batch_systems(seed: int = 3, count: int = 256, nmin: int = 1000, nmax: int = 65536):
    """Descriptions of the batched-solve workload: system s has a size drawn
    log-uniformly in [nmin, nmax], a 2-D 5-point (side ceil(sqrt n)) or 3-D
    7-point (side ceil(cbrt n), no row scaling) convection-diffusion matrix,
    precision 128 or 256 bits and 1-4 right-hand sides (the k-th one is
    b = A * ((k+1) * ones)).  Returns dicts with kind, m, p, nrhs, mseed."""
    s = np.arange(count, dtype=np.uint64)
    u = uniform(seed, S_MISC + 1, s)
    target = np.exp(math.log(nmin) + u * (math.log(nmax) - math.log(nmin)))
    kind = np.where(uniform(seed, S_MISC + 2, s) < 0.5, "2d", "3d")
    prec = np.where(uniform(seed, S_MISC + 3, s) < 0.5, 128, 256)
    nrhs = 1 + np.minimum((uniform(seed, S_MISC + 4, s) * 4).astype(np.int64), 3)
    out = []
    for i in range(count):
        if kind[i] == "2d":
            m = int(math.ceil(math.sqrt(target[i])))
        else:
            m = int(math.ceil(round(target[i] ** (1.0 / 3.0), 9)))
        out.append({"kind": str(kind[i]), "m": m, "p": int(prec[i]), "nrhs": int(nrhs[i]),
                    "mseed": seed * 1000 + i})
    return out


def batch_matrix(desc):
    """(rowptr, colidx, values) of one batch_systems entry."""
    if desc["kind"] == "2d":
        return stencil2d(desc["m"], seed=desc["mseed"])
    return stencil3d(desc["m"], seed=desc["mseed"], decades=0.0)


SPMV_N = 1_000_000


def spmv_pattern(n: int = SPMV_N, seed: int = 1):
    """Pattern of the SpMV throughput workload (seed 1, n = 10^6)."""
    return random_csr_pattern(n, seed=seed)


def spmv_values(p: int, nnz: int, n: int, seed: int = 1):
    """Values (1 % zeros) and x (no zeros) of the SpMV throughput workload."""
    vals = random_values(nnz, p, seed=seed)
    x = random_values(n, p, seed=seed + 1, stream0=1000, zero_frac=0.0)
    return vals, x


def ones(n: int, p: int) -> np.ndarray:
    """(L+1, n) planes holding 1.0 (= 0.1_2 * 2^1)."""
    L = p // 64
    out = np.zeros((L + 1, n), dtype=np.uint64)
    out[0] = head_words(np.ones(n, np.int64), np.zeros(n, np.int64))
    out[L] = np.uint64(1 << 63)
    return out


def zeros(n: int, p: int) -> np.ndarray:
    L = p // 64
    out = np.zeros((L + 1, n), dtype=np.uint64)
    out[0] = head_words(np.full(n, EXP_ZERO, np.int64), np.zeros(n, np.int64))
    return out


def small_random_csr(n: int, seed: int, density: float = 0.3, empty_rows: int = 0,
                     diag: bool = False):
    """Tiny random pattern for tests: each (i, j) present with probability
    ``density`` (plus the diagonal when ``diag``); the first ``empty_rows``
    rows are left empty."""
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    u = uniform(seed, S_MISC, np.arange(n * n, dtype=np.uint64)).reshape(n, n)
    mask = u < density
    if diag:
        mask |= ii == jj
    mask[:empty_rows] = False
    rows, cols = np.nonzero(mask)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    return np.cumsum(rowptr), cols.astype(np.int32)


def lotkin_pattern(n: int, s_percent: float, seed: int = 7):
    """Section 3's SpMV workload: the n x n Lotkin matrix (first row ones,
    a_ij = 1/(i+j-1) below it, 1-based) with each entry dropped with
    probability s_percent/100 (one draw per (i, j), row-major index).
    Returns (rowptr, colidx, num, den): the kept entries in row order, each
    the rational num/den (small integers as float64, exact)."""
    u = uniform(seed, S_MISC, np.arange(n * n, dtype=np.uint64)).reshape(n, n)
    rows, cols = np.nonzero(u >= s_percent / 100.0)
    rowptr = np.zeros(n + 1, np.int64)
    np.add.at(rowptr, rows + 1, 1)
    den = np.where(rows == 0, 1, rows + cols + 1).astype(np.float64)
    return np.cumsum(rowptr), cols.astype(np.int32), np.ones(len(cols)), den


def planes_to_records(planes: np.ndarray) -> np.ndarray:
    """(L+1, n) planes -> (n, L+1) records (the oracle's layout)."""
    return np.ascontiguousarray(planes.T)


def records_to_planes(recs: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(recs).T)
