"""The bench's models of the kernels, on the CPU: the issued-multiply count
of the windowed EXACT product follows the kernel's window rule (its guard
bits are the kernel's), and the count is right on a hand-worked case."""
import os
import re
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_guard_bits_match_the_kernel():
    src = open(os.path.join(ROOT, "paper_1411_2377_gb300", "csrc", "spmv.cu")).read()
    m = re.search(r"constexpr int kTopGuard = (\d+);", src)
    assert m, "the windowed EXACT kernel's guard constant"
    assert int(m.group(1)) == bench.TOP_GUARD


def _planes(exps, p):
    L = p // 64
    planes = np.zeros((L + 1, len(exps)), np.uint64)
    planes[0] = (np.asarray(exps, np.int64) * 2).view(np.uint64)  # heads: e * 2 + sign 0
    planes[1:] = np.uint64(1) << np.uint64(63)
    return planes


def test_issued_multiplies_on_a_hand_worked_row():
    """One row of two terms at p = 1024: the larger term's product skips the
    columns below the window, the smaller one (far below) skips more.  The
    count is recomputed here from the rule written out: NA = 36 limbs of a,
    NX = 37 of the shifted x, column k has min(NA-1, k) - max(0, k-NX+1) + 1
    products, the window starts at digit wb = (span + p - g) // 29 and a term
    at digit q = (E - emin) // 29 computes columns k >= wb - q."""
    p, g = 1024, bench.TOP_GUARD
    rowptr = np.array([0, 2], np.int64)
    colidx = np.array([0, 1], np.int32)
    v = _planes([10, -200], p)        # a exponents
    x = _planes([5, 7], p)            # x exponents
    E = [10 + 5, -200 + 7]
    span = max(E) - min(E)
    na, nx = 36, 37
    pairs = [min(na - 1, k) - max(0, k - nx + 1) + 1 for k in range(na + nx - 1)]
    wb = (span + p - g) // 29
    want = 0
    for e in E:
        q = (e - min(E)) // 29
        kmin = min(max(0, wb - q), len(pairs))
        want += sum(pairs[kmin:])
    got = bench.windowed_issued(p, rowptr, colidx, v, x, 2)
    assert got == want / 2
    assert got < na * nx  # something is skipped
