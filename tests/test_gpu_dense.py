"""Section 3's dense MV (mp_gemv) and the s%-sparse Lotkin workload: the
dense product with zeros stored equals the sparse product with them dropped,
and both equal the oracle, bit for bit; the device-built Lotkin entries equal
the oracle's RN(1/k)."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_bitwise, need_gpu, rand_planes, recs
from paper_1411_2377_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("p", (128, 256, 512, 1024))
def test_gemv_random_matches_oracle(p):
    mpk = need_gpu()
    m, n = 77, 45
    D = rand_planes(m * n, p, 61, zero_frac=0.3, emin=-20, emax=20)  # column-major
    X = rand_planes(n, p, 62, zero_frac=0.1, emin=-20, emax=20)
    y = mpk.gemv(mpk.Vec.from_planes(D, p), m, n, mpk.Vec.from_planes(X, p))
    # the oracle takes square matrices: the same rows as an m x m CSR whose
    # first n columns hold every entry of A (row-major order), x padded
    rowptr = np.arange(0, m * n + 1, n, dtype=np.int64)
    colidx = np.tile(np.arange(n, dtype=np.int32), m)
    order = (np.arange(n)[None, :] * m + np.arange(m)[:, None]).ravel()
    xpad = np.concatenate([recs(X), oracle.empty(p, m - n)])
    want, st = oracle.spmv(p, oracle.ORDERED, rowptr, colidx, recs(D)[order], xpad)
    assert st == oracle.OK
    assert_bitwise(y.planes(), want, f"gemv p={p}")


@pytest.mark.parametrize("p", (128, 1024))
@pytest.mark.parametrize("s", (0.0, 50.0, 90.0))
def test_lotkin_dense_equals_sparse_and_oracle(p, s):
    mpk = need_gpu()
    from paper_1411_2377_gb300 import lotkin

    n = 150
    A, D = lotkin.lotkin(n, s, p, seed=7)
    b = lotkin.rhs(A, n, p)
    ys = mpk.spmv(A, b, mode="ordered")
    assert A.nnz == int(synth.lotkin_pattern(n, s, 7)[0][-1])
    yd = mpk.gemv(D, n, n, b)
    rowptr, colidx, num, den = synth.lotkin_pattern(n, s, 7)
    vals, _ = oracle.ewise(p, oracle.OP_DIV, oracle.from_f64(p, num), oracle.from_f64(p, den))
    bo, _ = oracle.spmv(p, oracle.ORDERED, rowptr, colidx, vals,
                        oracle.from_f64(p, np.arange(1, n + 1, dtype=np.float64)))
    assert_bitwise(b.planes(), bo, f"b p={p} s={s}")
    want, _ = oracle.spmv(p, oracle.ORDERED, rowptr, colidx, vals, bo)
    assert_bitwise(ys.planes(), want, f"sparse p={p} s={s}")
    assert_bitwise(yd.planes(), want, f"dense p={p} s={s}")


def test_gemv_rejects_bad_shapes():
    mpk = need_gpu()
    p = 128
    A = mpk.Vec.zeros(12, p)
    x = mpk.Vec.zeros(4, p)
    with pytest.raises(mpk.MPError):
        mpk.gemv(A, 3, 5, x)  # 15 != 12 elements
    y = mpk.gemv(A, 3, 4, x)
    assert (y.to_f64().cpu().numpy() == 0).all()
