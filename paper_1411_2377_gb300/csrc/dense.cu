// dense.cu -- p-bit dense matrix-vector product (Section 3's comparison:
// the dense MV that the sparse product is measured against).
//
// The matrix is stored column-major per plane (element (i, j) at j*m + i of
// each of the L+1 planes), so that the threads of a warp, one row each, read
// consecutive words at every column while x_j is one broadcast.  Each thread
// runs the ORDERED row loop of the SpMV over all n columns: y_i = +0, then
// y_i = RN(y_i + RN(a_ij x_j)) for j ascending, a zero factor skipped (the
// zero fast path the paper credits for MPFR's cheap dense products), so the
// result equals the ORDERED SpMV of the same matrix with its zeros stored or
// dropped.
#include <algorithm>

#include "internal.h"
#include "mpdev.cuh"

namespace mpk {
namespace {

template <int W>
__global__ void __launch_bounds__(128) gemv_ordered_kernel(int64_t m, int64_t n,
                                                           const uint64_t* __restrict__ A,
                                                           int64_t lda,
                                                           const uint64_t* __restrict__ x,
                                                           int64_t ldx, uint64_t* __restrict__ y,
                                                           int64_t ldy) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= m) return;
  Num<W> acc;
  set_zero(acc, 0u);
  Num<W> an, xn;
  if (n > 0) {
    load<W>(an, A, lda, i);
    load<W>(xn, x, ldx, 0);
  }
  for (int64_t j = 0; j < n; ++j) {
    const Num<W> a = an, xv = xn;
    if (j + 1 < n) {  // the next column's operands in flight
      load<W>(an, A + (j + 1) * m, lda, i);
      load<W>(xn, x, ldx, j + 1);
    }
    if (zero_e(a.e) || zero_e(xv.e)) continue;
    Num<W> t, s;
    // the product forms of the sparse ORDERED kernel, so that the two compare
    // like with like: short column product from p = 512, columns at 256
    if constexpr (W >= 16)
      mul_rn_short<W>(a, xv, t);
    else if constexpr (W >= 8)
      mul_rn_cols<W>(a, xv, t);
    else
      mul_rn<W>(a, xv, t);
    add_rn<W>(acc, t, s);
    acc = s;
  }
  store<W>(acc, y, ldy, i);
}

}  // namespace
}  // namespace mpk

using namespace mpk;

extern "C" {

mp_status mp_gemv(int64_t m, int64_t n, mp_vec A, mp_vec x, mp_vec y, void* stream) {
  if (m < 0 || n < 0) return set_error(MP_ERR_ARG, "shape %lld x %lld", (long long)m, (long long)n);
  if (!prec_ok(A.prec_bits)) return set_error(MP_ERR_PREC, "precision %d", A.prec_bits);
  mp_status r;
  if ((r = check_vec(A, m * n, A.prec_bits, "A")) != MP_OK) return r;
  if ((r = check_vec(x, n, A.prec_bits, "x")) != MP_OK) return r;
  if ((r = check_vec(y, m, A.prec_bits, "y")) != MP_OK) return r;
  if (m > 0 && n > 0 && x.data == y.data) return set_error(MP_ERR_ARG, "x and y must not alias");
  if (m == 0) return MP_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // a row per thread: small m gets small blocks, to spread over the SMs
  const int tpb = m >= (int64_t)sms * 128 ? 128 : 32;
  const int blocks = (int)((m + tpb - 1) / tpb);
  return dispatch_w(A.prec_bits, [&](auto w) {
    constexpr int W = decltype(w)::value;
    gemv_ordered_kernel<W><<<blocks, tpb, 0, st>>>(m, n, A.data, A.ld, x.data, x.ld, y.data,
                                                  y.ld);
    count_launch();
    return launch_check("gemv_ordered_kernel");
  });
}

}  // extern "C"
