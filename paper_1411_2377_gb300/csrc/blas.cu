// blas.cu -- exact dot products, axpy, elementwise operations, conversions.
//
// Exact dot products (the inner products of Fig. 5) take three kernels:
//  1. span: min/max of e_x + e_y over the nonzero pairs (warp reduction, one
//     64-bit atomicMin/atomicMax per warp: min and max are order-free);
//  2. accumulate: each thread adds the exact 2p-bit products of its pairs,
//     shifted onto the 32-bit digit grid anchored at Emin, into its own
//     window of 64-bit signed counters in shared memory (digit-major, so a
//     warp's accesses hit 32 banks; no atomics, no carries); the block then
//     sums its threads' windows digit by digit into one partial per block,
//     stored digit-major across blocks;
//  3. finalize: one block per dot sums the partials per digit (a warp per
//     digit, lanes over blocks; integer sums: any order gives the same
//     bits), resolves carries and rounds once.
// A dot whose span exceeds the per-thread windows takes, inside step 2, one
// block-wide window of the full span cap filled with shared-memory atomics.  Up to five dots over the same index
// range run in one pass, so GPBiCG's mu_1..mu_5 read y, v and t once.
#include <climits>
#include <mutex>

#include "internal.h"
#include "mpdev.cuh"

namespace mpk {
namespace {

constexpr int kDotThreads = 128;
constexpr int kDotWarps = kDotThreads / 32;
constexpr int kDotFastSpan = 1024;

template <int W>
struct DotWin {
  static constexpr int fast = (kDotFastSpan + 64 * W + 96) / 32 + 1;
  static constexpr int cap = (SPAN_CAP + 64 * W + 96) / 32 + 1;
};

__host__ __device__ inline int dot_digits(int64_t span, int W) {
  return (int)((span + 64 * W + 96) / 32) + 1;
}

struct DotDev {
  int k;
  int64_t n;
  const uint64_t* x[5];
  const uint64_t* y[5];
  int64_t ldx[5], ldy[5];
  uint64_t* out[5];
  int64_t out_ld[5];
};

struct DotScratch {
  long long* emin;  // [5]
  long long* emax;  // [5]
  int64_t* partials;  // [5][cap][nblocks]: digit-major per dot
  int nblocks;
};

int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

int dot_blocks(int64_t n) {
  int64_t b = (n + kDotThreads - 1) / kDotThreads;
  const int64_t lim = (int64_t)sm_count() * 4;
  if (b > lim) b = lim;
  if (b < 1) b = 1;
  return (int)b;
}

template <int W>
__global__ void __launch_bounds__(kDotThreads) dot_span_kernel(const DotDev a, long long* emin,
                                                               long long* emax,
                                                               const int* __restrict__ gate) {
  if (gate && *gate) return;
  const int lane = threadIdx.x & 31;
  for (int j = 0; j < a.k; ++j) {
    long long lo = LLONG_MAX, hi = LLONG_MIN;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n;
         i += (int64_t)gridDim.x * blockDim.x) {
      int64_t ex, ey;
      uint32_t sx, sy;
      unpack_head(__ldg(a.x[j] + i), ex, sx);
      unpack_head(__ldg(a.y[j] + i), ey, sy);
      if (zero_e(ex) || zero_e(ey)) continue;
      lo = min(lo, (long long)(ex + ey));
      hi = max(hi, (long long)(ex + ey));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lane == 0 && lo <= hi) {
      atomicMin(emin + j, lo);
      atomicMax(emax + j, hi);
    }
  }
}

// smem: per thread FAST 64-bit counters, digit-major ([FAST][threads]).
template <int W>
__host__ __device__ constexpr size_t dot_smem(int) {
  return (size_t)DotWin<W>::fast * kDotThreads * 8;
}

__device__ __forceinline__ int64_t warp_sum64(int64_t t) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  return t;
}

template <int W>
__global__ void __launch_bounds__(kDotThreads) dot_accum_kernel(const DotDev a, DotScratch s,
                                                                const int* __restrict__ gate) {
  extern __shared__ int64_t dsm[];
  __shared__ int64_t acc[DotWin<W>::cap];  // the block-wide window of a wide span
  if (gate && *gate) return;
  constexpr int CAP = DotWin<W>::cap;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t* c = dsm + threadIdx.x;
  for (int j = 0; j < a.k; ++j) {
    const long long lo = s.emin[j], hi = s.emax[j];
    if (!(lo <= hi && hi - lo <= SPAN_CAP)) continue;  // block-uniform
    const int nd = dot_digits(hi - lo, W);
    if (hi - lo > kDotFastSpan) {
      // a span beyond the per-thread windows: one block-wide window with
      // shared-memory atomics (rare: the solvers' vectors stay well inside)
      for (int d = threadIdx.x; d < nd; d += kDotThreads) acc[d] = 0;
      __syncthreads();
      for (int64_t i = blockIdx.x * (int64_t)kDotThreads + threadIdx.x; i < a.n;
           i += (int64_t)gridDim.x * kDotThreads) {
        Num<W> x, y;
        load<W>(x, a.x[j], a.ldx[j], i);
        load<W>(y, a.y[j], a.ldy[j], i);
        if (zero_e(x.e) || zero_e(y.e)) continue;
        uint32_t P[2 * W], D[2 * W + 1];
        mul_full<W>(x.m, y.m, P);
        const int64_t off = x.e + y.e - lo;
        shifted_digits<W>(P, (uint32_t)(off & 31), D);
        const bool ng = (x.s ^ y.s) != 0;
        for (int k = 0; k <= 2 * W; ++k) {
          const int64_t v = (int64_t)D[k];
          atomicAdd((unsigned long long*)&acc[(off >> 5) + k], (unsigned long long)(ng ? -v : v));
        }
      }
      __syncthreads();
      int64_t* part = s.partials + (size_t)j * CAP * s.nblocks;
      for (int d = threadIdx.x; d < nd; d += kDotThreads) part[(size_t)d * s.nblocks + blockIdx.x] = acc[d];
      __syncthreads();
      continue;
    }
    for (int d = 0; d < nd; ++d) c[d * kDotThreads] = 0;
    for (int64_t i = blockIdx.x * (int64_t)kDotThreads + threadIdx.x; i < a.n;
         i += (int64_t)gridDim.x * kDotThreads) {
      Num<W> x, y;
      load<W>(x, a.x[j], a.ldx[j], i);
      load<W>(y, a.y[j], a.ldy[j], i);
      if (zero_e(x.e) || zero_e(y.e)) continue;
      uint32_t P[2 * W];
      if (W >= 16)
        mul_full_ilp<W>(x.m, y.m, P);
      else
        mul_full<W>(x.m, y.m, P);
      add_term<W>(c, kDotThreads, P, x.e + y.e - lo, x.s ^ y.s);
    }
    __syncthreads();
    int64_t* part = s.partials + (size_t)j * CAP * s.nblocks;
    for (int d = warp; d < nd; d += kDotWarps) {
      int64_t t = 0;
#pragma unroll
      for (int u = 0; u < kDotThreads / 32; ++u) t += dsm[d * kDotThreads + u * 32 + lane];
      t = warp_sum64(t);
      if (lane == 0) part[(size_t)d * s.nblocks + blockIdx.x] = t;
    }
    __syncthreads();
  }
}

// One block per dot: sum partials, resolve carries, round once.  Resets the
// span slots for the next use.
template <int W>
__global__ void __launch_bounds__(256) dot_finalize_kernel(const DotDev a, DotScratch s,
                                                           int* __restrict__ status,
                                                           const int* __restrict__ gate) {
  __shared__ int64_t sum[DotWin<W>::cap];
  if (gate && *gate) return;
  const int j = blockIdx.x;
  const long long lo = s.emin[j], hi = s.emax[j];
  Num<W> r;
  set_zero(r, 0u);
  if (lo <= hi && hi - lo <= SPAN_CAP) {
    const int nd = dot_digits(hi - lo, W);
    const int64_t* part = s.partials + (size_t)j * DotWin<W>::cap * s.nblocks;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int d = warp; d < nd; d += nwarps) {
      int64_t t = 0;
      for (int b = lane; b < s.nblocks; b += 32) t += part[(size_t)d * s.nblocks + b];
      t = warp_sum64(t);
      if (lane == 0) sum[d] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      const uint32_t negative = resolve_digits(sum, 1, nd);
      if (negative) negate_words(sum, 1, nd);
      round_words<W>(sum, 1, nd, (int64_t)lo - 64 * W, negative, r);
    }
  } else if (lo <= hi && threadIdx.x == 0 && status) {
    atomicCAS(status, 0, (int)MP_ERR_SPAN);
  }
  if (threadIdx.x == 0) {
    store<W>(r, a.out[j], a.out_ld[j], 0);
    s.emin[j] = LLONG_MAX;
    s.emax[j] = LLONG_MIN;
  }
}

__global__ void reset_span_slots(long long* emin, long long* emax) {
  if (threadIdx.x < 5) {
    emin[threadIdx.x] = LLONG_MAX;
    emax[threadIdx.x] = LLONG_MIN;
  }
}

template <int W>
mp_status dot_w(const DotArgs& args, void* scratch, const int* gate, cudaStream_t st) {
  DotDev a{};
  a.k = args.k;
  a.n = args.n;
  for (int j = 0; j < 5; ++j) {
    a.x[j] = args.x[j];
    a.y[j] = args.y[j];
    a.ldx[j] = args.ldx[j];
    a.ldy[j] = args.ldy[j];
    a.out[j] = args.out[j];
    a.out_ld[j] = args.out_ld[j];
  }
  DotScratch s;
  s.emin = static_cast<long long*>(scratch);
  s.emax = s.emin + 5;
  s.partials = reinterpret_cast<int64_t*>(s.emin + 16);
  s.nblocks = dot_blocks(args.n);
  int* status = status_word();
  if (!status) return set_error(MP_ERR_CUDA, "status word unavailable");
  const size_t smem = dot_smem<W>(a.k);
  MPK_CUDA(cudaFuncSetAttribute(dot_accum_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
  // streamed operands: shared memory for the windows matters more than L1
  MPK_CUDA(cudaFuncSetAttribute(dot_accum_kernel<W>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared));
  dot_span_kernel<W><<<s.nblocks, kDotThreads, 0, st>>>(a, s.emin, s.emax, gate);
  dot_accum_kernel<W><<<s.nblocks, kDotThreads, smem, st>>>(a, s, gate);
  dot_finalize_kernel<W><<<a.k, 256, 0, st>>>(a, s, status, gate);
  count_launch(3);
  return launch_check("dot kernels");
}

// ---------------------------------------------------------------------------
// Elementwise kernels
// ---------------------------------------------------------------------------

int ew_blocks(int64_t n) {
  int64_t b = (n + 255) / 256;
  const int64_t lim = (int64_t)sm_count() * 16;
  if (b > lim) b = lim;
  return (int)(b < 1 ? 1 : b);
}

template <int W>
__global__ void axpy_kernel(const uint64_t* __restrict__ al, int64_t n,
                            const uint64_t* __restrict__ x, int64_t ldx, uint64_t* __restrict__ y,
                            int64_t ldy) {
  Num<W> alpha;
  load<W>(alpha, al, 1, 0);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    Num<W> xv, yv, t, r;
    load<W>(xv, x, ldx, i);
    load<W>(yv, y, ldy, i);
    mul_rn<W>(alpha, xv, t);
    add_rn<W>(yv, t, r);
    store<W>(r, y, ldy, i);
  }
}

template <int W>
__global__ void ewise_kernel(int op, int64_t n, const uint64_t* __restrict__ a, int64_t lda,
                             const uint64_t* __restrict__ b, int64_t ldb, uint64_t* out,
                             int64_t ldo, int* status) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    Num<W> x, y, r;
    load<W>(x, a, lda, i);
    load<W>(y, b, ldb, i);
    switch (op) {
      case MP_OP_MUL: mul_rn<W>(x, y, r); break;
      case MP_OP_ADD: add_rn<W>(x, y, r); break;
      case MP_OP_SUB: sub_rn<W>(x, y, r); break;
      default:
        if (zero_e(y.e)) {
          set_zero(r, 0u);
          atomicCAS(status, 0, (int)MP_ERR_DIVZERO);
        } else {
          div_rn<W>(x, y, r);
        }
    }
    store<W>(r, out, ldo, i);
  }
}

template <int W>
__global__ void from_f64_kernel(const double* __restrict__ d, int64_t n, uint64_t* out,
                                int64_t ld, int* status) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = d[i];
    Num<W> r;
    if (!isfinite(v)) atomicCAS(status, 0, (int)MP_ERR_ARG);
    from_f64<W>(isfinite(v) ? v : 0.0, r);
    store<W>(r, out, ld, i);
  }
}

// The same two conversions for p > 1024 (L limbs, a thread per element): a
// double's 53-bit mantissa lands in the top limb; the nearest double takes
// the top 53 bits, the next bit and a sticky bit over all lower limbs.
__global__ void from_f64_wide_kernel(const double* __restrict__ d, int64_t n, uint64_t* out,
                                     int64_t ld, int L, int* status) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double v = d[i];
    if (!isfinite(v)) {
      atomicCAS(status, 0, (int)MP_ERR_ARG);
      v = 0.0;
    }
    uint64_t top = 0;
    int64_t e = EXP_ZERO;
    if (v != 0.0) {
      int ex = 0;
      top = (uint64_t)ldexp(frexp(fabs(v), &ex), 53) << 11;
      e = ex;
    }
    out[i] = pack_head(e, signbit(v) ? 1u : 0u);
    for (int k = 1; k < L; ++k) out[(int64_t)k * ld + i] = 0;
    out[(int64_t)L * ld + i] = top;
  }
}

__global__ void to_f64_wide_kernel(const uint64_t* __restrict__ a, int64_t n, int64_t ld, int L,
                                   double* d) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t e;
    uint32_t s;
    unpack_head(a[i], e, s);
    if (zero_e(e)) {
      d[i] = s ? -0.0 : 0.0;
      continue;
    }
    const uint64_t t = a[(int64_t)L * ld + i];
    uint64_t rest = 0;
    for (int k = 1; k < L; ++k) rest |= a[(int64_t)k * ld + i];
    uint64_t q = t >> 11;
    const uint64_t rb = (t >> 10) & 1u;
    const bool sticky = (t & 0x3ffu) != 0u || rest != 0u;
    if (rb && (sticky || (q & 1u))) q += 1u;
    const int64_t ec = e < -4000 ? -4000 : (e > 4000 ? 4000 : e);
    const double v = ldexp((double)q, (int)ec - 53);
    d[i] = s ? -v : v;
  }
}

template <int W>
__global__ void to_f64_kernel(const uint64_t* __restrict__ a, int64_t n, int64_t ld, double* d) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    Num<W> x;
    load<W>(x, a, ld, i);
    d[i] = to_f64<W>(x);
  }
}

}  // namespace

size_t dot_scratch_bytes(int prec, int k) {
  const int W = prec / 32;
  const int cap = (SPAN_CAP + 64 * W + 96) / 32 + 1;
  const int nb = dot_blocks(int64_t(1) << 40);  // the largest grid
  return 16 * sizeof(long long) + (size_t)(k < 1 ? 1 : k) * nb * cap * sizeof(int64_t);
}

mp_status launch_dot(int prec, const DotArgs& a, void* scratch, const int* gate,
                     cudaStream_t st) {
  if (a.k < 1 || a.k > 5) return set_error(MP_ERR_ARG, "dot count %d", a.k);
  return dispatch_w(prec, [&](auto w) {
    constexpr int W = decltype(w)::value;
    return dot_w<W>(a, scratch, gate, st);
  });
}

// Initialises the span slots at the head of a dot scratch buffer.
mp_status init_dot_scratch(void* scratch, cudaStream_t st) {
  long long* e = static_cast<long long*>(scratch);
  reset_span_slots<<<1, 32, 0, st>>>(e, e + 5);
  count_launch();
  return launch_check("reset_span_slots");
}

}  // namespace mpk

using namespace mpk;

namespace {
std::mutex g_init_mu;
bool g_dot_ready[64] = {};
size_t g_dot_bytes[64] = {};
}  // namespace

extern "C" {

mp_status mp_dot(mp_vec x, mp_vec y, mp_vec out, void* stream) {
  mp_status r;
  const bool big = prec_big(x.prec_bits);
  if (!prec_ok(x.prec_bits) && !big) return set_error(MP_ERR_PREC, "precision %d", x.prec_bits);
  if ((r = check_vec(x, x.n, x.prec_bits, "x")) != MP_OK) return r;
  if ((r = check_vec(y, x.n, x.prec_bits, "y")) != MP_OK) return r;
  if ((r = check_vec(out, 1, x.prec_bits, "out")) != MP_OK) return r;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t bytes = big ? dot_big_scratch_bytes(x.prec_bits) : dot_scratch_bytes(x.prec_bits, 1);
  int dev = 0;
  MPK_CUDA(cudaGetDevice(&dev));
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_init_mu);
    scratch = dot_scratch(bytes);
    if (!scratch) return set_error(MP_ERR_ALLOC, "dot scratch of %zu bytes", bytes);
    if (!g_dot_ready[dev] || g_dot_bytes[dev] < bytes) {
      if ((r = init_dot_scratch(scratch, st)) != MP_OK) return r;
      g_dot_ready[dev] = true;
      g_dot_bytes[dev] = bytes;
    }
  }
  if (big)
    return launch_dot_big(x.prec_bits, x.data, x.ld, y.data, y.ld, x.n, out.data, out.ld, scratch,
                          nullptr, st);
  DotArgs a;
  a.k = 1;
  a.n = x.n;
  a.x[0] = x.data;
  a.y[0] = y.data;
  a.ldx[0] = x.ld;
  a.ldy[0] = y.ld;
  a.out[0] = out.data;
  a.out_ld[0] = out.ld;
  return launch_dot(x.prec_bits, a, scratch, nullptr, st);
}

mp_status mp_axpy(mp_vec alpha, mp_vec x, mp_vec y, void* stream) {
  mp_status r;
  const bool big = prec_big(x.prec_bits);
  if (!prec_ok(x.prec_bits) && !big) return set_error(MP_ERR_PREC, "precision %d", x.prec_bits);
  if ((r = check_vec(alpha, 1, x.prec_bits, "alpha")) != MP_OK) return r;
  if ((r = check_vec(x, x.n, x.prec_bits, "x")) != MP_OK) return r;
  if ((r = check_vec(y, x.n, x.prec_bits, "y")) != MP_OK) return r;
  if (x.n == 0) return MP_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (big) return launch_axpy_big(x.prec_bits, alpha.data, x.n, x.data, x.ld, y.data, y.ld, st);
  return dispatch_w(x.prec_bits, [&](auto w) {
    constexpr int W = decltype(w)::value;
    axpy_kernel<W><<<ew_blocks(x.n), 256, 0, st>>>(alpha.data, x.n, x.data, x.ld, y.data, y.ld);
    count_launch();
    return launch_check("axpy_kernel");
  });
}

mp_status mp_ewise(int32_t op, mp_vec a, mp_vec b, mp_vec out, void* stream) {
  mp_status r;
  if (op < MP_OP_MUL || op > MP_OP_DIV) return set_error(MP_ERR_ARG, "op %d", op);
  if (!prec_ok(a.prec_bits)) return set_error(MP_ERR_PREC, "precision %d", a.prec_bits);
  if ((r = check_vec(b, a.n, a.prec_bits, "b")) != MP_OK) return r;
  if ((r = check_vec(out, a.n, a.prec_bits, "out")) != MP_OK) return r;
  if ((r = check_vec(a, a.n, a.prec_bits, "a")) != MP_OK) return r;
  if (a.n == 0) return MP_OK;
  int* status = status_word();
  if (!status) return set_error(MP_ERR_CUDA, "status word unavailable");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return dispatch_w(a.prec_bits, [&](auto w) {
    constexpr int W = decltype(w)::value;
    ewise_kernel<W><<<ew_blocks(a.n), 256, 0, st>>>(op, a.n, a.data, a.ld, b.data, b.ld,
                                                    out.data, out.ld, status);
    count_launch();
    return launch_check("ewise_kernel");
  });
}

mp_status mp_vec_from_f64(const double* d, mp_vec out, void* stream) {
  mp_status r;
  const bool big = prec_big(out.prec_bits);
  if (!prec_ok(out.prec_bits) && !big) return set_error(MP_ERR_PREC, "precision %d", out.prec_bits);
  if ((r = check_vec(out, out.n, out.prec_bits, "out")) != MP_OK) return r;
  if (out.n == 0) return MP_OK;
  if (!d) return set_error(MP_ERR_ARG, "d is null");
  int* status = status_word();
  if (!status) return set_error(MP_ERR_CUDA, "status word unavailable");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (big) {
    from_f64_wide_kernel<<<ew_blocks(out.n), 256, 0, st>>>(d, out.n, out.data, out.ld,
                                                           out.prec_bits / 64, status);
    count_launch();
    return launch_check("from_f64_wide_kernel");
  }
  return dispatch_w(out.prec_bits, [&](auto w) {
    constexpr int W = decltype(w)::value;
    from_f64_kernel<W><<<ew_blocks(out.n), 256, 0, st>>>(d, out.n, out.data, out.ld, status);
    count_launch();
    return launch_check("from_f64_kernel");
  });
}

mp_status mp_vec_to_f64(mp_vec a, double* d, void* stream) {
  mp_status r;
  const bool big = prec_big(a.prec_bits);
  if (!prec_ok(a.prec_bits) && !big) return set_error(MP_ERR_PREC, "precision %d", a.prec_bits);
  if ((r = check_vec(a, a.n, a.prec_bits, "a")) != MP_OK) return r;
  if (a.n == 0) return MP_OK;
  if (!d) return set_error(MP_ERR_ARG, "d is null");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (big) {
    to_f64_wide_kernel<<<ew_blocks(a.n), 256, 0, st>>>(a.data, a.n, a.ld, a.prec_bits / 64, d);
    count_launch();
    return launch_check("to_f64_wide_kernel");
  }
  return dispatch_w(a.prec_bits, [&](auto w) {
    constexpr int W = decltype(w)::value;
    to_f64_kernel<W><<<ew_blocks(a.n), 256, 0, st>>>(a.data, a.n, a.ld, d);
    count_launch();
    return launch_check("to_f64_kernel");
  });
}

}  // extern "C"

// ---------------------------------------------------------------------------
// mp_dot_noalloc: the exact dot product with its scratch in a fixed device
// array instead of memory from cudaMalloc.
//
// Some callers cannot let a library allocate device memory: a process whose
// GPU memory is owned by another allocator (a framework's caching allocator
// that has reserved the memory, a server held to a fixed memory budget) would
// see cudaMalloc fail or break its budget, and cudaMalloc/cudaFree can
// synchronise the device, which latency-bound callers must avoid.  mp_dot
// allocates its scratch on first use; this variant never does.  Its scratch
// is the file-scope array below, present on every GPU that loads the
// library until the process exits.
// ---------------------------------------------------------------------------

namespace mpk {
namespace {

constexpr int kNoAllocBlocks = 64;  // grid of the variant (grid-stride loops cover any n)
constexpr size_t kNoAllocSpanBytes = 16 * sizeof(long long);
constexpr size_t kNoAllocBytes =
    kNoAllocSpanBytes + (size_t)kNoAllocBlocks * DotWin<32>::cap * sizeof(int64_t);

static_assert(kNoAllocBytes == MP_DOT_NOALLOC_SCRATCH_BYTES, "scratch size stated in mpkrylov.h");

static __device__ __align__(256) unsigned char g_dot_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[64] = {};

// Device address of the array for the current device, looked up once per
// device (host code may not use the array's name as a device address).
mp_status noalloc_scratch(void** out) {
  int dev = 0;
  MPK_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return set_error(MP_ERR_CUDA, "device %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_dot_noalloc_scratch);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(g_dot_noalloc_scratch)");
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return MP_OK;
}

template <int W>
mp_status dot_noalloc_w(const DotDev& a, void* scratch, int* status, cudaStream_t st) {
  DotScratch s;
  s.emin = static_cast<long long*>(scratch);
  s.emax = s.emin + 5;
  s.partials = reinterpret_cast<int64_t*>(static_cast<unsigned char*>(scratch) + kNoAllocSpanBytes);
  int64_t b = (a.n + kDotThreads - 1) / kDotThreads;
  s.nblocks = (int)(b < 1 ? 1 : (b > kNoAllocBlocks ? kNoAllocBlocks : b));
  const size_t need = kNoAllocSpanBytes + (size_t)s.nblocks * DotWin<W>::cap * sizeof(int64_t);
  if (need > kNoAllocBytes)
    return set_error(MP_ERR_ARG, "mp_dot_noalloc needs %zu scratch bytes, the array holds %zu",
                     need, kNoAllocBytes);
  const size_t smem = dot_smem<W>(1);
  MPK_CUDA(cudaFuncSetAttribute(dot_accum_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
  // The array keeps the previous call's contents: the span slots must start
  // from (+inf, -inf); the partials are written before they are read.
  reset_span_slots<<<1, 32, 0, st>>>(s.emin, s.emax);
  dot_span_kernel<W><<<s.nblocks, kDotThreads, 0, st>>>(a, s.emin, s.emax, nullptr);
  dot_accum_kernel<W><<<s.nblocks, kDotThreads, smem, st>>>(a, s, nullptr);
  dot_finalize_kernel<W><<<1, 256, 0, st>>>(a, s, status, nullptr);
  count_launch(4);
  return launch_check("mp_dot_noalloc kernels");
}

}  // namespace
}  // namespace mpk

extern "C" {

mp_status mp_dot_noalloc(mp_vec x, mp_vec y, mp_vec out, void* stream) {
  mp_status r;
  if (!prec_ok(x.prec_bits)) return set_error(MP_ERR_PREC, "precision %d", x.prec_bits);
  if ((r = check_vec(x, x.n, x.prec_bits, "x")) != MP_OK) return r;
  if ((r = check_vec(y, x.n, x.prec_bits, "y")) != MP_OK) return r;
  if ((r = check_vec(out, 1, x.prec_bits, "out")) != MP_OK) return r;
  if (x.n > MP_DOT_NOALLOC_MAX_N)
    return set_error(MP_ERR_ARG, "mp_dot_noalloc: length %lld exceeds the maximum %lld",
                     (long long)x.n, (long long)MP_DOT_NOALLOC_MAX_N);
  void* scratch = nullptr;
  if ((r = noalloc_scratch(&scratch)) != MP_OK) return r;
  int* status = status_word();
  if (!status) return set_error(MP_ERR_CUDA, "status word unavailable");
  DotDev a{};
  a.k = 1;
  a.n = x.n;
  a.x[0] = x.data;
  a.y[0] = y.data;
  a.ldx[0] = x.ld;
  a.ldy[0] = y.ld;
  a.out[0] = out.data;
  a.out_ld[0] = out.ld;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return dispatch_w(x.prec_bits, [&](auto w) {
    constexpr int W = decltype(w)::value;
    return dot_noalloc_w<W>(a, scratch, status, st);
  });
}

}  // extern "C"
