// batch.cu -- many independent GPBiCG solves in one set of launches (not in
// the paper; its solver applied to a batch).
//
// K instances (system, right-hand side) of one precision are stacked into a
// block-diagonal matrix in the library's sliced layout, so one SpMV launch
// serves the whole batch.  Vectors are concatenated; instance k owns
// elements [off[k], off[k+1]).  Inner products are segmented: each block of
// the reduction kernels works inside one instance's range, and one finalize
// block per (instance, product) sums that instance's partial digit counters
// and rounds once.  Scalar recurrences run one thread per instance; vector
// updates look up each element's instance and leave finished instances
// untouched.  Each instance follows exactly the steps of mp_gpbicg (the same
// readings of Fig. 5), so its iterates equal a single-system solve bit for
// bit.  After the first iteration the whole batch iterates on the device in
// one graph launch: a conditional while node replays one captured iteration
// until the last instance finishes (or the time limit ends them).
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <vector>

#include "gpbicg.cuh"
#include "internal.h"
#include "mpdev.cuh"

struct mp_batch_s {
  mp_csr M = nullptr;
  int32_t k = 0;
  int32_t prec = 0;
  int64_t N = 0;
  std::vector<int64_t> off;  // host [k+1]
  int64_t* d_off = nullptr;  // device [k+1]
  int32_t* d_inst = nullptr; // device [N]
  // segmented reductions: block b covers [blk_lo[b], blk_hi[b]) of instance blk_inst[b]
  int32_t nblk = 0;
  int32_t* d_blk_inst = nullptr;
  int64_t* d_blk_lo = nullptr;
  int64_t* d_blk_hi = nullptr;
  int32_t* d_first = nullptr;  // [k] first block of each instance
  int32_t* d_count = nullptr;  // [k] blocks of each instance
};

// Compiled once per word count W = p/32 (MPK_W = 4, 8, 16, 32: the kernels
// and batch_entry<W>) and once with MPK_W = 0 (batch set-up and the C entry
// points), so that the precisions build in parallel.
#ifndef MPK_W
#define MPK_W 0
#endif

namespace mpk {

constexpr int64_t kBlkElems = 4096;   // elements per reduction block

template <int W>
mp_status batch_entry(mp_batch_s* B, const mp_vec& b, const mp_vec& x, const mp_solve_opts& o,
                      mp_solve_info* infos, cudaStream_t st);

}  // namespace mpk

#if MPK_W != 0
namespace mpk {
namespace {

constexpr int kBT = 128;              // threads of the reduction blocks
constexpr int kBW = kBT / 32;
constexpr int kBFast = 1024;          // per-warp exponent window (bits)

template <int W>
struct BWin {
  static constexpr int fast = (kBFast + 64 * W + 96) / 32 + 1;
  static constexpr int cap = (SPAN_CAP + 64 * W + 96) / 32 + 1;
};

__host__ __device__ inline int bdigits(int64_t span, int W) {
  return (int)((span + 64 * W + 96) / 32) + 1;
}

struct Seg {
  int32_t K, nblk;
  const int32_t* inst;
  const int32_t* blk_inst;
  const int64_t* blk_lo;
  const int64_t* blk_hi;
  const int32_t* first;
  const int32_t* count;
};

struct BState {
  int* done;         // [K]
  int* status;       // [K]
  long long* iters;  // [K]
  long long maxit;
  int* ndone;        // one word: instances finished
  int K;
  int has_loop;      // set in the captured iteration: `loop` runs it on the device
  cudaGraphConditionalHandle loop;
  unsigned long long* t0;       // device time (ns) at the set-up
  unsigned long long limit_ns;  // 0: no time limit
};

// Batched inner products: up to 5 pairs; out[j] is a K-vector of scalars.
struct BDot {
  int k;
  const uint64_t* x[5];
  const uint64_t* y[5];
  int64_t ld;
  uint64_t* out[5];  // plane-major K-vectors, ld = K
};

struct BScr {
  long long* emin;   // [5][K]
  long long* emax;   // [5][K]
  int64_t* partials; // [5][nblk][cap]
};

template <int W>
__global__ void __launch_bounds__(kBT) bdot_span_kernel(const BDot a, const Seg g, BScr s,
                                                        const int* done) {
  const int b = blockIdx.x;
  const int inst = g.blk_inst[b];
  if (done[inst]) return;
  const int64_t lo = g.blk_lo[b], hi = g.blk_hi[b];
  __shared__ long long rmin[kBW], rmax[kBW];
  for (int j = 0; j < a.k; ++j) {
    long long mn = LLONG_MAX, mx = LLONG_MIN;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
      int64_t ex, ey;
      uint32_t sx, sy;
      unpack_head(a.x[j][i], ex, sx);
      unpack_head(a.y[j][i], ey, sy);
      if (zero_e(ex) || zero_e(ey)) continue;
      mn = min(mn, (long long)(ex + ey));
      mx = max(mx, (long long)(ex + ey));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
      mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if ((threadIdx.x & 31) == 0) {
      rmin[threadIdx.x >> 5] = mn;
      rmax[threadIdx.x >> 5] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < kBW; ++w) {
        mn = min(mn, rmin[w]);
        mx = max(mx, rmax[w]);
      }
      if (mn <= mx) {
        atomicMin(s.emin + (size_t)j * g.K + inst, mn);
        atomicMax(s.emax + (size_t)j * g.K + inst, mx);
      }
    }
    __syncthreads();
  }
}

// smem: per thread FAST 64-bit counters, digit-major ([FAST][threads]).
template <int W>
__host__ __device__ constexpr size_t bdot_smem(int) {
  return (size_t)BWin<W>::fast * kBT * 8;
}

// Exact accumulation of one block's elements (one instance): each thread adds
// its pairs' products into its own counter window, then the block sums the
// windows digit by digit into the block's partial.
template <int W>
__global__ void __launch_bounds__(kBT) bdot_accum_kernel(const BDot a, const Seg g, BScr s,
                                                         const int* done) {
  extern __shared__ int64_t dsm[];
  const int b = blockIdx.x;
  const int inst = g.blk_inst[b];
  if (done[inst]) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t* c = dsm + threadIdx.x;
  const int64_t lo = g.blk_lo[b], hi = g.blk_hi[b];
  for (int j = 0; j < a.k; ++j) {
    const long long elo = s.emin[(size_t)j * g.K + inst], ehi = s.emax[(size_t)j * g.K + inst];
    if (!(elo <= ehi && (ehi - elo) <= kBFast)) continue;  // block-uniform
    const int nd = bdigits(ehi - elo, W);
    for (int d = 0; d < nd; ++d) c[d * kBT] = 0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += kBT) {
      Num<W> x, y;
      load<W>(x, a.x[j], a.ld, i);
      load<W>(y, a.y[j], a.ld, i);
      if (zero_e(x.e) || zero_e(y.e)) continue;
      uint32_t P[2 * W];
      if (W >= 16)
        mul_full_ilp<W>(x.m, y.m, P);
      else
        mul_full<W>(x.m, y.m, P);
      add_term<W>(c, kBT, P, x.e + y.e - elo, x.s ^ y.s);
    }
    __syncthreads();
    int64_t* part = s.partials + ((size_t)j * g.nblk + b) * BWin<W>::cap;
    for (int d = warp; d < nd; d += kBW) {
      int64_t t = 0;
#pragma unroll
      for (int u = 0; u < kBT / 32; ++u) t += dsm[d * kBT + u * 32 + lane];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0) part[d] = t;
    }
    __syncthreads();
  }
}

// Spans in (window, cap]: one block-wide window with shared atomics.
template <int W>
__global__ void __launch_bounds__(256) bdot_wide_kernel(const BDot a, const Seg g, BScr s,
                                                        const int* done) {
  __shared__ int64_t acc[BWin<W>::cap];
  const int b = blockIdx.x;
  const int inst = g.blk_inst[b];
  if (done[inst]) return;
  const int64_t lo = g.blk_lo[b], hi = g.blk_hi[b];
  for (int j = 0; j < a.k; ++j) {
    const long long elo = s.emin[(size_t)j * g.K + inst], ehi = s.emax[(size_t)j * g.K + inst];
    if (!(elo <= ehi && ehi - elo > kBFast && ehi - elo <= SPAN_CAP)) continue;
    const int nd = bdigits(ehi - elo, W);
    for (int d = threadIdx.x; d < nd; d += blockDim.x) acc[d] = 0;
    __syncthreads();
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
      Num<W> x, y;
      load<W>(x, a.x[j], a.ld, i);
      load<W>(y, a.y[j], a.ld, i);
      if (zero_e(x.e) || zero_e(y.e)) continue;
      uint32_t P[2 * W], D[2 * W + 1];
      mul_full<W>(x.m, y.m, P);
      const int64_t off = x.e + y.e - elo;
      shifted_digits<W>(P, (uint32_t)(off & 31), D);
      const bool ng = (x.s ^ y.s) != 0;
      for (int k = 0; k <= 2 * W; ++k) {
        const int64_t v = (int64_t)D[k];
        atomicAdd((unsigned long long*)&acc[(off >> 5) + k], (unsigned long long)(ng ? -v : v));
      }
    }
    __syncthreads();
    int64_t* part = s.partials + ((size_t)j * g.nblk + b) * BWin<W>::cap;
    for (int d = threadIdx.x; d < nd; d += blockDim.x) part[d] = acc[d];
    __syncthreads();
  }
}

// One block per (product, instance).
template <int W>
__global__ void __launch_bounds__(256) bdot_finalize_kernel(const BDot a, const Seg g, BScr s,
                                                            int* status, const int* done) {
  __shared__ int64_t sum[BWin<W>::cap];
  const int j = blockIdx.x / g.K, inst = blockIdx.x % g.K;
  if (done[inst]) return;
  const size_t slot = (size_t)j * g.K + inst;
  const long long lo = s.emin[slot], hi = s.emax[slot];
  Num<W> r;
  set_zero(r, 0u);
  if (lo <= hi && hi - lo <= SPAN_CAP) {
    const int nd = bdigits(hi - lo, W);
    const int b0 = g.first[inst], nb = g.count[inst];
    for (int d = threadIdx.x; d < nd; d += blockDim.x) {
      int64_t t = 0;
      for (int b = b0; b < b0 + nb; ++b) t += s.partials[((size_t)j * g.nblk + b) * BWin<W>::cap + d];
      sum[d] = t;
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
    store<W>(r, a.out[j], g.K, inst);
    s.emin[slot] = LLONG_MAX;
    s.emax[slot] = LLONG_MIN;
  }
}

__global__ void bspan_reset(long long* emin, long long* emax, int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    emin[i] = LLONG_MAX;
    emax[i] = LLONG_MIN;
  }
}

// ---- per-instance scalars: S_j is a K-vector (plane-major, ld = K) ---------

enum BScal { RHO, RHO_NEW, RHO_PREV, ALPHA, BETA, ZETA, ETA, DEN, MU1, MU2, MU3, MU4, MU5, RR, RR0, THR,
             NBS };

template <int W>
__device__ __forceinline__ void lds(Num<W>& a, const uint64_t* S, int K, int j, int k) {
  load<W>(a, S + (size_t)j * (W / 2 + 1) * K, K, k);
}
template <int W>
__device__ __forceinline__ void sts(const Num<W>& a, uint64_t* S, int K, int j, int k) {
  store<W>(a, S + (size_t)j * (W / 2 + 1) * K, K, k);
}

// Instance k ends; the thread that ends the last instance also ends the
// device-side loop that replays the iteration (one call: no race).
__device__ __forceinline__ void bfinish(const BState& b, int k, int status) {
  b.status[k] = status;
  b.done[k] = 1;
  if (atomicAdd(b.ndone, 1) + 1 == b.K && b.has_loop) cudaGraphSetConditional(b.loop, 0u);
}

#define INSTANCE_LOOP(k, K) \
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < (K); k += gridDim.x * blockDim.x)

template <int W>
__global__ void bsc_setup(BState b, uint64_t* S, int K, double rtol, double atol) {
  INSTANCE_LOOP(k, K) {
    Num<W> rt, at, T, A, t, thr, rr0, rho, z;
    from_f64<W>(rtol, rt);
    from_f64<W>(atol, at);
    mul_rn<W>(rt, rt, T);
    mul_rn<W>(at, at, A);
    lds<W>(rr0, S, K, RR0, k);
    mul_rn<W>(T, rr0, t);
    add_rn<W>(t, A, thr);
    sts<W>(thr, S, K, THR, k);
    set_zero(z, 0u);
    sts<W>(z, S, K, BETA, k);
    sts<W>(z, S, K, ETA, k);
    sts<W>(z, S, K, ZETA, k);
    lds<W>(rho, S, K, RHO, k);
    b.iters[k] = 0;
    b.status[k] = MP_OK;
    b.done[k] = 0;
    if (k == 0) *b.t0 = device_ns();
    if (cmp<W>(rr0, thr) <= 0)
      bfinish(b, k, MP_OK);
    else if (b.maxit <= 0)
      bfinish(b, k, MP_ERR_NOCONV);
    else if (zero_e(rho.e))
      bfinish(b, k, MP_ERR_BREAKDOWN);
  }
}

template <int W>
__global__ void bsc_alpha(BState b, uint64_t* S, int K) {
  INSTANCE_LOOP(k, K) {
    if (b.done[k]) continue;
    Num<W> rho, d, a;
    lds<W>(d, S, K, DEN, k);
    if (zero_e(d.e)) {
      bfinish(b, k, MP_ERR_BREAKDOWN);
      continue;
    }
    lds<W>(rho, S, K, RHO, k);
    div_rn<W>(rho, d, a);
    sts<W>(a, S, K, ALPHA, k);
  }
}

template <int W>
__global__ void bsc_zeta(BState b, uint64_t* S, int K, int first) {
  INSTANCE_LOOP(k, K) {
    if (b.done[k]) continue;
    Num<W> m1, m2, m3, m4, m5, x, y, c, tau, z;
    if (first) {
      lds<W>(m2, S, K, MU2, k);
      lds<W>(m5, S, K, MU5, k);
      if (zero_e(m5.e))
        set_zero(z, 0u);
      else
        div_rn<W>(m2, m5, z);
      sts<W>(z, S, K, ZETA, k);
      set_zero(z, 0u);
      sts<W>(z, S, K, ETA, k);
      continue;
    }
    lds<W>(m1, S, K, MU1, k);
    lds<W>(m4, S, K, MU4, k);
    lds<W>(m5, S, K, MU5, k);
    mul_rn<W>(m5, m1, x);
    mul_rn<W>(m4, m4, y);
    sub_rn<W>(x, y, tau);
    if (zero_e(tau.e)) {
      set_zero(z, 0u);
      sts<W>(z, S, K, ZETA, k);
      sts<W>(z, S, K, ETA, k);
      continue;
    }
    lds<W>(m2, S, K, MU2, k);
    lds<W>(m3, S, K, MU3, k);
    mul_rn<W>(m1, m2, x);
    mul_rn<W>(m3, m4, y);
    sub_rn<W>(x, y, c);
    div_rn<W>(c, tau, z);
    sts<W>(z, S, K, ZETA, k);
    mul_rn<W>(m5, m3, x);
    mul_rn<W>(m4, m2, y);
    sub_rn<W>(x, y, c);
    div_rn<W>(c, tau, z);
    sts<W>(z, S, K, ETA, k);
  }
}

template <int W>
__global__ void bsc_beta(BState b, uint64_t* S, int K) {
  INSTANCE_LOOP(k, K) {
    if (b.done[k]) continue;
    Num<W> rho, rp, q1, a, z, q2, bt;
    lds<W>(rho, S, K, RHO, k);
    lds<W>(rp, S, K, RHO_PREV, k);
    div_rn<W>(rho, rp, q1);
    lds<W>(a, S, K, ALPHA, k);
    lds<W>(z, S, K, ZETA, k);
    div_rn<W>(a, z, q2);
    mul_rn<W>(q1, q2, bt);
    sts<W>(bt, S, K, BETA, k);
  }
}

template <int W>
__global__ void bsc_check(BState b, uint64_t* S, int K) {
  INSTANCE_LOOP(k, K) {
    if (b.done[k]) continue;
    Num<W> rr, thr, rho, rn, z;
    b.iters[k] += 1;
    lds<W>(rr, S, K, RR, k);
    lds<W>(rho, S, K, RHO, k);
    lds<W>(rn, S, K, RHO_NEW, k);
    sts<W>(rho, S, K, RHO_PREV, k);
    sts<W>(rn, S, K, RHO, k);
    lds<W>(thr, S, K, THR, k);
    lds<W>(z, S, K, ZETA, k);
    if (cmp<W>(rr, thr) <= 0)
      bfinish(b, k, MP_OK);
    else if (zero_e(z.e))
      bfinish(b, k, MP_ERR_BREAKDOWN);
    else if (b.iters[k] >= b.maxit)
      bfinish(b, k, MP_ERR_NOCONV);
    else if (zero_e(rn.e))
      bfinish(b, k, MP_ERR_BREAKDOWN);
    else if (b.limit_ns != 0 && device_ns() - *b.t0 > b.limit_ns)
      bfinish(b, k, MP_ERR_TIMEOUT);
  }
}

// ---- vector updates (elements of finished instances are left alone) -------

#define ELEM_LOOP(i, N)                                                             \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (N);         \
       i += (int64_t)gridDim.x * blockDim.x)

template <int W>
__global__ void bcopy(const int* done, const int32_t* inst, const uint64_t* src, uint64_t* dst,
                      int64_t ld, int64_t N) {
  ELEM_LOOP(i, N) {
    if (done[inst[i]]) continue;
    for (int k = 0; k <= W / 2; ++k) dst[k * ld + i] = src[k * ld + i];
  }
}

template <int W>
__global__ void bzero(uint64_t* a, int64_t ld, int64_t N) {
  ELEM_LOOP(i, N) {
    Num<W> z;
    set_zero(z, 0u);
    store<W>(z, a, ld, i);
  }
}

struct BV {
  uint64_t* v[11];
  int64_t ld, N;
};

enum { VR, VRT, VP, VQ, VT, VV, VW, VY, VU, VZ, VS };

// The element steps are gpbicg.cuh's (the single solver's), per instance:
// its scalars are the K-vector entries of the element's instance.
template <int W>
__global__ void b_wp(const int* done, const int32_t* inst, const uint64_t* S, int K, const BV V) {
  ELEM_LOOP(i, V.N) {
    const int k = inst[i];
    if (done[k]) continue;
    Num<W> beta;
    lds<W>(beta, S, K, BETA, k);
    gp_wp_elem<W>(i, beta, V.v[VV], V.v[VQ], V.v[VR], V.v[VP], V.v[VU], V.v[VW], V.ld);
  }
}

template <int W>
__global__ void b_sty(const int* done, const int32_t* inst, const uint64_t* S, int K, const BV V,
                      int first) {
  ELEM_LOOP(i, V.N) {
    const int k = inst[i];
    if (done[k]) continue;
    Num<W> alpha;
    lds<W>(alpha, S, K, ALPHA, k);
    if (first) {  // t = r - alpha q;  y = alpha q - r
      Num<W> a, c, aq;
      load<W>(a, V.v[VQ], V.ld, i);
      mul_rn<W>(alpha, a, aq);
      load<W>(a, V.v[VR], V.ld, i);
      sub_rn<W>(a, aq, c);
      store<W>(c, V.v[VT], V.ld, i);
      sub_rn<W>(aq, a, c);
      store<W>(c, V.v[VY], V.ld, i);
      continue;
    }
    gp_sty_elem<W>(i, alpha, V.v[VR], V.v[VQ], V.v[VW], V.v[VS], V.v[VT], V.v[VY], V.ld);
  }
}

template <int W>
__global__ void b_uzxr(const int* done, const int32_t* inst, const uint64_t* S, int K, const BV V,
                       uint64_t* x, int64_t ldx) {
  Vecs U{};
  U.v[0] = V.v[VQ]; U.v[1] = V.v[VS]; U.v[2] = V.v[VU]; U.v[3] = V.v[VR]; U.v[4] = V.v[VZ];
  U.v[5] = V.v[VP]; U.v[6] = V.v[VT]; U.v[7] = V.v[VY]; U.v[8] = V.v[VV];
  U.ld = V.ld;
  U.n = V.N;
  ELEM_LOOP(i, V.N) {
    const int k = inst[i];
    if (done[k]) continue;
    Num<W> beta, eta, zeta, alpha;
    lds<W>(beta, S, K, BETA, k);
    lds<W>(eta, S, K, ETA, k);
    lds<W>(zeta, S, K, ZETA, k);
    lds<W>(alpha, S, K, ALPHA, k);
    gp_uzxr_elem<W>(i, beta, eta, zeta, alpha, U, x, ldx);
  }
}

int egrid(int64_t n) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t b = (n + 127) / 128;
  const int64_t lim = (int64_t)(sms > 0 ? sms : 1) * 8;
  return (int)(b < 1 ? 1 : (b > lim ? lim : b));
}

struct BWork {
  int K = 0, L = 0;
  int64_t N = 0;
  uint64_t* vecs = nullptr;  // 11 concatenated vectors, ld = N
  uint64_t* S = nullptr;     // NBS K-vectors
  int* words = nullptr;      // done[K], status[K], ndone
  long long* iters = nullptr;
  long long* span = nullptr;  // emin[5][K], emax[5][K]
  int64_t* partials = nullptr;
  uint64_t* vec(int k) const { return vecs + (size_t)k * (L + 1) * N; }
  uint64_t* scal(int j) const { return S + (size_t)j * (L + 1) * K; }
};

template <int W>
mp_status bdots(const BWork& w, const Seg& g, int k, const uint64_t* const* xs,
                const uint64_t* const* ys, const int* outs, cudaStream_t st) {
  BDot a{};
  a.k = k;
  a.ld = w.N;
  for (int j = 0; j < k; ++j) {
    a.x[j] = xs[j];
    a.y[j] = ys[j];
    a.out[j] = w.scal(outs[j]);
  }
  BScr s{w.span, w.span + 5 * (size_t)w.K, w.partials};
  const int* done = w.words;
  int* status = status_word();
  const size_t smem = bdot_smem<W>(k);
  MPK_CUDA(cudaFuncSetAttribute(bdot_accum_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
  MPK_CUDA(cudaFuncSetAttribute(bdot_accum_kernel<W>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared));
  bdot_span_kernel<W><<<g.nblk, kBT, 0, st>>>(a, g, s, done);
  bdot_accum_kernel<W><<<g.nblk, kBT, smem, st>>>(a, g, s, done);
  bdot_wide_kernel<W><<<g.nblk, 256, 0, st>>>(a, g, s, done);
  bdot_finalize_kernel<W><<<k * g.K, 256, 0, st>>>(a, g, s, status, done);
  count_launch(4);
  return launch_check("batched dots");
}

template <int W>
mp_status b_iteration(const mp_batch_s* B, const BWork& w, const Seg& g, const BState& bs,
                      const mp_vec& x, int mode, bool first, cudaStream_t st) {
  const int K = w.K;
  const int64_t N = w.N;
  const int eg = egrid(N);
  const int sg = (K + 127) / 128;
  BV V{};
  for (int k = 0; k < 11; ++k) V.v[k] = w.vec(k);
  V.ld = N;
  V.N = N;
  mp_status r;
  if (first) {
    bcopy<W><<<eg, 128, 0, st>>>(bs.done, g.inst, w.vec(VR), w.vec(VP), N, N);
    count_launch();
  } else {
    bsc_beta<W><<<sg, 128, 0, st>>>(bs, w.S, K);
    b_wp<W><<<eg, 128, 0, st>>>(bs.done, g.inst, w.S, K, V);
    count_launch(2);
  }
  if ((r = launch_spmv_batched(B->M, mode, w.vec(VP), N, w.vec(VQ), N, g.inst, w.words, st)) != MP_OK)
    return r;
  {
    const uint64_t* xs[1] = {w.vec(VRT)};
    const uint64_t* ys[1] = {w.vec(VQ)};
    const int outs[1] = {DEN};
    if ((r = bdots<W>(w, g, 1, xs, ys, outs, st)) != MP_OK) return r;
  }
  bsc_alpha<W><<<sg, 128, 0, st>>>(bs, w.S, K);
  b_sty<W><<<eg, 128, 0, st>>>(bs.done, g.inst, w.S, K, V, first ? 1 : 0);
  count_launch(2);
  if ((r = launch_spmv_batched(B->M, mode, w.vec(VT), N, w.vec(VV), N, g.inst, w.words, st)) != MP_OK)
    return r;
  if (first) {
    const uint64_t* xs[2] = {w.vec(VV), w.vec(VV)};
    const uint64_t* ys[2] = {w.vec(VT), w.vec(VV)};
    const int outs[2] = {MU2, MU5};
    if ((r = bdots<W>(w, g, 2, xs, ys, outs, st)) != MP_OK) return r;
  } else {
    const uint64_t* xs[5] = {w.vec(VY), w.vec(VV), w.vec(VY), w.vec(VV), w.vec(VV)};
    const uint64_t* ys[5] = {w.vec(VY), w.vec(VT), w.vec(VT), w.vec(VY), w.vec(VV)};
    const int outs[5] = {MU1, MU2, MU3, MU4, MU5};
    if ((r = bdots<W>(w, g, 5, xs, ys, outs, st)) != MP_OK) return r;
  }
  bsc_zeta<W><<<sg, 128, 0, st>>>(bs, w.S, K, first ? 1 : 0);
  b_uzxr<W><<<eg, 128, 0, st>>>(bs.done, g.inst, w.S, K, V, x.data, x.ld);
  count_launch(2);
  {
    const uint64_t* xs[2] = {w.vec(VR), w.vec(VRT)};
    const uint64_t* ys[2] = {w.vec(VR), w.vec(VR)};
    const int outs[2] = {RR, RHO_NEW};
    if ((r = bdots<W>(w, g, 2, xs, ys, outs, st)) != MP_OK) return r;
  }
  bsc_check<W><<<sg, 128, 0, st>>>(bs, w.S, K);
  count_launch();
  return launch_check("batched gpbicg iteration");
}

template <int W>
mp_status batch_solve_w(mp_batch_s* B, const mp_vec& b, const mp_vec& x,
                        const mp_solve_opts& o, mp_solve_info* infos, cudaStream_t st) {
  BWork w;
  w.K = B->k;
  w.L = W / 2;
  w.N = B->N;
  const int K = w.K;
  const int64_t N = w.N;
  const size_t cap = (size_t)BWin<W>::cap;
  auto free_all = [&]() {
    cudaFreeAsync(w.vecs, st);
    cudaFreeAsync(w.S, st);
    cudaFreeAsync(w.words, st);
    cudaFreeAsync(w.iters, st);
    cudaFreeAsync(w.span, st);
    cudaFreeAsync(w.partials, st);
    cudaStreamSynchronize(st);
  };
  cudaError_t ca = cudaMallocAsync((void**)&w.vecs, sizeof(uint64_t) * 11 * (w.L + 1) * (size_t)N, st);
  if (ca == cudaSuccess)
    ca = cudaMallocAsync((void**)&w.S, sizeof(uint64_t) * NBS * (w.L + 1) * (size_t)K, st);
  if (ca == cudaSuccess) ca = cudaMallocAsync((void**)&w.words, sizeof(int) * (2 * (size_t)K + 1), st);
  if (ca == cudaSuccess)
    ca = cudaMallocAsync((void**)&w.iters, sizeof(long long) * ((size_t)K + 1), st);
  if (ca == cudaSuccess) ca = cudaMallocAsync((void**)&w.span, sizeof(long long) * 10 * (size_t)K, st);
  if (ca == cudaSuccess)
    ca = cudaMallocAsync((void**)&w.partials, sizeof(int64_t) * 5 * (size_t)B->nblk * cap, st);
  if (ca != cudaSuccess) {
    free_all();
    return cuda_error(ca, "batch work memory");
  }
  Seg g{K, B->nblk, B->d_inst, B->d_blk_inst, B->d_blk_lo, B->d_blk_hi, B->d_first, B->d_count};
  BState bs{w.words, w.words + K, w.iters, (long long)o.maxit, w.words + 2 * K, K, 0, {},
             reinterpret_cast<unsigned long long*>(w.iters + K),
             (unsigned long long)o.time_limit_ms * 1000000ull};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, st);
  mp_status r = MP_OK;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int ndone = 0;
  do {
    cudaError_t cez = cudaMemsetAsync(w.words, 0, sizeof(int) * (2 * (size_t)K + 1), st);
    if (cez != cudaSuccess) { r = cuda_error(cez, "batch state reset"); break; }
    bspan_reset<<<egrid(5 * K), 128, 0, st>>>(w.span, w.span + 5 * (size_t)K, 5 * (int64_t)K);
    count_launch();
    const int eg = egrid(N);
    for (int k = 0; k < 11; ++k) {
      bzero<W><<<eg, 128, 0, st>>>(w.vec(k), N, N);
      count_launch();
    }
    // r0 = b - A x0 (exact rows), r~ = r0, (r0,r0), rho = (r~, r0)
    if ((r = launch_spmv(B->M, B->M->A, MP_EXACT, x.data, x.ld, w.vec(VR), N, b.data, b.ld, nullptr,
                         st)) != MP_OK)
      break;
    bcopy<W><<<eg, 128, 0, st>>>(w.words, B->d_inst, w.vec(VR), w.vec(VRT), N, N);
    count_launch();
    {
      const uint64_t* xs[2] = {w.vec(VR), w.vec(VRT)};
      const uint64_t* ys[2] = {w.vec(VR), w.vec(VR)};
      const int outs[2] = {RR0, RHO};
      if ((r = bdots<W>(w, g, 2, xs, ys, outs, st)) != MP_OK) break;
    }
    bsc_setup<W><<<(K + 127) / 128, 128, 0, st>>>(bs, w.S, K, o.rtol, o.atol);
    count_launch();
    if ((r = b_iteration<W>(B, w, g, bs, x, o.mode, true, st)) != MP_OK) break;
    cudaError_t cer = cudaMemcpyAsync(&ndone, bs.ndone, sizeof ndone, cudaMemcpyDeviceToHost, st);
    if (cer == cudaSuccess) cer = cudaStreamSynchronize(st);
    if (cer != cudaSuccess) { r = cuda_error(cer, "reading the batch state"); break; }
    if (ndone >= K) break;
    // The remaining iterations run on the device in one graph launch: a
    // conditional while node whose body is one captured iteration; the
    // instance that finishes last ends the loop (bfinish).
    cudaGraphConditionalHandle loop{};
    cudaGraphNodeParams cp{};
    cudaGraphNode_t node = nullptr;
    cudaError_t ce = cudaGraphCreate(&graph, 0);
    if (ce == cudaSuccess)
      ce = cudaGraphConditionalHandleCreate(&loop, graph, 1u, cudaGraphCondAssignDefault);
    if (ce == cudaSuccess) {
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = loop;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      ce = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
    }
    if (ce != cudaSuccess) { r = cuda_error(ce, "building the batched iteration loop"); break; }
    cudaGraph_t bodyg = cp.conditional.phGraph_out[0];
    BState lbs = bs;
    lbs.has_loop = 1;
    lbs.loop = loop;
    ce = cudaStreamBeginCaptureToGraph(st, bodyg, nullptr, nullptr, 0,
                                       cudaStreamCaptureModeRelaxed);
    if (ce != cudaSuccess) { r = cuda_error(ce, "cudaStreamBeginCaptureToGraph"); break; }
    const int64_t before = mp_launch_count(0);
    mp_status rb = b_iteration<W>(B, w, g, lbs, x, o.mode, false, st);
    const int64_t per = mp_launch_count(0) - before;
    ce = cudaStreamEndCapture(st, &bodyg);
    count_launch(-(int)per);
    if (rb != MP_OK) { r = rb; break; }
    if (ce != cudaSuccess) { r = cuda_error(ce, "cudaStreamEndCapture"); break; }
    ce = cudaGraphInstantiate(&exec, graph, 0);
    if (ce != cudaSuccess) { r = cuda_error(ce, "cudaGraphInstantiate"); break; }
    ce = cudaGraphLaunch(exec, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&ndone, bs.ndone, sizeof ndone, cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) { r = cuda_error(ce, "batched iteration loop"); break; }
  } while (false);
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  cudaEventRecord(e1, st);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  if (r == MP_OK && infos) {
    std::vector<int> status(K);
    std::vector<long long> iters(K);
    cudaMemcpyAsync(status.data(), w.words + K, sizeof(int) * K, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(iters.data(), w.iters, sizeof(long long) * K, cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    for (int k = 0; k < K; ++k) {
      infos[k].iters = iters[k];
      infos[k].status = status[k];
      infos[k].relres = 0.0;
      infos[k].ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  free_all();
  return r;
}

}  // namespace

template <int W>
mp_status batch_entry(mp_batch_s* B, const mp_vec& b, const mp_vec& x, const mp_solve_opts& o,
                      mp_solve_info* infos, cudaStream_t st) {
  return batch_solve_w<W>(B, b, x, o, infos, st);
}
template mp_status batch_entry<MPK_W>(mp_batch_s*, const mp_vec&, const mp_vec&,
                                      const mp_solve_opts&, mp_solve_info*, cudaStream_t);

}  // namespace mpk

#else  // MPK_W == 0

namespace mpk {
namespace {

template <class T>
mp_status upload(T** d, const std::vector<T>& h, cudaStream_t st) {
  MPK_CUDA(cudaMalloc((void**)d, sizeof(T) * std::max<size_t>(h.size(), 1)));
  if (!h.empty()) MPK_CUDA(cudaMemcpyAsync(*d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, st));
  return MP_OK;
}

}  // namespace
}  // namespace mpk

using namespace mpk;

extern "C" {

mp_status mp_batch_create_f64(int32_t k, const int64_t* n_each, const int64_t* const* rowptrs,
                              const int32_t* const* colidxs, const double* const* values,
                              int32_t prec_bits, void* stream, mp_batch* out) {
  if (!out) return set_error(MP_ERR_ARG, "out is null");
  *out = nullptr;
  if (k < 1) return set_error(MP_ERR_ARG, "batch of %d instances", k);
  if (!prec_ok(prec_bits)) return set_error(MP_ERR_PREC, "precision %d", prec_bits);
  if (!n_each || !rowptrs || !colidxs || !values) return set_error(MP_ERR_ARG, "null array");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::vector<int64_t> off(k + 1, 0);
  int64_t nnz = 0;
  for (int i = 0; i < k; ++i) {
    if (n_each[i] < 0 || !rowptrs[i]) return set_error(MP_ERR_ARG, "instance %d: bad size", i);
    off[i + 1] = off[i] + n_each[i];
    nnz += rowptrs[i][n_each[i]];
  }
  const int64_t N = off[k];
  if (N >= (int64_t(1) << 31)) return set_error(MP_ERR_ARG, "batch too large");
  // block-diagonal CSR: instance i's columns shifted by off[i]
  std::vector<int64_t> rp(N + 1, 0);
  std::vector<int32_t> ci;
  std::vector<double> va;
  ci.reserve(nnz);
  va.reserve(nnz);
  for (int i = 0; i < k; ++i) {
    const int64_t* r = rowptrs[i];
    if (r[0] != 0) return set_error(MP_ERR_ARG, "instance %d: rowptr[0] != 0", i);
    for (int64_t row = 0; row < n_each[i]; ++row) {
      for (int64_t e = r[row]; e < r[row + 1]; ++e) {
        const int32_t c = colidxs[i][e];
        if (c < 0 || c >= n_each[i])
          return set_error(MP_ERR_ARG, "instance %d row %lld: column %d out of range", i, (long long)row, c);
        ci.push_back((int32_t)(c + off[i]));
        va.push_back(values[i][e]);
      }
      rp[off[i] + row + 1] = (int64_t)ci.size();
    }
  }
  mp_csr M = nullptr;
  mp_status r = mp_csr_create_f64(N, rp.data(), ci.data(), va.data(), prec_bits, 0, stream, &M);
  if (r != MP_OK) return r;
  mp_batch_s* B = new (std::nothrow) mp_batch_s;
  if (!B) {
    mp_csr_destroy(M);
    return set_error(MP_ERR_ALLOC, "host allocation failed");
  }
  B->M = M;
  B->k = k;
  B->prec = prec_bits;
  B->N = N;
  B->off = off;
  std::vector<int32_t> inst(N);
  std::vector<int32_t> blk_inst, first(k), count(k);
  std::vector<int64_t> blk_lo, blk_hi;
  for (int i = 0; i < k; ++i) {
    for (int64_t e = off[i]; e < off[i + 1]; ++e) inst[e] = i;
    first[i] = (int32_t)blk_inst.size();
    int64_t lo = off[i];
    do {  // an instance with no rows still gets one (empty) block
      const int64_t hi = std::min(off[i + 1], lo + kBlkElems);
      blk_inst.push_back(i);
      blk_lo.push_back(lo);
      blk_hi.push_back(hi);
      lo = hi;
    } while (lo < off[i + 1]);
    count[i] = (int32_t)blk_inst.size() - first[i];
  }
  B->nblk = (int32_t)blk_inst.size();
  if ((r = upload(&B->d_off, off, st)) != MP_OK || (r = upload(&B->d_inst, inst, st)) != MP_OK ||
      (r = upload(&B->d_blk_inst, blk_inst, st)) != MP_OK ||
      (r = upload(&B->d_blk_lo, blk_lo, st)) != MP_OK ||
      (r = upload(&B->d_blk_hi, blk_hi, st)) != MP_OK ||
      (r = upload(&B->d_first, first, st)) != MP_OK ||
      (r = upload(&B->d_count, count, st)) != MP_OK) {
    mp_batch_destroy(B);
    return r;
  }
  cudaError_t ce = cudaStreamSynchronize(st);
  if (ce != cudaSuccess) {
    mp_batch_destroy(B);
    return cuda_error(ce, "batch upload");
  }
  *out = B;
  return MP_OK;
}

mp_status mp_batch_destroy(mp_batch B) {
  if (!B) return MP_OK;
  cudaDeviceSynchronize();
  mp_csr_destroy(B->M);
  cudaFree(B->d_off);
  cudaFree(B->d_inst);
  cudaFree(B->d_blk_inst);
  cudaFree(B->d_blk_lo);
  cudaFree(B->d_blk_hi);
  cudaFree(B->d_first);
  cudaFree(B->d_count);
  delete B;
  return MP_OK;
}

mp_status mp_batch_info(mp_batch B, int32_t* k, int64_t* total_n, int64_t* offsets) {
  if (!B) return set_error(MP_ERR_ARG, "batch is null");
  if (k) *k = B->k;
  if (total_n) *total_n = B->N;
  if (offsets) memcpy(offsets, B->off.data(), sizeof(int64_t) * (B->k + 1));
  return MP_OK;
}

mp_status mp_batch_matrix(mp_batch B, mp_csr* out) {
  if (!B || !out) return set_error(MP_ERR_ARG, "batch or out is null");
  *out = B->M;
  return MP_OK;
}

mp_status mp_batch_gpbicg(mp_batch B, mp_vec b, mp_vec x, const mp_solve_opts* opts,
                          mp_solve_info* infos, void* stream) {
  if (!B) return set_error(MP_ERR_ARG, "batch is null");
  if (!opts) return set_error(MP_ERR_ARG, "opts is null");
  mp_status r;
  if ((r = check_vec(b, B->N, B->prec, "b")) != MP_OK) return r;
  if ((r = check_vec(x, B->N, B->prec, "x")) != MP_OK) return r;
  if (b.data == x.data) return set_error(MP_ERR_ARG, "b and x must not alias");
  if (!(opts->rtol >= 0) || !(opts->atol >= 0) || opts->maxit < 0 ||
      (opts->mode != MP_ORDERED && opts->mode != MP_EXACT) || opts->transpose != 0 ||
      opts->history.data != nullptr)
    return set_error(MP_ERR_ARG, "unsupported batched solve options");
  if (!status_word()) return set_error(MP_ERR_CUDA, "status word unavailable");
  cudaStream_t cu = static_cast<cudaStream_t>(stream);
  cudaStream_t st = nullptr;
  cudaEvent_t fence = nullptr;
  if ((r = private_stream_open(cu, &st, &fence)) != MP_OK) return r;
  r = dispatch_w(B->prec, [&](auto w) {
    constexpr int W = decltype(w)::value;
    return batch_entry<W>(B, b, x, *opts, infos, st);
  });
  private_stream_close(cu, st, fence);
  return r;
}

}  // extern "C"

#endif  // MPK_W
