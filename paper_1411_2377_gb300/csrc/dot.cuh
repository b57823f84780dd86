// dot.cuh -- exact dot products (the inner products (.,.) of Fig. 5) in two
// kernels, shared by mp_dot, mp_dot_noalloc and the solvers.
//
//  1. accumulate (a grid of nblocks x k: blockIdx.y is the dot, so the k
//     dots of a group run at once): each block first finds the exponent
//     range [lo_b, hi_b] of e_x + e_y over its own nonzero pairs (for its
//     dot), anchors its digit grid at
//     a_b = lo_b rounded down to a multiple of 32, and adds the exact 2p-bit
//     products into per-thread windows of 64-bit signed counters in shared
//     memory (digit-major, so a warp's accesses hit 32 banks; no atomics, no
//     carries); the block sums its threads' windows digit by digit into one
//     partial per block (digit-major across blocks).  A block whose own span
//     exceeds the per-thread windows takes one block-wide window with
//     shared-memory atomics instead.
//  2. finalize: one block per dot takes the global range (min of the lo_b,
//     max of the hi_b: the span cap is checked on it), anchors at A = lo
//     rounded down to a multiple of 32, and adds each block's partial into a
//     shared window at the block's digit offset (block b's digit d is global
//     digit d + (a_b - A)/32: whole digits; all threads stride over the
//     (block, digit) pairs, reading each block's digits coalesced, and add
//     them with 64-bit shared atomics -- exact integer addition, so the order
//     does not matter), resolves carries and rounds once.
// The last finalize block to finish (an arrival counter; nothing waits) can
// run a caller-supplied step on the results -- the solvers' scalar
// recurrences -- so that a solver iteration needs no separate scalar launch.
// Up to five dots over the same index range run in one pass.
#pragma once
#include <climits>
#include <type_traits>

#include "internal.h"
#include "mpdev.cuh"
#include "pdl.cuh"

namespace mpk {

constexpr int kDotThreads = 128;
constexpr int kDotWarps = kDotThreads / 32;
constexpr int kDotFastSpan = 1024;    // span (bits) the per-thread windows cover
constexpr int kDotMaxBlocks = 1024;   // grid bound of the accumulate kernel

__host__ __device__ inline int dot_digits(int64_t span, int W) {
  return (int)((span + 64 * W + 96) / 32) + 1;
}

template <int W>
struct DotWin {
  static constexpr int fast = (kDotFastSpan + 64 * W + 96) / 32 + 1;
  // a range up to the span cap, measured from its anchor (up to 31 bits lower)
  static constexpr int cap = (SPAN_CAP + 31 + 64 * W + 96) / 32 + 1;
};

struct DotDev {
  int k;
  int64_t n;
  const uint64_t* x[5];
  const uint64_t* y[5];
  int64_t ldx[5], ldy[5];
  uint64_t* out[5];
  int64_t out_ld[5];
};

// Scratch layout: a 16-word head (word 0: the finalize's arrival counter),
// then per (dot, block) the range lo/hi, then the partials [k][nblocks][cap]
// (block-major: a block's digits are contiguous, read coalesced by the
// finalize whatever the block's digit offset).
constexpr int kDotHeadWords = 16;

struct DotScratch {
  int* arrive;
  long long* lo;      // [5][nblocks]
  long long* hi;      // [5][nblocks]
  int64_t* partials;  // [5][nblocks][cap]
  int nblocks;
};

template <int W>
constexpr size_t dot_scratch_size(int k, int nblocks) {
  return (size_t)kDotHeadWords * 8 + (size_t)2 * k * nblocks * 8 +
         (size_t)k * nblocks * DotWin<W>::cap * 8;
}

template <int W>
inline DotScratch dot_scratch_view(void* base, int k, int nblocks) {
  DotScratch s;
  long long* h = static_cast<long long*>(base);
  s.arrive = reinterpret_cast<int*>(h);
  s.lo = h + kDotHeadWords;
  s.hi = s.lo + (size_t)k * nblocks;
  s.partials = reinterpret_cast<int64_t*>(s.hi + (size_t)k * nblocks);
  s.nblocks = nblocks;
  return s;
}

__device__ __forceinline__ int64_t warp_sum64(int64_t t) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  return t;
}

// smem of the accumulate kernel: per thread `fast` 64-bit counters,
// digit-major ([fast][threads]).
template <int W>
__host__ __device__ constexpr size_t dot_smem() {
  return (size_t)DotWin<W>::fast * kDotThreads * 8;
}

// Block-wide min and max (every thread returns them).
__device__ __forceinline__ void block_minmax(long long& lo, long long& hi, long long* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  __syncthreads();  // red may hold a previous call's values still being read
  if (lane == 0) {
    red[warp] = lo;
    red[32 + warp] = hi;
  }
  __syncthreads();
  lo = red[0];
  hi = red[32];
  for (int w = 1; w < nw; ++w) {
    lo = min(lo, red[w]);
    hi = max(hi, red[32 + w]);
  }
}

// P[0..2W) = a b exactly from radix-2^29 column sums (p >= 512): NA limbs
// of each operand, column sums C_k < 2^64 (at most NA products of < 2^58,
// plus a carry < 2^35), one carry pass into 29-bit digits, and the digits
// packed into 32-bit words as they are produced (the word count and bit
// position are compile-time constants of the unrolled loop).  One 32x32->64
// multiply-add per limb pair and no carry instructions, against three
// instructions per word product for the schoolbook rows.
template <int W>
__device__ __forceinline__ void mul_full_cols(const uint32_t (&a)[W], const uint32_t (&b)[W],
                                              uint32_t (&P)[2 * W]) {
  constexpr int NA = Cols<W>::NA;
  static_assert(2 * NA * kR >= 64 * W, "the digits cover the product");
  uint32_t al[NA], bl[NA];
  cut_limbs<W, NA>(a, al);
  cut_limbs<W, NA>(b, bl);
  uint64_t carry = 0u, buf = 0u;
  int nb = 0, w = 0;
#pragma unroll
  for (int k = 0; k < 2 * NA; ++k) {
    uint64_t acc = carry;
#pragma unroll
    for (int i = (k - NA + 1 > 0 ? k - NA + 1 : 0); i <= (k < NA - 1 ? k : NA - 1); ++i)
      acc += (uint64_t)al[i] * bl[k - i];
    carry = acc >> kR;
    buf |= (acc & kRMask) << nb;  // nb <= 31: at most 60 bits
    nb += kR;
    if (nb >= 32 && w < 2 * W) {
      P[w++] = (uint32_t)buf;
      buf >>= 32;
      nb -= 32;
    }
  }
#pragma unroll
  for (int j = 0; j < 2 * W; ++j)
    if (j >= w) {  // the product's top words not yet emitted (the loop ran out of digits)
      P[j] = (uint32_t)buf;
      buf >>= 32;
    }
}

// The elements one block takes for a dot: i = base + threadIdx.x + m stride
// (m >= 0) while i < end, read through map[i] when map is not null (a
// negative entry: no element).  The accumulate kernel's grid-stride share is
// (blockIdx.x T, gridDim.x T, n, null).
struct DotRange {
  int64_t base, stride, end;
  const int32_t* map;
};

// The partial of dot j over block b's elements of r (all kDotThreads threads
// of the block call it; block-uniform returns): the block's exponent range
// goes to s.lo/s.hi, its digits to s.partials.  dsm: dot_smem<W>() bytes of
// per-thread windows; acc: DotWin<W>::cap counters; red: 64 words.
template <int W>
__device__ void dot_block_partial(const DotDev& a, const DotScratch& s, int j, int b,
                                  const DotRange r, int64_t* dsm, int64_t* acc, long long* red) {
  constexpr int CAP = DotWin<W>::cap;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nb = s.nblocks;
  int64_t* c = dsm + threadIdx.x;
  auto index = [&](int64_t t) -> int64_t { return r.map ? (int64_t)__ldg(r.map + t) : t; };
  // this block's exponent range of the nonzero pairs (heads only)
  long long lo = LLONG_MAX, hi = LLONG_MIN;
  for (int64_t t = r.base + threadIdx.x; t < r.end; t += r.stride) {
    const int64_t i = index(t);
    if (i < 0) continue;
    int64_t ex, ey;
    uint32_t sx, sy;
    unpack_head(__ldg(a.x[j] + i), ex, sx);
    unpack_head(__ldg(a.y[j] + i), ey, sy);
    if (zero_e(ex) || zero_e(ey)) continue;
    lo = min(lo, (long long)(ex + ey));
    hi = max(hi, (long long)(ex + ey));
  }
  block_minmax(lo, hi, red);
  if (threadIdx.x == 0) {
    s.lo[(size_t)j * nb + b] = lo;
    s.hi[(size_t)j * nb + b] = hi;
  }
  // nothing to add, or a range the finalize rejects (the global span is
  // at least this block's): no partial is written or read
  if (!(lo <= hi && hi - lo <= SPAN_CAP)) return;  // block-uniform
  const long long anchor = (lo >> 5) * 32;            // lo rounded down to a multiple of 32
  const int nd = dot_digits(hi - anchor, W);
  int64_t* part = s.partials + ((size_t)j * nb + b) * CAP;
  if (hi - anchor > kDotFastSpan) {
    // a span beyond the per-thread windows: one block-wide window with
    // shared-memory atomics (rare: the solvers' vectors stay well inside)
    for (int d = threadIdx.x; d < nd; d += kDotThreads) acc[d] = 0;
    __syncthreads();
    for (int64_t t = r.base + threadIdx.x; t < r.end; t += r.stride) {
      const int64_t i = index(t);
      if (i < 0) continue;
      Num<W> x, y;
      load<W>(x, a.x[j], a.ldx[j], i);
      load<W>(y, a.y[j], a.ldy[j], i);
      if (zero_e(x.e) || zero_e(y.e)) continue;
      uint32_t P[2 * W], D[2 * W + 1];
      mul_full<W>(x.m, y.m, P);
      const int64_t off = x.e + y.e - anchor;
      shifted_digits<W>(P, (uint32_t)(off & 31), D);
      const bool ng = (x.s ^ y.s) != 0;
      for (int k = 0; k <= 2 * W; ++k) {
        const int64_t v = (int64_t)D[k];
        atomicAdd((unsigned long long*)&acc[(off >> 5) + k], (unsigned long long)(ng ? -v : v));
      }
    }
    __syncthreads();
    for (int d = threadIdx.x; d < nd; d += kDotThreads) part[d] = acc[d];
    return;
  }
  for (int d = 0; d < nd; ++d) c[d * kDotThreads] = 0;
  auto accumulate = [&](const Num<W>& x, const Num<W>& y) {
    if (zero_e(x.e) || zero_e(y.e)) return;
    uint32_t P[2 * W];
    if constexpr (W >= 16)
      mul_full_cols<W>(x.m, y.m, P);
    else
      mul_full<W>(x.m, y.m, P);
    add_term<W>(c, kDotThreads, P, x.e + y.e - anchor, x.s ^ y.s);
  };
  if constexpr (W <= 16) {
    // the next element's operands are loaded before the current one is
    // multiplied and added (its load latency overlaps that work)
    int64_t t = r.base + threadIdx.x;
    int64_t in = t < r.end ? index(t) : -1;
    Num<W> xn, yn;
    if (in >= 0) {
      load<W>(xn, a.x[j], a.ldx[j], in);
      load<W>(yn, a.y[j], a.ldy[j], in);
    }
    while (t < r.end) {
      const int64_t i = in;
      const Num<W> x = xn, y = yn;
      t += r.stride;
      in = t < r.end ? index(t) : -1;
      if (in >= 0) {
        load<W>(xn, a.x[j], a.ldx[j], in);
        load<W>(yn, a.y[j], a.ldy[j], in);
      }
      if (i >= 0) accumulate(x, y);
    }
  } else {
    for (int64_t t = r.base + threadIdx.x; t < r.end; t += r.stride) {
      const int64_t i = index(t);
      if (i < 0) continue;
      Num<W> x, y;
      load<W>(x, a.x[j], a.ldx[j], i);
      load<W>(y, a.y[j], a.ldy[j], i);
      accumulate(x, y);
    }
  }
  __syncthreads();
  for (int d = warp; d < nd; d += kDotWarps) {
    int64_t t = 0;
#pragma unroll
    for (int u = 0; u < kDotThreads / 32; ++u) t += dsm[d * kDotThreads + u * 32 + lane];
    t = warp_sum64(t);
    if (lane == 0) part[d] = t;
  }
}

template <int W>
__global__ void __launch_bounds__(kDotThreads) dot_accum_kernel(const DotDev a, DotScratch s,
                                                                const int* __restrict__ gate) {
  extern __shared__ int64_t dsm[];
  __shared__ int64_t acc[DotWin<W>::cap];  // the block-wide window of a wide block span
  __shared__ long long red[64];
  pdl_begin();
  if (gate && *gate) return;
  const DotRange r{blockIdx.x * (int64_t)kDotThreads, (int64_t)gridDim.x * kDotThreads, a.n,
                   nullptr};
  dot_block_partial<W>(a, s, (int)blockIdx.y, (int)blockIdx.x, r, dsm, acc, red);
}

// The finalize kernel's default: no step after the dots.  A step is called
// by the 32 threads of the last block's first warp with their lane index.
struct NoPost {
  __device__ void operator()(int) const {}
};

// Shared memory of one block's finalize of a dot.  The partials are summed
// into kFinGroups windows (the warps of a block split into groups) and the
// windows then into sum: many blocks' digits landing on the same few global
// digits would otherwise serialise on those addresses' shared atomics.
constexpr int kFinGroups = 4;

template <int W>
struct DotFinSmem {
  int64_t sum[DotWin<W>::cap];
  int64_t part[kFinGroups * DotWin<W>::cap];  // group g's window: part[g * nd ...]
  long long red[64];
  int off_of[kDotMaxBlocks];  // block b's digit offset (its nd_of[b] = 0: no partial)
  int nd_of[kDotMaxBlocks];
  int ndmax;
};

// Dot j by the calling block (any block size that is a multiple of 32): the
// global range from the blocks' ranges, the span cap, the partials summed
// per global digit, carries resolved, one rounding, stored to a.out[j].
template <int W>
__device__ void dot_finalize_one(const DotDev& a, const DotScratch& s, int j,
                                 int* __restrict__ status, DotFinSmem<W>& f) {
  const int nb = s.nblocks;
  const long long* blo = s.lo + (size_t)j * nb;
  const long long* bhi = s.hi + (size_t)j * nb;
  long long lo = LLONG_MAX, hi = LLONG_MIN;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    lo = min(lo, __ldcg(blo + b));
    hi = max(hi, __ldcg(bhi + b));
  }
  block_minmax(lo, hi, f.red);
  Num<W> r;
  set_zero(r, 0u);
  if (lo <= hi && hi - lo <= SPAN_CAP) {
    const long long A = (lo >> 5) * 32;
    const int nd = dot_digits(hi - A, W);
    if (threadIdx.x == 0) f.ndmax = 0;
    for (int d = threadIdx.x; d < kFinGroups * nd; d += blockDim.x) f.part[d] = 0;
    __syncthreads();
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
      const long long l = __ldcg(blo + b), h = __ldcg(bhi + b);
      int ndb = 0, off = 0;
      if (l <= h) {  // else no nonzero pairs in that block
        const long long ab = (l >> 5) * 32;
        off = (int)((ab - A) >> 5);
        ndb = dot_digits(h - ab, W);
      }
      f.off_of[b] = off;
      f.nd_of[b] = ndb;
      atomicMax(&f.ndmax, ndb);
    }
    __syncthreads();
    // every (block, digit) pair: block b's digit d enters global digit
    // d + off_of[b] by a shared 64-bit atomic add (integer: any order);
    // consecutive items are consecutive digits of one block (coalesced)
    const int m = f.ndmax;
    const int64_t* part = s.partials + (size_t)j * nb * DotWin<W>::cap;
    const int grp = (int)((threadIdx.x >> 5) % kFinGroups);
    int64_t* win = f.part + (size_t)grp * nd;
    for (int q = threadIdx.x; q < nb * m; q += blockDim.x) {
      const int b = q / m, d = q - b * m;
      if (d < f.nd_of[b])
        atomicAdd(reinterpret_cast<unsigned long long*>(&win[f.off_of[b] + d]),
                  (unsigned long long)__ldcg(part + (size_t)b * DotWin<W>::cap + d));
    }
    __syncthreads();
    for (int d = threadIdx.x; d < nd; d += blockDim.x) {
      int64_t t = 0;
#pragma unroll
      for (int g = 0; g < kFinGroups; ++g) t += f.part[(size_t)g * nd + d];
      f.sum[d] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      const uint32_t negative = resolve_digits(f.sum, 1, nd);
      if (negative) negate_words(f.sum, 1, nd);
      round_words<W>(f.sum, 1, nd, (int64_t)A - 64 * W, negative, r);
    }
  } else if (lo <= hi && threadIdx.x == 0 && status) {
    atomicCAS(status, 0, (int)MP_ERR_SPAN);
  }
  if (threadIdx.x == 0) store<W>(r, a.out[j], a.out_ld[j], 0);
}

// Counts one finished dot of a group of k on the scratch's arrival counter;
// true in the block that finished the last one (it then sees every dot's
// result: each is fenced before it is counted, and must be read with loads
// that bypass L1).  Called by every thread of the block.
__device__ __forceinline__ bool dot_arrive_last(const DotScratch& s, int k) {
  __shared__ int is_last;
  if (threadIdx.x == 0) {
    __threadfence();
    is_last = atomicAdd(s.arrive, 1) == k - 1;
    if (is_last) {
      atomicExch(s.arrive, 0);
      __threadfence();
    }
  }
  __syncthreads();
  return is_last != 0;
}

// One block per dot; the block that finishes last then runs post(lane) on
// its first warp.
template <int W, class Post = NoPost>
__global__ void __launch_bounds__(256) dot_finalize_kernel(const DotDev a, DotScratch s,
                                                           int* __restrict__ status,
                                                           const int* __restrict__ gate,
                                                           Post post) {
  __shared__ DotFinSmem<W> f;
  pdl_begin();
  if (gate && *gate) return;
  dot_finalize_one<W>(a, s, (int)blockIdx.x, status, f);
  if constexpr (!std::is_same<Post, NoPost>::value) {
    // one dot: this block is the last (its result is thread 0's own store)
    bool last = true;
    if (gridDim.x > 1)
      last = dot_arrive_last(s, (int)gridDim.x);
    else
      __syncthreads();
    if (last && threadIdx.x < 32) post((int)threadIdx.x);
  }
}

// Sets the head of a dot scratch buffer (the arrival counter) to zero.
template <int = 0>
__global__ void reset_dot_head(long long* head) {
  if (threadIdx.x < kDotHeadWords) head[threadIdx.x] = 0;
}

inline int dot_sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

// Blocks of the accumulate kernel: one per 128 elements, at most one wave
// of resident blocks (as many per SM as their digit windows fit in its
// shared memory, at most 4): more blocks would only add partials for the
// finalize to merge.
template <int W>
inline int dot_blocks(int64_t n) {
  int dev = 0, smem_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  const size_t per_block =
      dot_smem<W>() + sizeof(int64_t) * DotWin<W>::cap + sizeof(long long) * 64 + 1024;
  int fit = smem_sm > 0 ? (int)((size_t)smem_sm / per_block) : 1;
  fit = fit < 1 ? 1 : (fit > 4 ? 4 : fit);
  int64_t lim = (int64_t)dot_sm_count() * fit;
  if (lim > kDotMaxBlocks) lim = kDotMaxBlocks;
  int64_t b = (n + kDotThreads - 1) / kDotThreads;
  if (b > lim) b = lim;
  if (b < 1) b = 1;
  return (int)b;
}

// Launches the two kernels of k <= 5 dots on `st` (scratch: at least
// dot_scratch_size<W>(a.k, nblocks) bytes whose arrival counter is zero).
template <int W, class Post = NoPost>
mp_status dot_launch(const DotDev& a, void* scratch, int nblocks, int* status, const int* gate,
                     cudaStream_t st, Post post = Post()) {
  const DotScratch s = dot_scratch_view<W>(scratch, a.k, nblocks);
  const size_t smem = dot_smem<W>();
  MPK_CUDA(cudaFuncSetAttribute(dot_accum_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
  // streamed operands: shared memory for the windows matters more than L1
  MPK_CUDA(cudaFuncSetAttribute(dot_accum_kernel<W>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared));
  launch_pdl(dot_accum_kernel<W>, dim3(nblocks, a.k), dim3(kDotThreads), smem, st, a, s, gate);
  launch_pdl(dot_finalize_kernel<W, Post>, dim3(a.k), dim3(256), 0, st, a, s, status, gate, post);
  count_launch(2);
  return launch_check("dot kernels");
}

}  // namespace mpk
