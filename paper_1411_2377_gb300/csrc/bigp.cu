// bigp.cu -- CSR SpMV (ORDERED and EXACT), exact dot products and axpy at
// p = 2048, 4096 and 8192 bits, the precisions at which the paper's solves of
// Tables 1-2 converge.
//
// Above 1024 bits a value no longer fits in one thread's registers, so each
// value is handled by a whole warp.  Mantissas sit in the warp's slice of
// shared memory; the 32 lanes split the W^2 partial products of a product
// (lane l takes the schoolbook columns k = l mod 32, each column a 96-bit
// mad.lo.cc / madc.hi.cc / addc chain); carries, the sign, the leading bit and
// the rounding are resolved across the lanes, each lane owning a contiguous
// run of words (carries move up one lane per round by shuffles, a round-up
// increment by one ballot).  Four warp steps build every operation:
//   product   a*x exactly, as 64-bit counters per 32-bit digit;
//   window    a signed sum of terms placed at bit offsets, as counters;
//   resolve   counters -> 32-bit words and the sign;
//   round     leading bit, p bits, round to nearest, ties to even.
// The semantics are those of the p <= 1024 kernels and of Section 3:
// ORDERED y <- RN(y + RN(a x)) over the row in CSR column order from +0 with
// zero factors skipped; EXACT one rounding of the exact row sum (same span
// cap); a dot one rounding of the exact sum; axpy y <- RN(y + RN(alpha x)).
// The work is bound by the 32-bit multiplies ((p/32)^2 per product), not by
// bytes: at p = 2048 a stored nonzero carries 4096 multiplies for 264 bytes.
#include <climits>

#include "internal.h"
#include "mpdev.cuh"

namespace mpk {
namespace {

constexpr int kBigWarps = 4;
constexpr int kBigThreads = 32 * kBigWarps;
constexpr unsigned kFull = 0xffffffffu;
constexpr int64_t kMask32 = 0xffffffffLL;

// Per-warp shared memory: [cnt int64 x kCnt][acc int64 x kAcc (exact forms)]
// [A, X, Y, T: W words each][P0, P1, P2: 2W words each].
template <int W>
struct BigMem {
  static constexpr int kP = 32 * W;
  static constexpr int kCnt = 2 * W + 4;  // product counters, then the two-term window
  static constexpr int kAcc = (SPAN_CAP + 2 * kP + 96) / 32 + 2;  // exact window at the span cap
  __host__ __device__ static constexpr size_t bytes(bool exact) {
    return 8 * (size_t)(kCnt + (exact ? kAcc : 0)) + 4 * (size_t)(4 * W + 6 * W);
  }
};

struct WarpMem {
  int64_t* cnt;
  int64_t* acc;
  uint32_t *A, *X, *Y, *T, *P0, *P1, *P2;
};

template <int W>
__device__ __forceinline__ WarpMem carve(unsigned char* smem, int warp, bool exact) {
  unsigned char* b = smem + (size_t)warp * BigMem<W>::bytes(exact);
  WarpMem m;
  m.cnt = reinterpret_cast<int64_t*>(b);
  m.acc = m.cnt + BigMem<W>::kCnt;
  uint32_t* w = reinterpret_cast<uint32_t*>(m.cnt + BigMem<W>::kCnt + (exact ? BigMem<W>::kAcc : 0));
  m.A = w;
  m.X = w + W;
  m.Y = w + 2 * W;
  m.T = w + 3 * W;
  m.P0 = w + 4 * W;
  m.P1 = w + 6 * W;
  m.P2 = w + 8 * W;
  return m;
}

// ---- plane-major records <-> shared memory ----------------------------------

template <int W>
__device__ __forceinline__ void wload(uint32_t* dst, const uint64_t* __restrict__ v, int64_t ld,
                                      int64_t i, int lane) {
  for (int k = lane; k < W / 2; k += 32) {
    const uint64_t limb = __ldg(v + (int64_t)(k + 1) * ld + i);
    dst[2 * k] = (uint32_t)limb;
    dst[2 * k + 1] = (uint32_t)(limb >> 32);
  }
}

template <int W>
__device__ __forceinline__ void wstore(const uint32_t* src, int64_t e, uint32_t s,
                                       uint64_t* __restrict__ v, int64_t ld, int64_t i, int lane) {
  const bool z = zero_e(e);
  for (int k = lane; k < W / 2; k += 32)
    v[(int64_t)(k + 1) * ld + i] = z ? 0ull : ((uint64_t)src[2 * k] | ((uint64_t)src[2 * k + 1] << 32));
  if (lane == 0) v[i] = pack_head(z ? EXP_ZERO : e, s);
}

// ---- the four warp steps -----------------------------------------------------

// One step of a column sum: (c2:c1:c0) += u * v.
__device__ __forceinline__ void mac96(uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t u,
                                      uint32_t v) {
  asm("mad.lo.cc.u32 %0, %3, %4, %0;\n\t"
      "madc.hi.cc.u32 %1, %3, %4, %1;\n\t"
      "addc.u32 %2, %2, 0;"
      : "+r"(c0), "+r"(c1), "+r"(c2)
      : "r"(u), "r"(v));
}

// cnt[0 .. 2W+2) <- counters with sum_k cnt[k] 2^(32k) = a * b exactly (each
// in [0, 3 * 2^32)).  Column k of the schoolbook product, sum over i of
// a_i b_(k-i), is at most W (2^32-1)^2 < 2^72: three words (c0, c1, c2),
// which land on digits k, k+1, k+2.  A lane takes the column pairs
// (2g, 2g+1), g = lane (mod 32): the pair walks one range of i, and the b
// word of column 2g at step i is the one column 2g+1 needs at step i+1, so a
// step loads one a and one b word for two multiply-adds (out-of-range
// operands are taken as 0).  Pairs g and g + 32 t give every lane about the
// same number of steps.
template <int W>
__device__ __forceinline__ void wmul(const uint32_t* a, const uint32_t* b, const WarpMem& m,
                                     int lane) {
  for (int g = lane; g < W; g += 32) {
    const int k = 2 * g;
    const int lo = k < W ? 0 : k - W + 1, hi = k + 1 < W ? k + 1 : W - 1;
    uint32_t c0 = 0, c1 = 0, c2 = 0, d0 = 0, d1 = 0, d2 = 0;
    uint32_t bn = (k + 1 - lo <= W - 1) ? b[k + 1 - lo] : 0u;  // column k+1's b at i = lo
    for (int i = lo; i <= hi; ++i) {
      const uint32_t u = a[i];
      const uint32_t bk = (k - i >= 0) ? b[k - i] : 0u;
      mac96(c0, c1, c2, u, bk);
      mac96(d0, d1, d2, u, bn);
      bn = bk;
    }
    m.P0[k] = c0;
    m.P1[k] = c1;
    m.P2[k] = c2;
    m.P0[k + 1] = d0;
    m.P1[k + 1] = d1;
    m.P2[k + 1] = d2;
  }
  __syncwarp();
  for (int k = lane; k < 2 * W + 2; k += 32) {
    int64_t v = 0;
    if (k < 2 * W) v += m.P0[k];
    if (k >= 1 && k <= 2 * W) v += m.P1[k - 1];
    if (k >= 2) v += m.P2[k - 2];
    m.cnt[k] = v;
  }
  __syncwarp();
}

__device__ __forceinline__ void run_of(int n, int lane, int& b, int& e) {
  const int per = (n + 31) >> 5;
  b = min(lane * per, n);
  e = min(b + per, n);
}

// Signed counters c[0..n) -> words in [0, 2^32) (kept in the int64 slots).
// Returns the carry out of the top word: 0 for a non-negative total, -1 for a
// negative one (the window is sized so that the total fits).  Each lane
// resolves its own run; the carry out of lane l enters lane l+1 in the next
// round, so at most 32 rounds run.
__device__ __forceinline__ int64_t wresolve(int64_t* c, int n, int lane) {
  int b, e;
  run_of(n, lane, b, e);
  int64_t carry = 0;
  for (int i = b; i < e; ++i) {
    const int64_t v = c[i] + carry;
    c[i] = v & kMask32;
    carry = v >> 32;
  }
  int64_t top = 0;
  for (int round = 0; round < 33; ++round) {
    top += __shfl_sync(kFull, carry, 31);
    int64_t cin = __shfl_up_sync(kFull, carry, 1);
    if (lane == 0) cin = 0;
    if (!__any_sync(kFull, cin != 0)) break;
    for (int i = b; i < e && cin != 0; ++i) {
      const int64_t v = c[i] + cin;
      c[i] = v & kMask32;
      cin = v >> 32;
    }
    carry = cin;
  }
  return top;
}

// Two's complement of the words c[0..n): invert, then +1 (a lane takes the
// carry when every lower lane's run was all ones after the inversion).
__device__ __forceinline__ void wnegate(int64_t* c, int n, int lane) {
  int b, e;
  run_of(n, lane, b, e);
  bool ones = true;
  for (int i = b; i < e; ++i) {
    c[i] = (~c[i]) & kMask32;
    ones = ones && c[i] == kMask32;
  }
  const unsigned m = __ballot_sync(kFull, ones);
  const unsigned lower = (1u << lane) - 1u;
  if ((~m & lower) == 0u) {
    for (int i = b; i < e; ++i) {
      c[i] = (c[i] + 1) & kMask32;
      if (c[i] != 0) break;
    }
  }
}

// Index of the highest set bit of the words c[0..n), or -1 for zero.
__device__ __forceinline__ int wtopbit(const int64_t* c, int n, int lane) {
  int b, e;
  run_of(n, lane, b, e);
  int best = -1;
  for (int i = e - 1; i >= b; --i) {
    if (c[i] != 0) {
      best = i * 32 + 31 - __clz((unsigned)c[i]);
      break;
    }
  }
  return __reduce_max_sync(kFull, best);
}

// 32 bits of the integer c[0..n) starting at bit pos (bits outside are 0).
__device__ __forceinline__ uint32_t wbits32(const int64_t* c, int n, int64_t pos) {
  if (pos >= 32LL * n || pos <= -32) return 0u;
  const int64_t q = pos >> 5;
  const int r = (int)(pos & 31);
  const uint64_t lo = (q >= 0 && q < n) ? (uint64_t)(uint32_t)c[q] : 0ull;
  const uint64_t hi = (q + 1 < n) ? (uint64_t)(uint32_t)c[q + 1] : 0ull;
  return (uint32_t)(((hi << 32) | lo) >> r);
}

// out[0..W) <- the p = 32W bits of c[0..n) below and including bit B (the
// leading bit), rounded to nearest with ties to even on the bits below.
// Returns 1 when the rounding carried out of the top (the mantissa is then
// 2^(p-1) and the caller raises the exponent), else 0.
template <int W>
__device__ __forceinline__ int wround(const int64_t* c, int n, int B, uint32_t* out, int lane) {
  const int64_t s = (int64_t)B - 32 * W + 1;  // bit of c that becomes the result's lsb
  for (int j = lane; j < W; j += 32) out[j] = wbits32(c, n, s + 32 * (int64_t)j);
  uint32_t rbit = 0;
  bool sticky = false;
  if (s > 0) {
    const int64_t rb = s - 1;  // the round bit; sticky = any bit below it
    rbit = (uint32_t)(c[rb >> 5] >> (rb & 31)) & 1u;
    int b, e;
    run_of(n, lane, b, e);
    uint64_t any = 0;
    for (int i = b; i < e; ++i) {
      const int64_t w0 = 32LL * i;
      if (w0 + 32 <= rb)
        any |= (uint64_t)c[i];
      else if (w0 < rb)
        any |= (uint64_t)c[i] & ((1ull << (rb - w0)) - 1ull);
    }
    sticky = __any_sync(kFull, any != 0);
  }
  __syncwarp();
  if (!(rbit && (sticky || (out[0] & 1u)))) return 0;
  constexpr int per = W / 32;
  const int b = lane * per;
  bool ones = true;
  for (int i = b; i < b + per; ++i) ones = ones && out[i] == 0xffffffffu;
  const unsigned m = __ballot_sync(kFull, ones);
  const unsigned lower = (1u << lane) - 1u;
  if ((~m & lower) == 0u) {
    for (int i = b; i < b + per; ++i)
      if (++out[i] != 0u) break;
  }
  __syncwarp();
  if (m != kFull) return 0;
  for (int j = lane; j < W; j += 32) out[j] = (j == W - 1) ? 0x80000000u : 0u;
  __syncwarp();
  return 1;
}

// out <- RN(a * b) for nonzero a, b (mantissas in shared memory); e = ea + eb.
// Returns the result's exponent.
template <int W>
__device__ __forceinline__ int64_t wmul_rn(const uint32_t* a, const uint32_t* b, int64_t e,
                                           const WarpMem& m, uint32_t* out, int lane) {
  wmul<W>(a, b, m, lane);
  wresolve(m.cnt, 2 * W + 2, lane);
  __syncwarp();
  const int B = wtopbit(m.cnt, 2 * W + 2, lane);  // 2p-2 or 2p-1
  const int inc = wround<W>(m.cnt, 2 * W + 2, B, out, lane);
  return e + B + 1 - 64LL * W + inc;
}

// (Y, ye, ys) <- RN(y + t) for nonzero y and t.  Exact sum of the two on the
// grid of the smaller exponent, then one rounding; when the exponents differ
// by p + 2 or more the smaller is below a quarter ulp of the larger and the
// sum rounds to the larger.  An exact cancellation gives +0.
template <int W>
__device__ __forceinline__ void wadd(uint32_t* Y, int64_t& ye, uint32_t& ys, const uint32_t* T,
                                     int64_t te, uint32_t ts, int64_t* win, int lane) {
  const bool ybig = ye >= te;
  const uint32_t* big = ybig ? Y : T;
  const uint32_t* sml = ybig ? T : Y;
  const int64_t eb = ybig ? ye : te, es = ybig ? te : ye;
  const uint32_t sb = ybig ? ys : ts, ss = ybig ? ts : ys;
  const int64_t d = eb - es;
  if (d >= 32LL * W + 2) {
    if (!ybig) {
      for (int j = lane; j < W; j += 32) Y[j] = T[j];
      ye = te;
      ys = ts;
      __syncwarp();
    }
    return;
  }
  constexpr int N = 2 * W + 4;
  const bool sub = sb != ss;
  for (int i = lane; i < N; i += 32)
    win[i] = i < W ? (sub ? -(int64_t)sml[i] : (int64_t)sml[i]) : 0;
  __syncwarp();
  const int q = (int)(d >> 5), r = (int)(d & 31);
  for (int k = lane; k < W; k += 32) win[q + k] += (uint32_t)((uint64_t)big[k] << r);
  __syncwarp();
  for (int k = lane; k < W; k += 32) win[q + k + 1] += (uint32_t)(((uint64_t)big[k] << r) >> 32);
  __syncwarp();
  const bool neg = wresolve(win, N, lane) < 0;
  __syncwarp();
  if (neg) {
    wnegate(win, N, lane);
    __syncwarp();
  }
  const int B = wtopbit(win, N, lane);
  if (B < 0) {
    ye = EXP_ZERO;
    ys = 0u;
    return;
  }
  const int inc = wround<W>(win, N, B, Y, lane);
  ye = es + B + 1 - 32LL * W + inc;
  ys = sb ^ (neg ? 1u : 0u);
}

// acc[q ..] += (-1)^neg * (the 2W words in m.cnt) * 2^off, off = 32q + r.
template <int W>
__device__ __forceinline__ void wplace(int64_t* acc, const WarpMem& m, int64_t off, bool neg,
                                       int lane) {
  const int64_t q = off >> 5;
  const int r = (int)(off & 31);
  for (int k = lane; k < 2 * W; k += 32) {
    const int64_t v = (int64_t)(uint32_t)((uint64_t)m.cnt[k] << r);
    acc[q + k] += neg ? -v : v;
  }
  __syncwarp();
  for (int k = lane; k < 2 * W; k += 32) {
    const int64_t v = (int64_t)(uint32_t)(((uint64_t)m.cnt[k] << r) >> 32);
    acc[q + k + 1] += neg ? -v : v;
  }
  __syncwarp();
}

// Rounds the exact window acc[0..n) (bit i of weight 2^(e0 + i)) into
// (Y, e, s); an exactly zero window gives +0.
template <int W>
__device__ __forceinline__ void wfinish(int64_t* acc, int n, int64_t e0, uint32_t* Y, int64_t& e,
                                        uint32_t& s, int lane) {
  const bool neg = wresolve(acc, n, lane) < 0;
  __syncwarp();
  if (neg) {
    wnegate(acc, n, lane);
    __syncwarp();
  }
  const int B = wtopbit(acc, n, lane);
  if (B < 0) {
    e = EXP_ZERO;
    s = 0u;
    return;
  }
  const int inc = wround<W>(acc, n, B, Y, lane);
  e = e0 + B + 1 + inc;  // M 2^(e - p) with M's lsb at bit B - p + 1 of the window
  s = neg ? 1u : 0u;
}

__device__ __forceinline__ int exact_words(int64_t span, int W) {
  return (int)((span + 64LL * W + 96) / 32) + 1;
}

// ---- SpMV ----------------------------------------------------------------------

struct BigSell {
  int64_t nslots, nchunks;
  const int64_t* chunk_off;
  const int32_t* row_of;
  const int32_t* row_len;
  const int32_t* col;
  const uint64_t* val;
};

// Rows go to warps through a work counter (next, zero at launch): row slots
// come longest first (the layout sorts chunks by length), so the longest rows
// start first and the short ones fill in, which a fixed round-robin split of
// a few rows per warp cannot balance.
__device__ __forceinline__ int64_t next_row(unsigned* next, int lane) {
  unsigned r = 0;
  if (lane == 0) r = atomicAdd(next, 1u);
  return (int64_t)__shfl_sync(kFull, r, 0);
}

template <int W>
__global__ void __launch_bounds__(kBigThreads) big_ordered_kernel(BigSell S,
                                                                  const uint64_t* __restrict__ x,
                                                                  int64_t ldx, uint64_t* y,
                                                                  int64_t ldy, unsigned* next,
                                                                  const int* __restrict__ gate) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (gate && *gate) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const WarpMem m = carve<W>(smem, warp, false);
  const int64_t nrs = S.nchunks * 32;
  for (int64_t rs = next_row(next, lane); rs < nrs; rs = next_row(next, lane)) {
    const int row = S.row_of[rs];
    if (row < 0) continue;
    const int len = S.row_len[rs];
    const int64_t base = S.chunk_off[rs >> 5] + (rs & 31);
    int64_t ye = EXP_ZERO;
    uint32_t ys = 0u;
    for (int j = 0; j < len; ++j) {
      const int64_t slot = base + 32LL * j;
      int64_t ea, ex;
      uint32_t sa, sx;
      unpack_head(__ldg(S.val + slot), ea, sa);
      if (zero_e(ea)) continue;
      const int c = __ldg(S.col + slot);
      unpack_head(__ldg(x + c), ex, sx);
      if (zero_e(ex)) continue;
      wload<W>(m.A, S.val, S.nslots, slot, lane);
      wload<W>(m.X, x, ldx, c, lane);
      __syncwarp();
      const int64_t te = wmul_rn<W>(m.A, m.X, ea + ex, m, m.T, lane);
      const uint32_t ts = sa ^ sx;
      if (zero_e(ye)) {
        for (int k = lane; k < W; k += 32) m.Y[k] = m.T[k];
        ye = te;
        ys = ts;
        __syncwarp();
      } else {
        wadd<W>(m.Y, ye, ys, m.T, te, ts, m.cnt, lane);
      }
    }
    wstore<W>(m.Y, ye, ys, y, ldy, row, lane);
    __syncwarp();
  }
}

template <int W>
__global__ void __launch_bounds__(kBigThreads) big_exact_kernel(BigSell S,
                                                                const uint64_t* __restrict__ x,
                                                                int64_t ldx, uint64_t* y,
                                                                int64_t ldy, int* status,
                                                                unsigned* next,
                                                                const int* __restrict__ gate) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (gate && *gate) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const WarpMem m = carve<W>(smem, warp, true);
  const int64_t nrs = S.nchunks * 32;
  for (int64_t rs = next_row(next, lane); rs < nrs; rs = next_row(next, lane)) {
    const int row = S.row_of[rs];
    if (row < 0) continue;
    const int len = S.row_len[rs];
    const int64_t base = S.chunk_off[rs >> 5] + (rs & 31);
    // exponent span of the row's nonzero products, lanes over the entries
    long long lo = LLONG_MAX, hi = LLONG_MIN;
    for (int j = lane; j < len; j += 32) {
      const int64_t slot = base + 32LL * j;
      int64_t ea, ex;
      uint32_t sa, sx;
      unpack_head(__ldg(S.val + slot), ea, sa);
      if (zero_e(ea)) continue;
      unpack_head(__ldg(x + __ldg(S.col + slot)), ex, sx);
      if (zero_e(ex)) continue;
      lo = min(lo, (long long)(ea + ex));
      hi = max(hi, (long long)(ea + ex));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo = min(lo, __shfl_xor_sync(kFull, lo, o));
      hi = max(hi, __shfl_xor_sync(kFull, hi, o));
    }
    int64_t ye = EXP_ZERO;
    uint32_t ys = 0u;
    if (lo <= hi && hi - lo > SPAN_CAP) {
      if (lane == 0 && status) atomicCAS(status, 0, (int)MP_ERR_SPAN);
    } else if (lo <= hi) {
      const int n = exact_words(hi - lo, W);
      for (int i = lane; i < n; i += 32) m.acc[i] = 0;
      __syncwarp();
      for (int j = 0; j < len; ++j) {
        const int64_t slot = base + 32LL * j;
        int64_t ea, ex;
        uint32_t sa, sx;
        unpack_head(__ldg(S.val + slot), ea, sa);
        if (zero_e(ea)) continue;
        const int c = __ldg(S.col + slot);
        unpack_head(__ldg(x + c), ex, sx);
        if (zero_e(ex)) continue;
        wload<W>(m.A, S.val, S.nslots, slot, lane);
        wload<W>(m.X, x, ldx, c, lane);
        __syncwarp();
        wmul<W>(m.A, m.X, m, lane);
        wresolve(m.cnt, 2 * W + 2, lane);
        __syncwarp();
        wplace<W>(m.acc, m, ea + ex - lo, (sa ^ sx) != 0u, lane);
      }
      // bit i of the window weighs 2^(lo - 2p + i)
      wfinish<W>(m.acc, n, (int64_t)lo - 64LL * W, m.Y, ye, ys, lane);
    }
    wstore<W>(m.Y, ye, ys, y, ldy, row, lane);
    __syncwarp();
  }
}

// ---- dot -------------------------------------------------------------------------

// Span slots are the dot scratch's header (slot 0: lowest, slot 5: highest
// e_x + e_y), reset to (+inf, -inf) by the finalize for the next use.
__global__ void big_dot_span_kernel(const uint64_t* __restrict__ x, const uint64_t* __restrict__ y,
                                    int64_t n, long long* emin, long long* emax) {
  long long lo = LLONG_MAX, hi = LLONG_MIN;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t ex, ey;
    uint32_t sx, sy;
    unpack_head(__ldg(x + i), ex, sx);
    unpack_head(__ldg(y + i), ey, sy);
    if (zero_e(ex) || zero_e(ey)) continue;
    lo = min(lo, (long long)(ex + ey));
    hi = max(hi, (long long)(ex + ey));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = min(lo, __shfl_xor_sync(kFull, lo, o));
    hi = max(hi, __shfl_xor_sync(kFull, hi, o));
  }
  if ((threadIdx.x & 31) == 0 && lo <= hi) {
    atomicMin(emin, lo);
    atomicMax(emax, hi);
  }
}

// Each warp adds the exact products of its elements into its own window; the
// block then sums its four windows into one digit-major partial.
template <int W>
__global__ void __launch_bounds__(kBigThreads) big_dot_accum_kernel(
    const uint64_t* __restrict__ x, int64_t ldx, const uint64_t* __restrict__ y, int64_t ldy,
    int64_t n, const long long* __restrict__ span, int64_t* part, int nb) {
  extern __shared__ __align__(16) unsigned char smem[];
  const long long lo = span[0], hi = span[5];
  if (!(lo <= hi && hi - lo <= SPAN_CAP)) return;  // block-uniform
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const WarpMem m = carve<W>(smem, warp, true);
  const int nw = exact_words(hi - lo, W);
  for (int i = lane; i < nw; i += 32) m.acc[i] = 0;
  __syncwarp();
  for (int64_t i = (int64_t)blockIdx.x * kBigWarps + warp; i < n;
       i += (int64_t)gridDim.x * kBigWarps) {
    int64_t ex, ey;
    uint32_t sx, sy;
    unpack_head(__ldg(x + i), ex, sx);
    unpack_head(__ldg(y + i), ey, sy);
    if (zero_e(ex) || zero_e(ey)) continue;
    wload<W>(m.A, x, ldx, i, lane);
    wload<W>(m.X, y, ldy, i, lane);
    __syncwarp();
    wmul<W>(m.A, m.X, m, lane);
    wresolve(m.cnt, 2 * W + 2, lane);
    __syncwarp();
    wplace<W>(m.acc, m, ex + ey - lo, (sx ^ sy) != 0u, lane);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < nw; d += kBigThreads) {
    int64_t t = 0;
#pragma unroll
    for (int w = 0; w < kBigWarps; ++w) t += carve<W>(smem, w, true).acc[d];
    part[(int64_t)d * nb + blockIdx.x] = t;
  }
}

// One block: digit sums over the blocks (a warp per digit), then warp 0
// resolves, rounds and stores; resets the span slots.
template <int W>
__global__ void __launch_bounds__(256) big_dot_finalize_kernel(long long* span,
                                                               const int64_t* __restrict__ part,
                                                               int nb, uint64_t* out,
                                                               int64_t ldo, int* status) {
  extern __shared__ __align__(16) unsigned char smem[];
  const long long lo = span[0], hi = span[5];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const WarpMem m = carve<W>(smem, 0, true);
  int64_t e = EXP_ZERO;
  uint32_t s = 0u;
  if (lo <= hi && hi - lo <= SPAN_CAP) {
    const int nw = exact_words(hi - lo, W);
    for (int d = warp; d < nw; d += 8) {
      int64_t t = 0;
      for (int b = lane; b < nb; b += 32) t += part[(int64_t)d * nb + b];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(kFull, t, o);
      if (lane == 0) m.acc[d] = t;
    }
    __syncthreads();
    if (warp == 0) wfinish<W>(m.acc, nw, (int64_t)lo - 64LL * W, m.Y, e, s, lane);
  } else if (lo <= hi && threadIdx.x == 0 && status) {
    atomicCAS(status, 0, (int)MP_ERR_SPAN);
  }
  if (warp == 0) wstore<W>(m.Y, e, s, out, ldo, 0, lane);
  __syncthreads();
  if (threadIdx.x == 0) {
    span[0] = LLONG_MAX;
    span[5] = LLONG_MIN;
  }
}

// ---- axpy --------------------------------------------------------------------------

// y_i <- RN(y_i + RN(alpha x_i)), a warp per element (signed-zero rules of
// round-to-nearest: a zero product leaves y, +0 + -0 = +0, -0 + -0 = -0).
template <int W>
__global__ void __launch_bounds__(kBigThreads) big_axpy_kernel(const uint64_t* __restrict__ al,
                                                               int64_t n,
                                                               const uint64_t* __restrict__ x,
                                                               int64_t ldx, uint64_t* y,
                                                               int64_t ldy) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const WarpMem m = carve<W>(smem, warp, false);
  int64_t ea;
  uint32_t sa;
  unpack_head(__ldg(al), ea, sa);
  if (!zero_e(ea)) wload<W>(m.A, al, 1, 0, lane);
  __syncwarp();
  for (int64_t i = (int64_t)blockIdx.x * kBigWarps + warp; i < n;
       i += (int64_t)gridDim.x * kBigWarps) {
    int64_t ex, ey;
    uint32_t sx, sy;
    unpack_head(__ldg(x + i), ex, sx);
    unpack_head(y[i], ey, sy);
    __syncwarp();  // every lane has read y's head before lane 0 may rewrite it
    const uint32_t ts = sa ^ sx;
    if (zero_e(ea) || zero_e(ex)) {  // the product is a zero of sign ts
      if (zero_e(ey) && lane == 0) y[i] = pack_head(EXP_ZERO, sy & ts);
      continue;
    }
    wload<W>(m.X, x, ldx, i, lane);
    __syncwarp();
    const int64_t te = wmul_rn<W>(m.A, m.X, ea + ex, m, m.T, lane);
    if (zero_e(ey)) {
      wstore<W>(m.T, te, ts, y, ldy, i, lane);
    } else {
      wload<W>(m.Y, y, ldy, i, lane);
      __syncwarp();
      wadd<W>(m.Y, ey, sy, m.T, te, ts, m.cnt, lane);
      wstore<W>(m.Y, ey, sy, y, ldy, i, lane);
    }
    __syncwarp();
  }
}

// ---- host side ----------------------------------------------------------------------

template <class F>
mp_status dispatch_big(int p, F&& f) {
  switch (p) {
    case 2048: return f(std::integral_constant<int, 64>{});
    case 4096: return f(std::integral_constant<int, 128>{});
    case 8192: return f(std::integral_constant<int, 256>{});
    default: return set_error(MP_ERR_PREC, "precision %d not in {2048,4096,8192}", p);
  }
}

int big_sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

// Grid of a warp-per-unit kernel over `units`: resident blocks of all SMs at
// most (grid-stride loops cover the rest).
template <class K>
mp_status big_grid(K kernel, size_t smem, int64_t units, int* grid) {
  MPK_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  MPK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBigThreads, smem));
  if (per_sm < 1) return set_error(MP_ERR_CUDA, "no resident block for %zu shared bytes", smem);
  int64_t b = (units + kBigWarps - 1) / kBigWarps;
  const int64_t lim = (int64_t)big_sm_count() * per_sm;
  if (b > lim) b = lim;
  *grid = (int)(b < 1 ? 1 : b);
  return MP_OK;
}

template <int W>
int big_dot_blocks(int64_t n) {
  int64_t b = (n + 4 * kBigWarps - 1) / (4 * kBigWarps);  // about four elements per warp
  const int64_t lim = (int64_t)big_sm_count() * 2;
  if (b > lim) b = lim;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

mp_status launch_spmv_big(const mp_csr_s* M, const Sell& S, int mode, const uint64_t* x,
                          int64_t ldx, uint64_t* y, int64_t ldy, const int* gate,
                          cudaStream_t st) {
  if (S.nchunks == 0) return MP_OK;
  BigSell B{S.nslots, S.nchunks, S.chunk_off, S.row_of, S.row_len, S.col, S.val};
  // the matrix's overflow-list word (unused at these precisions) is the row counter
  unsigned* next = reinterpret_cast<unsigned*>(M->ovf);
  MPK_CUDA(cudaMemsetAsync(next, 0, sizeof(unsigned), st));
  return dispatch_big(M->prec, [&](auto w) -> mp_status {
    constexpr int W = decltype(w)::value;
    int grid = 0;
    mp_status r;
    if (mode == MP_ORDERED) {
      const size_t sm = (size_t)kBigWarps * BigMem<W>::bytes(false);
      if ((r = big_grid(big_ordered_kernel<W>, sm, S.nchunks * 32, &grid)) != MP_OK) return r;
      big_ordered_kernel<W><<<grid, kBigThreads, sm, st>>>(B, x, ldx, y, ldy, next, gate);
    } else {
      const size_t sm = (size_t)kBigWarps * BigMem<W>::bytes(true);
      if ((r = big_grid(big_exact_kernel<W>, sm, S.nchunks * 32, &grid)) != MP_OK) return r;
      int* status = status_word();
      if (!status) return set_error(MP_ERR_CUDA, "status word unavailable");
      big_exact_kernel<W><<<grid, kBigThreads, sm, st>>>(B, x, ldx, y, ldy, status, next, gate);
    }
    count_launch();
    return launch_check(mode == MP_ORDERED ? "big_ordered_kernel" : "big_exact_kernel");
  });
}

size_t dot_big_scratch_bytes(int prec) {
  const int W = prec / 32;
  const int nw = (SPAN_CAP + 64 * W + 96) / 32 + 2;
  return 16 * sizeof(long long) + (size_t)nw * (size_t)big_sm_count() * 2 * sizeof(int64_t);
}

mp_status launch_dot_big(int prec, const uint64_t* x, int64_t ldx, const uint64_t* y, int64_t ldy,
                         int64_t n, uint64_t* out, int64_t ldo, void* scratch, cudaStream_t st) {
  int* status = status_word();
  if (!status) return set_error(MP_ERR_CUDA, "status word unavailable");
  long long* span = static_cast<long long*>(scratch);
  int64_t* part = reinterpret_cast<int64_t*>(span + 16);
  return dispatch_big(prec, [&](auto w) -> mp_status {
    constexpr int W = decltype(w)::value;
    const int nb = big_dot_blocks<W>(n);
    const size_t sm = (size_t)kBigWarps * BigMem<W>::bytes(true);
    MPK_CUDA(cudaFuncSetAttribute(big_dot_accum_kernel<W>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    const size_t sm1 = BigMem<W>::bytes(true);
    MPK_CUDA(cudaFuncSetAttribute(big_dot_finalize_kernel<W>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1));
    int sgrid = (int)((n + 255) / 256);
    if (sgrid > big_sm_count() * 4) sgrid = big_sm_count() * 4;
    if (sgrid < 1) sgrid = 1;
    big_dot_span_kernel<<<sgrid, 256, 0, st>>>(x, y, n, span, span + 5);
    big_dot_accum_kernel<W><<<nb, kBigThreads, sm, st>>>(x, ldx, y, ldy, n, span, part, nb);
    big_dot_finalize_kernel<W><<<1, 256, sm1, st>>>(span, part, nb, out, ldo, status);
    count_launch(3);
    return launch_check("big dot kernels");
  });
}

mp_status launch_axpy_big(int prec, const uint64_t* al, int64_t n, const uint64_t* x, int64_t ldx,
                          uint64_t* y, int64_t ldy, cudaStream_t st) {
  if (n == 0) return MP_OK;
  return dispatch_big(prec, [&](auto w) -> mp_status {
    constexpr int W = decltype(w)::value;
    const size_t sm = (size_t)kBigWarps * BigMem<W>::bytes(false);
    int grid = 0;
    mp_status r;
    if ((r = big_grid(big_axpy_kernel<W>, sm, n, &grid)) != MP_OK) return r;
    big_axpy_kernel<W><<<grid, kBigThreads, sm, st>>>(al, n, x, ldx, y, ldy);
    count_launch();
    return launch_check("big_axpy_kernel");
  });
}

}  // namespace mpk
