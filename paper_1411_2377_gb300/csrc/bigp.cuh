// bigp.cuh -- warp-level p-bit arithmetic for p = 2048, 4096, 8192 (one
// value per warp, mantissas in the warp's shared memory), shared by the
// products, dots and axpy (bigp.cu) and the solvers (bigp_solve.cu).
#pragma once
#include <climits>

#include "internal.h"
#include "mpdev.cuh"

namespace mpk {
namespace bigp {

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
  uint32_t* w =
      reinterpret_cast<uint32_t*>(m.cnt + BigMem<W>::kCnt + (exact ? BigMem<W>::kAcc : 0));
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
    v[(int64_t)(k + 1) * ld + i] =
        z ? 0ull : ((uint64_t)src[2 * k] | ((uint64_t)src[2 * k + 1] << 32));
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
// which land on digits k, k+1, k+2.  A lane takes column pairs (2g, 2g+1):
// the pair walks one range of i, and the b word of column 2g at step i is the
// one column 2g+1 needs at step i+1, so a step loads one a and one b word for
// two multiply-adds.  The W pairs are dealt out longest walk first, 32 per
// pass, so that the lanes of a pass (which run in lockstep) have walks of
// nearly equal length.
template <int W>
__device__ __forceinline__ void wmul(const uint32_t* a, const uint32_t* b, const WarpMem& m,
                                     int lane) {
  for (int r = lane; r < W; r += 32) {
    // pairs taken in order of their walk length (W, W-1, W-2, ...): the 32
    // lanes of one pass walk nearly the same number of steps
    const int g = (r & 1) ? W / 2 + (r >> 1) : W / 2 - 1 - (r >> 1);
    const int k = 2 * g;
    const int lo = k < W ? 0 : k - W + 1, hi = k + 1 < W ? k + 1 : W - 1;
    uint32_t c0 = 0, c1 = 0, c2 = 0, d0 = 0, d1 = 0, d2 = 0;
    uint32_t bn = (k + 1 - lo <= W - 1) ? b[k + 1 - lo] : 0u;  // column k+1's b at i = lo
    const int last = hi < k ? hi : k;  // i <= k: column k's b index stays >= 0
#pragma unroll 4
    for (int i = lo; i <= last; ++i) {
      const uint32_t u = a[i];
      const uint32_t bk = b[k - i];
      mac96(c0, c1, c2, u, bk);
      mac96(d0, d1, d2, u, bn);
      bn = bk;
    }
    if (hi > last) mac96(d0, d1, d2, a[hi], bn);  // i = k + 1 < W: column k+1 alone
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

// q = RN(a / b) for nonzero a, b (mantissas Ma, Mb in shared memory): the
// quotient Q = floor(N / Mb) of N = Ma 2^(p+2) by schoolbook long division in
// base 2^32 (Knuth, TAOCP vol. 2, 4.3.1, Algorithm D; Mb has its top bit set,
// so it needs no normalisation), then S = 2Q + [remainder != 0] rounded once
// (S carries the exact round and sticky bits; a quotient of two p-bit numbers
// is never exactly a midpoint).  Each of the W + 2 quotient words: the
// estimate from the top two words of the running remainder and the divisor's
// top two words (uniform across the warp), then the remainder window minus
// the estimate times Mb as signed 64-bit counters (lanes over words),
// resolved across lanes; a negative window takes Mb back once and the
// estimate one less.  U (2W + 2 words), C (W + 2 counters), Q (W + 4 words)
// and S (W + 5 counters) are shared-memory scratch.  Returns the exponent.
template <int W>
__device__ int64_t wdiv(const uint32_t* Ma, int64_t ea, const uint32_t* Mb, int64_t eb,
                        uint32_t* U, int64_t* C, uint32_t* Q, int64_t* S, uint32_t* out, int lane) {
  constexpr int n = W, m = W + 1, P = 32 * W, NQ = W + 4, NS = W + 5;
  for (int k = lane; k < 2 * W + 2; k += 32) {  // U = (4 Ma) 2^(32 W)
    uint32_t v = 0u;
    if (k >= W && k <= 2 * W) {
      const int i = k - W;
      const uint32_t lo = i < W ? Ma[i] : 0u, below = i > 0 ? Ma[i - 1] : 0u;
      v = (lo << 2) | (below >> 30);
    }
    U[k] = v;
  }
  for (int k = lane; k < NQ; k += 32) Q[k] = 0u;
  __syncwarp();
  const uint32_t v1 = Mb[n - 1], v2 = Mb[n - 2];
  const uint32_t vinv = (uint32_t)(~uint64_t(0) / v1);  // div2by1's reciprocal of v1
  for (int j = m; j >= 0; --j) {
    // estimate from the top two words (the top word never exceeds v1; when
    // equal the estimate is 2^32 - 1 with remainder U[j+n-1] + v1)
    uint64_t qh, rh;
    if (U[j + n] >= v1) {
      qh = 0xffffffffu;
      rh = (uint64_t)U[j + n - 1] + v1;
    } else {
      uint32_t rr;
      qh = div2by1(U[j + n], U[j + n - 1], v1, vinv, rr);
      rh = rr;
    }
    while ((rh >> 32) == 0u && qh * v2 > ((rh << 32) | U[j + n - 2])) {
      qh -= 1;
      rh += v1;
    }
    for (int k = lane; k <= n; k += 32) {
      const uint64_t t0 = k < n ? qh * Mb[k] : 0ull, t1 = k > 0 ? qh * Mb[k - 1] : 0ull;
      C[k] = (int64_t)U[j + k] - (int64_t)(uint32_t)t0 - (int64_t)(t1 >> 32);
    }
    __syncwarp();
    const int64_t top = wresolve(C, n + 1, lane);
    __syncwarp();
    if (top < 0) {  // the estimate was one too large
      qh -= 1;
      for (int k = lane; k < n; k += 32) C[k] += Mb[k];
      __syncwarp();
      wresolve(C, n + 1, lane);
      __syncwarp();
    }
    for (int k = lane; k <= n; k += 32) U[j + k] = (uint32_t)C[k];
    if (lane == 0) Q[j] = (uint32_t)qh;
    __syncwarp();
  }
  bool rnz = false;
  for (int k = lane; k < n; k += 32) rnz = rnz || U[k] != 0u;
  const uint32_t sticky = __any_sync(kFull, rnz) ? 1u : 0u;
  for (int k = lane; k < NS; k += 32) {  // S = 2 Q + sticky
    const uint32_t lo = (k < NQ) ? Q[k] : 0u, below = (k > 0) ? Q[k - 1] : 0u;
    S[k] = (int64_t)(uint32_t)((lo << 1) | (below >> 31) | (k == 0 ? sticky : 0u));
  }
  __syncwarp();
  const int B = wtopbit(S, NS, lane);
  const int inc = wround<W>(S, NS, B, out, lane);
  return (int64_t)B + 1 + ea - eb - P - 3 + inc;
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

// ---- host helpers ---------------------------------------------------------------

inline int big_sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

// Grid of a warp-per-unit kernel over `units`: at most the blocks all SMs
// hold at once (grid-stride loops and work counters cover the rest).
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

}  // namespace bigp
}  // namespace mpk
