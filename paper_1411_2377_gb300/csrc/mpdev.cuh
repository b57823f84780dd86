// mpdev.cuh -- device-side p-bit floating-point arithmetic for sm_103a.
//
// A value is (-1)^s * M * 2^(e-p) with 2^(p-1) <= M < 2^p (the MPFR convention
// 0.1xxx_2 * 2^e of the paper's Section 2), or a signed zero (e == EXP_ZERO).
// In registers the mantissa is W = p/32 little-endian 32-bit words; in memory a
// vector is plane-major: plane 0 holds head words e*2 + s, planes 1..L (L = W/2)
// the 64-bit limbs, least significant first.
//
// Every operation rounds to nearest with ties to even (MPFR's RN).  All loops
// over words have compile-time trip counts and are fully unrolled so the words
// stay in registers; variable shifts are done by log-depth barrel stages of
// predicated selects plus one funnel shift.
#pragma once
#include <cstdint>

#include "chains.cuh"

namespace mpk {

constexpr int64_t EXP_ZERO = -(int64_t(1) << 61);
constexpr int SPAN_CAP = 16384;  // largest exponent span an exact sum accepts

// The device's global nanosecond timer (solver time limits).
__device__ __forceinline__ unsigned long long device_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

template <int W>
struct Num {
  uint32_t m[W];
  int64_t e;
  uint32_t s;
};

__device__ __forceinline__ bool zero_e(int64_t e) { return e == EXP_ZERO; }

__device__ __forceinline__ void unpack_head(uint64_t h, int64_t& e, uint32_t& s) {
  const int64_t v = (int64_t)h;
  s = (uint32_t)(v & 1);
  e = v >> 1;  // arithmetic shift
}

__device__ __forceinline__ uint64_t pack_head(int64_t e, uint32_t s) {
  return (uint64_t)(e * 2 + (int64_t)s);
}

template <int W>
__device__ __forceinline__ void set_zero(Num<W>& r, uint32_t s) {
#pragma unroll
  for (int k = 0; k < W; ++k) r.m[k] = 0u;
  r.e = EXP_ZERO;
  r.s = s;
}

// ---------------------------------------------------------------------------
// Memory <-> registers (plane-major vectors)
// ---------------------------------------------------------------------------

template <int W>
__device__ __forceinline__ void load_limbs(uint32_t (&m)[W], const uint64_t* __restrict__ base,
                                           int64_t ld, int64_t i) {
#pragma unroll
  for (int k = 0; k < W / 2; ++k) {
    const uint64_t l = __ldg(base + (int64_t)(k + 1) * ld + i);
    m[2 * k] = (uint32_t)l;
    m[2 * k + 1] = (uint32_t)(l >> 32);
  }
}

template <int W>
__device__ __forceinline__ void load(Num<W>& a, const uint64_t* __restrict__ base, int64_t ld,
                                     int64_t i) {
  unpack_head(__ldg(base + i), a.e, a.s);
  load_limbs<W>(a.m, base, ld, i);
}

// As load, for data read once (a matrix's limbs): the limb words are loaded
// with the streaming (evict-first) cache hint so that they do not push
// reusable data (the gathered x) out of L2; the head keeps the normal path
// (EXACT reads it twice).
template <int W>
__device__ __forceinline__ void load_stream(Num<W>& a, const uint64_t* __restrict__ base,
                                            int64_t ld, int64_t i) {
  unpack_head(__ldg(base + i), a.e, a.s);
#pragma unroll
  for (int k = 0; k < W / 2; ++k) {
    const uint64_t l = __ldcs(base + (int64_t)(k + 1) * ld + i);
    a.m[2 * k] = (uint32_t)l;
    a.m[2 * k + 1] = (uint32_t)(l >> 32);
  }
}

template <int W>
__device__ __forceinline__ void store(const Num<W>& a, uint64_t* __restrict__ base, int64_t ld,
                                      int64_t i) {
  base[i] = pack_head(a.e, a.s);
#pragma unroll
  for (int k = 0; k < W / 2; ++k)
    base[(int64_t)(k + 1) * ld + i] = (uint64_t)a.m[2 * k] | ((uint64_t)a.m[2 * k + 1] << 32);
}

// ---------------------------------------------------------------------------
// Word-array helpers
// ---------------------------------------------------------------------------

// Carry-flag chains (chains.cuh) are whole inline-PTX statements: a chain's
// add.cc / addc.cc / mad*.cc steps and the carry flag between them are never
// split across statements.

// m += inc (inc in {0,1}); a carry out of the top means M reached 2^p, which is
// renormalised to 2^(p-1) with the exponent raised by one.
template <int W>
__device__ __forceinline__ void round_increment(uint32_t (&m)[W], int64_t& e, uint32_t inc) {
  const uint32_t c = chain_inc<W>(m, inc);
  if (c) {
    m[W - 1] = 0x80000000u;
    e += 1;
  }
}

// Right shift of N words by sh bits (0 <= sh < 32*N + 32); returns the OR of
// all bits shifted out (the sticky information).
template <int N, int NS>
__device__ __forceinline__ uint32_t shift_right_sticky(uint32_t (&x)[N], uint32_t sh) {
  uint32_t sticky = 0u;
  const uint32_t ws = sh >> 5, bs = sh & 31u;
#pragma unroll
  for (int st = 0; st < NS; ++st) {
    const int b = 1 << st;
    const bool on = (ws >> st) & 1u;
    uint32_t lost = 0u;
#pragma unroll
    for (int k = 0; k < b && k < N; ++k) lost |= x[k];
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const uint32_t src = (k + b < N) ? x[k + b] : 0u;
      x[k] = on ? src : x[k];
    }
    sticky |= on ? lost : 0u;
  }
  sticky |= (bs != 0u) ? (x[0] << (32u - bs)) : 0u;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const uint32_t hi = (k + 1 < N) ? x[k + 1] : 0u;
    x[k] = __funnelshift_r(x[k], hi, bs);
  }
  return sticky;
}

// Left shift of N words by sh bits (0 <= sh < 32*N), zeros shifted in.
template <int N, int NS>
__device__ __forceinline__ void shift_left(uint32_t (&x)[N], uint32_t sh) {
  const uint32_t ws = sh >> 5, bs = sh & 31u;
#pragma unroll
  for (int st = 0; st < NS; ++st) {
    const int b = 1 << st;
    const bool on = (ws >> st) & 1u;
#pragma unroll
    for (int k = N - 1; k >= 0; --k) {
      const uint32_t src = (k - b >= 0) ? x[k - b] : 0u;
      x[k] = on ? src : x[k];
    }
  }
#pragma unroll
  for (int k = N - 1; k >= 0; --k) {
    const uint32_t lo = (k > 0) ? x[k - 1] : 0u;
    x[k] = __funnelshift_l(lo, x[k], bs);
  }
}

template <int N>
__device__ __forceinline__ uint32_t count_leading_zeros(const uint32_t (&x)[N]) {
  uint32_t lz = 0u;
  bool found = false;
#pragma unroll
  for (int k = N - 1; k >= 0; --k) {
    const bool nz = x[k] != 0u;
    lz += found ? 0u : (nz ? (uint32_t)__clz(x[k]) : 32u);
    found = found || nz;
  }
  return lz;
}

// Stage count of a barrel shifter for word shifts 0..maxw.
__host__ __device__ constexpr int stages_for(int maxw) {
  return maxw <= 0 ? 0 : (maxw < 2 ? 1 : 1 + stages_for(maxw / 2));
}

// r[0..2W) = a * b, schoolbook over 32-bit words.  Row i adds a_i*b in two
// carry chains: the low halves of a_i*b_j into r[i+j], then the high halves
// into r[i+j+1]; each 32x32 product costs one mad.lo and one mad.hi and no
// separate carry additions.  r[i+W] holds the previous row's final carry
// when row i starts.
template <int W>
__device__ __forceinline__ void mul_full(const uint32_t (&a)[W], const uint32_t (&b)[W],
                                         uint32_t (&r)[2 * W]) {
  uint32_t R[2 * W + 1];  // R[2W] takes the top row's final carry (zero)
#pragma unroll
  for (int k = 0; k <= 2 * W; ++k) R[k] = 0u;
#pragma unroll
  for (int i = 0; i < W; ++i) {
    uint32_t win[W + 2];
#pragma unroll
    for (int k = 0; k < W + 2; ++k) win[k] = (i + k <= 2 * W) ? R[i + k] : 0u;
    chain_mul_row<W>(win, a[i], b);
#pragma unroll
    for (int k = 0; k < W + 2; ++k)
      if (i + k <= 2 * W) R[i + k] = win[k];
  }
#pragma unroll
  for (int k = 0; k < 2 * W; ++k) r[k] = R[k];
}

// As mul_full, written with 64-bit products and plain additions: no carry
// flag is involved, so the compiler can overlap the independent products of a
// row (more instruction-level parallelism, more ALU instructions).  Used where
// few warps share an SM.
template <int W>
__device__ __forceinline__ void mul_full_ilp(const uint32_t (&a)[W], const uint32_t (&b)[W],
                                             uint32_t (&r)[2 * W]) {
#pragma unroll
  for (int k = 0; k < 2 * W; ++k) r[k] = 0u;
#pragma unroll
  for (int i = 0; i < W; ++i) {
    uint32_t carry = 0u;
#pragma unroll
    for (int j = 0; j < W; ++j) {
      const uint64_t t = (uint64_t)a[i] * b[j] + r[i + j] + carry;
      r[i + j] = (uint32_t)t;
      carry = (uint32_t)(t >> 32);
    }
    r[i + W] = carry;
  }
}

// ---------------------------------------------------------------------------
// Correctly rounded operations
// ---------------------------------------------------------------------------

// r = RN(a*b).  The exact product Ma*Mb has 2p or 2p-1 bits; keep the top p
// bits, round with the next bit and the OR of the rest.
template <int W>
__device__ __forceinline__ void mul_rn(const Num<W>& a, const Num<W>& b, Num<W>& r) {
  const uint32_t s = a.s ^ b.s;
  if (zero_e(a.e) || zero_e(b.e)) {
    set_zero(r, s);
    return;
  }
  uint32_t P[2 * W];
  mul_full<W>(a.m, b.m, P);
  const uint32_t sh = 1u - (P[2 * W - 1] >> 31);  // 1 when the product has 2p-1 bits
#pragma unroll
  for (int k = 0; k < W; ++k) r.m[k] = __funnelshift_l(P[W + k - 1], P[W + k], sh);
  const uint32_t g = P[W - 1] << sh;
  uint32_t st = g << 1;
#pragma unroll
  for (int k = 0; k < W - 1; ++k) st |= P[k];
  r.e = a.e + b.e - (int64_t)sh;
  r.s = s;
  round_increment<W>(r.m, r.e, (g >> 31) & ((st != 0u) | (r.m[0] & 1u)));
}

// r = RN(a+b) with the IEEE/MPFR signed-zero rules of round-to-nearest:
// (+0)+(-0) = +0, (-0)+(-0) = -0, x + (+-0) = x, exact cancellation = +0.
//
// The operand of larger magnitude X and the other one Y sit in a frame of
// W+1 words whose low word guards the kept bits; Y is shifted right by the
// exponent difference d, bits below the frame collapsing into `sticky`.  One
// carry chain forms X + Y (same signs) or X - Y - [sticky != 0] = X + ~Y +
// [sticky == 0] (opposite signs): the true difference exceeds that floor by
// less than one guard unit, and sticky stays set.  The (W+2)-word result is
// normalised by one left shift that puts its leading one at the top (a
// carry-out gives a shift of 31, cancellation more than 32), then rounded.
template <int W>
__device__ __forceinline__ void add_rn(const Num<W>& a_, const Num<W>& b_, Num<W>& r) {
  const bool az = zero_e(a_.e), bz = zero_e(b_.e);
  if (az | bz) {
    if (az & bz) {
      set_zero(r, a_.s & b_.s);
    } else {
      r = az ? b_ : a_;
    }
    return;
  }
  // |b| > |a| ?  (exponents first, mantissas only when they tie)
  const uint32_t mlt = chain_borrow<W>(a_.m, b_.m);
  const bool sw = (b_.e > a_.e) || (b_.e == a_.e && mlt);
  uint32_t X[W + 1], Y[W + 1];
  X[0] = 0u;
  Y[0] = 0u;
#pragma unroll
  for (int k = 0; k < W; ++k) {
    X[k + 1] = sw ? b_.m[k] : a_.m[k];
    Y[k + 1] = sw ? a_.m[k] : b_.m[k];
  }
  int64_t e = sw ? b_.e : a_.e;
  const uint32_t s = sw ? b_.s : a_.s;
  const uint32_t ys = sw ? a_.s : b_.s;
  const int64_t d = sw ? (b_.e - a_.e) : (a_.e - b_.e);
  if (d >= (int64_t)(32 * W + 2)) {
    // |smaller| < ulp(larger)/4: the larger operand is the rounded sum.
#pragma unroll
    for (int k = 0; k < W; ++k) r.m[k] = X[k + 1];
    r.e = e;
    r.s = s;
    return;
  }
  const uint32_t sticky = shift_right_sticky<W + 1, stages_for(W)>(Y, (uint32_t)d);
  const uint32_t sub = (s != ys) ? 1u : 0u;
  const uint32_t inv = 0u - sub;
  uint32_t T[W + 2], Yi[W + 1];
#pragma unroll
  for (int k = 0; k <= W; ++k) Yi[k] = Y[k] ^ inv;
  // X[0] is 0, so the carry-in enters through the low word
  chain_add_frame<W>(T, X, Yi, sub & (sticky == 0u ? 1u : 0u));
  T[W + 1] &= (sub ^ 1u);
  uint32_t rb, st;
  const uint32_t carry = T[W + 1] & 1u;
  if (carry == 0u && T[W] == 0u) {
    // 32 or more leading bits cancelled (a difference with d <= 1 only), or
    // all of them: count the leading zeros and shift them out
    uint32_t any = 0u;
#pragma unroll
    for (int k = 0; k < W + 2; ++k) any |= T[k];
    if (any == 0u) {  // exact cancellation
      set_zero(r, 0u);
      return;
    }
    const uint32_t lz = count_leading_zeros<W + 2>(T);
    shift_left<W + 2, stages_for(W + 1)>(T, lz);
    e += 32 - (int64_t)lz;
    rb = T[1] >> 31;
    st = (T[1] << 1) | T[0] | sticky;
#pragma unroll
    for (int k = 0; k < W; ++k) r.m[k] = T[k + 2];
  } else {
    // the leading one is the carry out (bit 32W+32 of T) or a bit of T[W]
    // (lz0 = its leading zeros: 0 for a sum without carry, 1 for a far
    // difference, up to 31 for a near one).  With U = T one word down on a
    // carry, the kept words are the funnel shifts of U by s = 31 (carry) or
    // lz0; the word below them gives the round bit and, with what U drops
    // and the frame's sticky bit, the sticky bit.  One path for every lane.
    const uint32_t lz0 = __clz(T[W]);
    const uint32_t sh = carry ? 31u : lz0;
    uint32_t U[W + 1];
#pragma unroll
    for (int k = 0; k <= W; ++k) U[k] = carry ? T[k + 1] : T[k];
    const uint32_t um1 = carry ? T[0] : 0u;
#pragma unroll
    for (int k = 0; k < W; ++k) r.m[k] = __funnelshift_l(U[k], U[k + 1], sh);
    const uint32_t v = __funnelshift_l(um1, U[0], sh);
    rb = v >> 31;
    st = (v << 1) | (um1 << sh) | sticky;
    e += carry ? (int64_t)1 : -(int64_t)lz0;
  }
  r.e = e;
  r.s = s;
  round_increment<W>(r.m, r.e, rb & ((st != 0u) | (r.m[0] & 1u)));
}

template <int W>
__device__ __forceinline__ void neg(Num<W>& a) {
  a.s ^= 1u;
}

template <int W>
__device__ __forceinline__ void sub_rn(const Num<W>& a, const Num<W>& b, Num<W>& r) {
  Num<W> nb = b;
  nb.s ^= 1u;
  add_rn<W>(a, nb, r);
}

// floor((u1 2^32 + u0) / d) and its remainder for a normalised word d (top
// bit set) and u1 < d, from the reciprocal v = floor((2^64 - 1)/d) - 2^32
// computed once per divisor: the 2/1 division by an invariant integer of
// Moller and Granlund ("Improved division by invariant integers", IEEE
// Trans. Computers 60(2), 2011): one 32x32->64 multiply, a two-word add, one
// low multiply and at most two corrections, instead of a 64-bit division.
__device__ __forceinline__ uint32_t div2by1(uint32_t u1, uint32_t u0, uint32_t d, uint32_t v,
                                            uint32_t& rem) {
  const uint64_t q = (uint64_t)v * u1 + (((uint64_t)u1 << 32) | u0);  // < 2^64 as u1 < d
  uint32_t q1 = (uint32_t)(q >> 32) + 1u;
  const uint32_t q0 = (uint32_t)q;
  uint32_t r = u0 - q1 * d;
  if (r > q0) {
    q1 -= 1u;
    r += d;
  }
  if (r >= d) {
    q1 += 1u;
    r -= d;
  }
  rem = r;
  return q1;
}

// r = RN(a/b) for b != 0 (callers test b first).  Knuth's algorithm D in base
// 2^32 divides N = Ma * 2^(32(W+1)) by Mb (normalised: top bit set), giving a
// (W+2)-word quotient Q of 32W+32 or 32W+33 bits and a remainder R; the kept
// p bits, the next bit of Q and sticky = (rest of Q or R nonzero) round it.
// Each quotient word is estimated from the top two remainder words and Mb's
// top word by div2by1 (Mb's top word is the invariant divisor), then
// corrected with the next word as the algorithm prescribes.
template <int W>
__device__ __noinline__ void div_rn(const Num<W>& a, const Num<W>& b, Num<W>& r) {
  const uint32_t s = a.s ^ b.s;
  if (zero_e(a.e)) {
    set_zero(r, s);
    return;
  }
  uint32_t u[2 * W + 2];
#pragma unroll
  for (int k = 0; k <= W; ++k) u[k] = 0u;
#pragma unroll
  for (int k = 0; k < W; ++k) u[W + 1 + k] = a.m[k];
  u[2 * W + 1] = 0u;
  uint32_t q[W + 2];
  const uint64_t vt = b.m[W - 1], vt2 = b.m[W - 2];
  const uint32_t vinv = (uint32_t)(~uint64_t(0) / vt);  // floor((2^64-1)/vt) - 2^32
#pragma unroll
  for (int j = W + 1; j >= 0; --j) {
    // the remainder's top word never exceeds vt; when equal the estimate is
    // 2^32 - 1 with remainder u0 + vt (which may exceed a word)
    uint64_t qhat, rhat;
    if (u[j + W] >= (uint32_t)vt) {
      qhat = 0xffffffffu;
      rhat = (uint64_t)u[j + W - 1] + vt;
    } else {
      uint32_t rr;
      qhat = div2by1(u[j + W], u[j + W - 1], (uint32_t)vt, vinv, rr);
      rhat = rr;
    }
    const uint64_t u2 = (j + W - 2 >= 0) ? u[j + W - 2] : 0u;
    while ((rhat >> 32) == 0u && qhat * vt2 > ((rhat << 32) | u2)) {
      qhat -= 1u;
      rhat += vt;
    }
    uint64_t carry = 0u;
    uint32_t bw = 0u;
#pragma unroll
    for (int i = 0; i < W; ++i) {
      const uint64_t pr = qhat * b.m[i] + carry;
      carry = pr >> 32;
      const uint64_t t = (uint64_t)u[i + j] - (uint32_t)pr - bw;
      u[i + j] = (uint32_t)t;
      bw = (uint32_t)(t >> 63);
    }
    const uint64_t t = (uint64_t)u[j + W] - carry - bw;
    u[j + W] = (uint32_t)t;
    q[j] = (uint32_t)qhat;
    if ((t >> 63) != 0u) {  // qhat was one too large: add the divisor back
      q[j] -= 1u;
      uint32_t c = 0u;
#pragma unroll
      for (int i = 0; i < W; ++i) {
        const uint64_t s2 = (uint64_t)u[i + j] + b.m[i] + c;
        u[i + j] = (uint32_t)s2;
        c = (uint32_t)(s2 >> 32);
      }
      u[j + W] += c;
    }
  }
  uint32_t rem = 0u;
#pragma unroll
  for (int k = 0; k < W; ++k) rem |= u[k];
  const uint32_t top = q[W + 1] & 1u;  // Q has 32W+33 bits
  // keep bits [32+top, 32W+32+top) of Q
#pragma unroll
  for (int k = 0; k < W; ++k) r.m[k] = __funnelshift_r(q[k + 1], q[k + 2], top);
  const uint32_t g = top ? (q[1] << 31) | (q[0] >> 1) : q[0];
  const uint32_t rb = g >> 31;
  const uint32_t st = (g << 1) | (top ? (q[0] & 1u) : 0u) | rem;
  r.e = a.e - b.e + (int64_t)top;
  r.s = s;
  round_increment<W>(r.m, r.e, rb & ((st != 0u) | (r.m[0] & 1u)));
}

// -1, 0, 1 (zeros of either sign compare equal).
template <int W>
__device__ __forceinline__ int cmp(const Num<W>& a, const Num<W>& b) {
  const int sa = zero_e(a.e) ? 0 : (a.s ? -1 : 1);
  const int sb = zero_e(b.e) ? 0 : (b.s ? -1 : 1);
  if (sa != sb) return sa < sb ? -1 : 1;
  if (sa == 0) return 0;
  int mag = 0;
  if (a.e != b.e) {
    mag = a.e > b.e ? 1 : -1;
  } else {
#pragma unroll
    for (int k = W - 1; k >= 0; --k)
      mag = (mag != 0) ? mag : ((a.m[k] > b.m[k]) ? 1 : ((a.m[k] < b.m[k]) ? -1 : 0));
  }
  return sa > 0 ? mag : -mag;
}

// Exact conversion of an IEEE double (53 <= p).
template <int W>
__device__ __forceinline__ void from_f64(double d, Num<W>& r) {
  const uint64_t bits = (uint64_t)__double_as_longlong(d);
  const uint32_t s = (uint32_t)(bits >> 63);
  const int be = (int)((bits >> 52) & 0x7ffu);
  const uint64_t f = bits & ((uint64_t(1) << 52) - 1u);
  set_zero(r, s);
  if (be == 0 && f == 0u) return;
  uint64_t top;
  int64_t e;
  if (be == 0) {  // subnormal: f * 2^-1074
    const int lz = __clzll((long long)f);
    top = f << lz;
    e = (int64_t)(64 - lz) - 1074;
  } else {
    top = ((uint64_t(1) << 52) | f) << 11;
    e = (int64_t)be - 1022;
  }
  r.m[W - 1] = (uint32_t)(top >> 32);
  r.m[W - 2] = (uint32_t)top;
  r.e = e;
}

// Nearest double (for reporting; huge exponents saturate).
template <int W>
__device__ __forceinline__ double to_f64(const Num<W>& a) {
  if (zero_e(a.e)) return a.s ? -0.0 : 0.0;
  const uint64_t t = ((uint64_t)a.m[W - 1] << 32) | a.m[W - 2];
  uint32_t rest = 0u;
#pragma unroll
  for (int k = 0; k < W - 2; ++k) rest |= a.m[k];
  uint64_t q = t >> 11;
  const uint32_t rb = (uint32_t)(t >> 10) & 1u;
  const bool st = ((t & 0x3ffu) != 0u) || rest != 0u;
  if (rb && (st || (q & 1u))) q += 1u;
  const int64_t e = a.e < -4000 ? -4000 : (a.e > 4000 ? 4000 : a.e);
  const double v = ldexp((double)q, (int)e - 53);
  return a.s ? -v : v;
}

// ---------------------------------------------------------------------------
// Exact sums: 64-bit signed digit counters over 32-bit digits
// ---------------------------------------------------------------------------
// A term P * 2^(E - 2p) (P the exact 2W-word product) enters an accumulator
// whose digit 0 has weight 2^(Emin - 2p) as P * 2^(E - Emin): 2W+1 digits
// starting at digit (E - Emin) / 32 after a funnel shift by (E - Emin) % 32.
// Counters absorb signed 32-bit digits without carries; carries are resolved
// once, when the sum is rounded.

template <int W>
__device__ __forceinline__ void shifted_digits(const uint32_t (&P)[2 * W], uint32_t bs,
                                               uint32_t (&D)[2 * W + 1]) {
#pragma unroll
  for (int k = 0; k <= 2 * W; ++k) {
    const uint32_t lo = (k > 0) ? P[k - 1] : 0u;
    const uint32_t hi = (k < 2 * W) ? P[k] : 0u;
    D[k] = __funnelshift_l(lo, hi, bs);
  }
}

// Adds (-1)^neg * P * 2^off into counters c[d*stride].
template <int W>
__device__ __forceinline__ void add_term(int64_t* c, int stride, const uint32_t (&P)[2 * W],
                                         int64_t off, uint32_t neg) {
  uint32_t D[2 * W + 1];
  shifted_digits<W>(P, (uint32_t)(off & 31), D);
  int64_t* p = c + (off >> 5) * stride;
  // G digits at a time: loads together, then stores together (one
  // shared-memory latency per group instead of one per digit)
  constexpr int G = 2 * W + 1 < 12 ? 2 * W + 1 : 12;
#pragma unroll
  for (int k0 = 0; k0 <= 2 * W; k0 += G) {
    int64_t v[G];
#pragma unroll
    for (int u = 0; u < G; ++u)
      if (k0 + u <= 2 * W) v[u] = p[(k0 + u) * stride];
#pragma unroll
    for (int u = 0; u < G; ++u) {
      if (k0 + u <= 2 * W) {
        const int64_t d = (int64_t)D[k0 + u];
        p[(k0 + u) * stride] = v[u] + (neg ? -d : d);
      }
    }
  }
}

// Resolve carries of nd signed digit counters c[d*stride] into 32-bit words
// (stored back into the counters' slots), returning 1 when the total is
// negative.  The counters are then the two's complement words of the sum.
__device__ __forceinline__ uint32_t resolve_digits(int64_t* c, int stride, int nd) {
  int64_t carry = 0;
  for (int d = 0; d < nd; ++d) {
    const int64_t t = c[d * stride] + carry;
    c[d * stride] = (int64_t)(uint32_t)t;
    carry = t >> 32;
  }
  return carry < 0 ? 1u : 0u;
}

// Negate the nd two's complement words in place (magnitude of a negative sum).
__device__ __forceinline__ void negate_words(int64_t* c, int stride, int nd) {
  uint32_t carry = 1u;
  for (int d = 0; d < nd; ++d) {
    const uint64_t t = (uint64_t)(uint32_t)~(uint32_t)c[d * stride] + carry;
    c[d * stride] = (int64_t)(uint32_t)t;
    carry = (uint32_t)(t >> 32);
  }
}

// r = RN( (-1)^neg * S * 2^k ) for the natural S held in nd 32-bit words
// c[d*stride]; S == 0 gives +0.
template <int W>
__device__ __forceinline__ void round_words(const int64_t* c, int stride, int nd, int64_t k,
                                            uint32_t neg, Num<W>& r) {
  int t = nd - 1;
  while (t >= 0 && (uint32_t)c[t * stride] == 0u) --t;
  if (t < 0) {
    set_zero(r, 0u);
    return;
  }
  const int64_t nb = 32 * (int64_t)t + (32 - __clz((uint32_t)c[t * stride]));
  const int64_t pos = nb - 32 * W;  // lowest kept bit (negative: exact)
  auto word = [&](int64_t i) -> uint32_t {
    return (i >= 0 && i < nd) ? (uint32_t)c[i * stride] : 0u;
  };
  auto bits32 = [&](int64_t at) -> uint32_t {  // bits [at, at+32)
    const int64_t q = (at >= 0) ? at / 32 : -((-at + 31) / 32);
    const uint32_t sh = (uint32_t)(at - 32 * q);
    return __funnelshift_r(word(q), word(q + 1), sh);
  };
#pragma unroll
  for (int j = 0; j < W; ++j) r.m[j] = bits32(pos + 32 * j);
  uint32_t rb = 0u, st = 0u;
  if (pos > 0) {
    rb = (bits32(pos - 1) & 1u);
    const int64_t below = pos - 1;  // bits [0, below) form the sticky
    const int64_t fw = below / 32;
    for (int64_t i = 0; i < fw; ++i) st |= word(i);
    const uint32_t rem = (uint32_t)(below - 32 * fw);
    if (rem) st |= word(fw) << (32u - rem);
  }
  r.e = nb + k;
  r.s = neg;
  round_increment<W>(r.m, r.e, rb & ((st != 0u) | (r.m[0] & 1u)));
}

// ---------------------------------------------------------------------------
// Exact sums over radix-2^29 column sums (high precision)
// ---------------------------------------------------------------------------
// With the operands cut into 29-bit limbs, a 32x32-bit multiply-add of two
// limbs into a 64-bit column sum never overflows: a column of the product
// sums at most 37 limb products < 2^58 each.  So the exact product
// Ma * (Mx << s) is formed as column sums C_k = sum_{i+j=k} a_i x_j with one
// IMAD.WIDE per limb pair and no carry handling, and each C_k enters the
// counters split as (C_k mod 2^29) at digit k and (C_k >> 29) at digit k+1.
// Counter digit d has weight 2^(29 d); a term at bit offset off goes to digit
// off / 29 after shifting one operand left by off mod 29.

constexpr int kR = 29;
constexpr uint32_t kRMask = (1u << kR) - 1u;

template <int W>
struct Cols {
  static constexpr int NA = (32 * W + kR - 1) / kR;           // limbs of Ma
  static constexpr int NX = (32 * W + kR - 1 + kR - 1) / kR;  // limbs of Mx << s, s < 29
  static constexpr int NC = NA + NX - 1;                      // columns of the product
};

// l[i] = bits [29 i, 29 i + 29) of the NW-word number w.
template <int NW, int NL>
__device__ __forceinline__ void cut_limbs(const uint32_t (&w)[NW], uint32_t (&l)[NL]) {
#pragma unroll
  for (int i = 0; i < NL; ++i) {
    const int b = kR * i, q = b / 32, r = b % 32;
    const uint32_t lo = (q < NW) ? w[q] : 0u;
    const uint32_t hi = (q + 1 < NW) ? w[q + 1] : 0u;
    l[i] = (r + kR <= 32 ? (lo >> r) : __funnelshift_r(lo, hi, r)) & kRMask;
  }
}

// Limbs of M << s (0 <= s < 29).
template <int W, int NL>
__device__ __forceinline__ void cut_limbs_shifted(const uint32_t (&m)[W], uint32_t s,
                                                  uint32_t (&l)[NL]) {
  uint32_t t[W + 1];
  t[0] = m[0] << s;
#pragma unroll
  for (int k = 1; k < W; ++k) t[k] = __funnelshift_l(m[k - 1], m[k], s);
  t[W] = __funnelshift_l(m[W - 1], 0u, s);
  cut_limbs<W + 1, NL>(t, l);
}

// c[(q + k) * stride] += (-1)^neg * D_k for the digits D of the term
// Ma * Mx * 2^off, off = 29 q + s.
template <int W, int G = 8>
__device__ __forceinline__ void add_product_cols(int64_t* c, int stride, const uint32_t (&a)[W],
                                                 const uint32_t (&x)[W], uint32_t off,
                                                 uint32_t neg) {
  constexpr int NA = Cols<W>::NA, NX = Cols<W>::NX, NC = Cols<W>::NC;
  const uint32_t q = off / kR, s = off - kR * q;
  uint32_t al[NA], xl[NX];
  cut_limbs<W, NA>(a, al);
  cut_limbs_shifted<W, NX>(x, s, xl);
  const uint64_t m = neg ? ~0ull : 0ull;  // (d ^ m) - m = -d when neg
  int64_t* p = c + (int64_t)q * stride;
  uint64_t carry = 0u;
  // G columns at a time: their counters are loaded together, then updated
  // and stored together, so the shared-memory latency is paid once per group
#pragma unroll
  for (int k0 = 0; k0 <= NC; k0 += G) {
    uint64_t dd[G], acc[G];
    int64_t v[G];
    // the group's counters are read first (their latency overlaps the
    // multiply-adds), then the G columns' multiply-adds run interleaved: G
    // independent chains
#pragma unroll
    for (int u = 0; u < G; ++u)
      if (k0 + u <= NC) v[u] = p[(k0 + u) * stride];
#pragma unroll
    for (int u = 0; u < G; ++u) acc[u] = 0u;
#pragma unroll
    for (int i = 0; i < NA; ++i) {
#pragma unroll
      for (int u = 0; u < G; ++u) {
        const int j = k0 + u - i;
        if (k0 + u < NC && j >= 0 && j < NX) acc[u] += (uint64_t)al[i] * xl[j];
      }
    }
#pragma unroll
    for (int u = 0; u < G; ++u) {
      const int k = k0 + u;
      if (k < NC) {
        dd[u] = (uint64_t)((uint32_t)acc[u] & kRMask) + carry;
        carry = acc[u] >> kR;
      } else if (k == NC) {
        dd[u] = carry;
      }
    }
#pragma unroll
    for (int u = 0; u < G; ++u)
      if (k0 + u <= NC) p[(k0 + u) * stride] = v[u] + (int64_t)((dd[u] ^ m) - m);
  }
}

// r = RN(a*b) as mul_rn, with the exact product formed from radix-2^29
// column sums: NA^2 multiply-adds into 64-bit columns, one carry pass over
// the 2 NA digits, then the top W+1 words are reassembled from the digits and
// everything below them only feeds the sticky bit.
template <int W>
__device__ __forceinline__ void mul_rn_cols(const Num<W>& a, const Num<W>& b, Num<W>& r) {
  constexpr int NA = Cols<W>::NA;
  constexpr int ND = 2 * NA;                // digits of the product
  constexpr int WLO = W - 1;                // lowest product word kept (then up to 2W-1)
  constexpr int KLO = (32 * WLO) / kR;      // first digit reaching word WLO
  constexpr int R0 = 32 * WLO - kR * KLO;   // bits of digit KLO below word WLO
  const uint32_t s = a.s ^ b.s;
  if (zero_e(a.e) || zero_e(b.e)) {
    set_zero(r, s);
    return;
  }
  uint32_t al[NA], bl[NA];
  cut_limbs<W, NA>(a.m, al);
  cut_limbs<W, NA>(b.m, bl);
  uint32_t D[ND - KLO];
  uint32_t st = 0u;
  uint64_t carry = 0u;
#pragma unroll
  for (int k = 0; k < ND - 1; ++k) {
    uint64_t acc = carry;
#pragma unroll
    for (int i = (k - NA + 1 > 0 ? k - NA + 1 : 0); i <= (k < NA - 1 ? k : NA - 1); ++i)
      acc += (uint64_t)al[i] * bl[k - i];
    const uint32_t d = (uint32_t)acc & kRMask;
    carry = acc >> kR;
    if (k < KLO)
      st |= d;
    else
      D[k - KLO] = d;
  }
  D[ND - 1 - KLO] = (uint32_t)carry;
  if (R0 > 0) st |= D[0] & ((1u << R0) - 1u);
  // P[WLO + j] for j = 0..W: bits [32 (WLO + j), +32) of the product
  uint32_t T[W + 1];
#pragma unroll
  for (int j = 0; j <= W; ++j) {
    const int bit = 32 * (WLO + j), kk = bit / kR - KLO, rr = bit % kR;
    uint32_t v = D[kk] >> rr;
    if (kk + 1 < ND - KLO) v |= D[kk + 1] << (kR - rr);
    if (2 * kR - rr < 32 && kk + 2 < ND - KLO) v |= D[kk + 2] << (2 * kR - rr);
    T[j] = v;
  }
  const uint32_t sh = 1u - (T[W] >> 31);  // 1 when the product has 2p-1 bits
#pragma unroll
  for (int k = 0; k < W; ++k) r.m[k] = __funnelshift_l(T[k], T[k + 1], sh);
  const uint32_t g = T[0] << sh;
  st |= g << 1;
  r.e = a.e + b.e - (int64_t)sh;
  r.s = s;
  round_increment<W>(r.m, r.e, (g >> 31) & ((st != 0u) | (r.m[0] & 1u)));
}

// The column product's rare exact path, out of line (keeps the hot loop small).
template <int W>
__device__ __noinline__ void mul_rn_cols_full(const Num<W>& a, const Num<W>& b, Num<W>& r) {
  mul_rn_cols<W>(a, b, r);
}

// r = RN(a*b) from the upper columns only (a short product): columns below
// K0 are skipped, so the computed digits T miss a part delta < 2^(29 K0 + 63)
// of the exact product P = T + delta.  The bits of T from digit KG = K0 + 3
// up to the round bit (a guard region of >= 36 bits) decide the rounding
// unless they are all ones (delta could carry into the round bit) or all
// zeros with the round bit set (the sticky bit is then unknown); those rare
// cases take the full product.  Saves 28 % (p = 512) and 38 % (p = 1024) of
// the multiply-adds.
template <int W>
__device__ __forceinline__ void mul_rn_short(const Num<W>& a, const Num<W>& b, Num<W>& r) {
  constexpr int NA = Cols<W>::NA;
  constexpr int ND = 2 * NA;
  constexpr int WLO = W - 1;
  constexpr int KLO = (32 * WLO) / kR;
  constexpr int R0 = 32 * WLO - kR * KLO;
  constexpr int K0A = (32 * W - 97) / kR;
  constexpr int K0 = K0A < KLO - 3 ? K0A : KLO - 3;
  constexpr int KG = K0 + 3;
  static_assert(K0 > 0 && KG <= KLO, "short product needs p >= 512");
  const uint32_t s = a.s ^ b.s;
  if (zero_e(a.e) || zero_e(b.e)) {
    set_zero(r, s);
    return;
  }
  uint32_t al[NA], bl[NA];
  cut_limbs<W, NA>(a.m, al);
  cut_limbs<W, NA>(b.m, bl);
  uint32_t D[ND - KG];  // digits KG .. ND-1
  uint64_t carry = 0u;
#pragma unroll
  for (int k = K0; k < ND - 1; ++k) {
    uint64_t acc = carry;
#pragma unroll
    for (int i = (k - NA + 1 > 0 ? k - NA + 1 : 0); i <= (k < NA - 1 ? k : NA - 1); ++i)
      acc += (uint64_t)al[i] * bl[k - i];
    carry = acc >> kR;
    if (k >= KG) D[k - KG] = (uint32_t)acc & kRMask;
  }
  D[ND - 1 - KG] = (uint32_t)carry;
  uint32_t T[W + 1];
#pragma unroll
  for (int j = 0; j <= W; ++j) {
    const int bit = 32 * (WLO + j), kk = bit / kR - KG, rr = bit % kR;
    uint32_t v = D[kk] >> rr;
    if (kk + 1 < ND - KG) v |= D[kk + 1] << (kR - rr);
    if (2 * kR - rr < 32 && kk + 2 < ND - KG) v |= D[kk + 2] << (2 * kR - rr);
    T[j] = v;
  }
  const uint32_t sh = 1u - (T[W] >> 31);
  const uint32_t g = T[0] << sh;
  const uint32_t rb = g >> 31;
  const uint32_t below = g << 1;  // 31 - sh bits under the round bit, then zeros
  // guard region: digits KG .. KLO-1, the low R0 bits of digit KLO, `below`
  uint32_t any = below, all = below | ((1u << (1 + sh)) - 1u);
#pragma unroll
  for (int k = KG; k < KLO; ++k) {
    any |= D[k - KG];
    all &= D[k - KG] | ~kRMask;
  }
  if (R0 > 0) {
    const uint32_t lowm = (1u << R0) - 1u;
    any |= D[KLO - KG] & lowm;
    all &= D[KLO - KG] | ~lowm;
  }
  if (all == 0xffffffffu || (rb != 0u && any == 0u)) {
    mul_rn_cols_full<W>(a, b, r);
    return;
  }
#pragma unroll
  for (int k = 0; k < W; ++k) r.m[k] = __funnelshift_l(T[k], T[k + 1], sh);
  r.e = a.e + b.e - (int64_t)sh;
  r.s = s;
  round_increment<W>(r.m, r.e, rb & ((any != 0u) | (r.m[0] & 1u)));
}

// r = RN(a*b) in the cheaper form for the precision: the short column
// product from p = 512, the word product below.  Both are correctly
// rounded, so the result is the same.
template <int W>
__device__ __forceinline__ void mul_rn_fast(const Num<W>& a, const Num<W>& b, Num<W>& r) {
  if constexpr (W >= 16)
    mul_rn_short<W>(a, b, r);
  else
    mul_rn<W>(a, b, r);
}

// As add_product_cols for a window of counters that starts qrel digits above
// the term's own digit 0 (qrel = q - window base, may be negative): columns
// below the window (k < -qrel) are skipped, and errp is set when a skipped
// column may be nonzero (it is zero when k < la + lx, the indices of the two
// operands' lowest nonzero limbs).
template <int W, int G = 8>
__device__ __forceinline__ void add_product_cols_top(int64_t* c, int stride, const uint32_t (&a)[W],
                                                     const uint32_t (&x)[W], int qrel, uint32_t s,
                                                     uint32_t neg, bool& errp) {
  constexpr int NA = Cols<W>::NA, NX = Cols<W>::NX, NC = Cols<W>::NC;
  const int kmin = qrel < 0 ? -qrel : 0;
  if (kmin > NC) {  // the whole term lies below the window
    errp = true;
    return;
  }
  uint32_t al[NA], xl[NX];
  cut_limbs<W, NA>(a, al);
  cut_limbs_shifted<W, NX>(x, s, xl);
  if (kmin > 0 && !errp) {  // once a skipped column may be nonzero, the row is checked anyway
    int la = NA, lx = NX;
#pragma unroll
    for (int i = NA - 1; i >= 0; --i) la = al[i] ? i : la;
#pragma unroll
    for (int j = NX - 1; j >= 0; --j) lx = xl[j] ? j : lx;
    errp = errp || kmin > la + lx;
  }
  const uint64_t m = neg ? ~0ull : 0ull;
  int64_t* p = c + (int64_t)qrel * stride;
  uint64_t carry = 0u;
#pragma unroll
  for (int k0 = 0; k0 <= NC; k0 += G) {
    if (k0 + G <= kmin) continue;  // the group lies below the window
    uint64_t dd[G], acc[G];
    int64_t v[G];
#pragma unroll
    for (int u = 0; u < G; ++u)
      if (k0 + u <= NC && k0 + u >= kmin) v[u] = p[(k0 + u) * stride];
#pragma unroll
    for (int u = 0; u < G; ++u) acc[u] = 0u;
#pragma unroll
    for (int i = 0; i < NA; ++i) {
#pragma unroll
      for (int u = 0; u < G; ++u) {
        const int j = k0 + u - i;
        if (k0 + u < NC && j >= 0 && j < NX && k0 + u >= kmin) acc[u] += (uint64_t)al[i] * xl[j];
      }
    }
#pragma unroll
    for (int u = 0; u < G; ++u) {
      const int k = k0 + u;
      if (k < NC) {
        dd[u] = (uint64_t)((uint32_t)acc[u] & kRMask) + carry;
        carry = acc[u] >> kR;  // 0 below the window: that column's high part is skipped too
      } else if (k == NC) {
        dd[u] = carry;
      }
    }
#pragma unroll
    for (int u = 0; u < G; ++u)
      if (k0 + u <= NC && k0 + u >= kmin) p[(k0 + u) * stride] = v[u] + (int64_t)((dd[u] ^ m) - m);
  }
}

// Whether the bits [lo, hi) of the nw-word magnitude c[.*stride] decide a
// rounding that an error of magnitude below 2^lo cannot change: they must be
// neither all zeros nor all ones, and at least 8 of them.
__device__ __forceinline__ bool guard_bits_decide(const int64_t* c, int stride, int nw, int64_t lo,
                                                  int64_t hi) {
  if (hi - lo < 8) return false;
  uint32_t any = 0u, all = 0xffffffffu;
  for (int64_t w = lo >> 5; w <= (hi - 1) >> 5 && w < nw; ++w) {
    const int64_t b0 = w << 5;
    const uint32_t from = lo > b0 ? (uint32_t)(lo - b0) : 0u;
    const uint32_t to = hi < b0 + 32 ? (uint32_t)(hi - b0) : 32u;  // bits [from, to)
    const uint32_t mask = (to == 32u ? 0xffffffffu : ((1u << to) - 1u)) & ~((1u << from) - 1u);
    const uint32_t word = (uint32_t)c[w * stride];
    any |= word & mask;
    all &= word | ~mask;
  }
  return any != 0u && all != 0xffffffffu;
}

// c[(q + j) * stride] += (-1)^neg * limb_j(M << s) for the value M * 2^off.
template <int W>
__device__ __forceinline__ void add_value_cols(int64_t* c, int stride, const uint32_t (&mv)[W],
                                               uint32_t off, uint32_t neg) {
  constexpr int NX = Cols<W>::NX;
  const uint32_t q = off / kR, s = off - kR * q;
  uint32_t xl[NX];
  cut_limbs_shifted<W, NX>(mv, s, xl);
  int64_t* p = c + (int64_t)q * stride;
#pragma unroll
  for (int j = 0; j < NX; ++j) p[j * stride] += neg ? -(int64_t)xl[j] : (int64_t)xl[j];
}

// Resolves nd signed radix-2^29 counters into the magnitude of their total as
// 32-bit words stored back in c[0 .. *nw) (slot stride `stride`); returns 1
// when the total is negative.
__device__ __forceinline__ uint32_t resolve_cols(int64_t* c, int stride, int nd, int* nw) {
  int64_t carry = 0;
  for (int d = 0; d < nd; ++d) {
    const int64_t t = c[d * stride] + carry;
    c[d * stride] = t & kRMask;
    carry = t >> kR;
  }
  const uint32_t negative = carry < 0 ? 1u : 0u;
  if (negative) {  // -total = sum of (-digit) 2^(29 d) + 2^(29 nd)
    carry = 0;
    for (int d = 0; d < nd; ++d) {
      const int64_t t = carry - c[d * stride];
      c[d * stride] = t & kRMask;
      carry = t >> kR;
    }
  }
  // repack 29-bit digits into 32-bit words in place (word w <= digit d)
  uint64_t buf = 0u;
  int nb = 0, w = 0;
  for (int d = 0; d < nd; ++d) {
    buf |= (uint64_t)c[d * stride] << nb;
    nb += kR;
    if (nb >= 32) {
      c[w * stride] = (int64_t)(uint32_t)buf;
      ++w;
      buf >>= 32;
      nb -= 32;
    }
  }
  if (nb > 0) c[(w++) * stride] = (int64_t)(uint32_t)buf;
  *nw = w;
  return negative;
}

}  // namespace mpk
