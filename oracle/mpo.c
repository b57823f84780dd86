/* mpo.c -- CPU oracle for p-bit CSR SpMV, exact dot products, BiCG, GPBiCG,
 * CGS, BiCGSTAB, ILU(0) and BiCGSTAB preconditioned with ILU(0).
 *
 * TEST INFRASTRUCTURE ONLY (see mpo.h).  Deliberately plain and slow: natural
 * numbers are little-endian arrays of 32-bit words handled by schoolbook
 * loops, every result goes through the single rounding routine round_nat(),
 * and the solvers take the steps of the paper's Fig. 5 in the paper's order.
 *
 * Parity of every function here is pinned by the tests under tests/ against
 * exact rational arithmetic (Python fractions), an independent correctly
 * rounded library (mpmath, where installed) and mathematical properties
 * (closed forms, invariants, known solutions).
 */
#include "mpo.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

/* 32-bit words of the largest mantissa this build holds: 32 (p <= 1024) by
 * default, 256 (p <= 8192) in the wide build (-DWMAX=256). */
#ifndef WMAX
#define WMAX 32
#endif

typedef struct {
  int neg;  /* 1 = negative */
  int zero; /* 1 = the value is a (signed) zero */
  int64_t e;
  uint32_t m[WMAX]; /* p/32 words, little-endian; top bit set when nonzero */
} num;

static void die(const char *msg) {
  fprintf(stderr, "mpo oracle: %s\n", msg);
  abort();
}

static int prec_ok(int p) {
  return (p == 128 || p == 256 || p == 512 || p == 1024 || p == 2048 || p == 4096 || p == 8192) &&
         p / 32 <= WMAX;
}

/* ------------------------------------------------------------------------ */
/* Natural numbers: little-endian 32-bit words                              */
/* ------------------------------------------------------------------------ */

static int64_t nat_bitlen(const uint32_t *s, int64_t nw) {
  for (int64_t i = nw - 1; i >= 0; i--) {
    if (s[i]) {
      int64_t b = 32;
      uint32_t w = s[i];
      while (!(w & 0x80000000u)) {
        w <<= 1;
        b--;
      }
      return 32 * i + b;
    }
  }
  return 0;
}

static uint32_t nat_word(const uint32_t *s, int64_t nw, int64_t i) {
  return (i >= 0 && i < nw) ? s[i] : 0u;
}

static int64_t floor_div32(int64_t a) { return (a >= 0) ? a / 32 : -((-a + 31) / 32); }

/* Bits [pos, pos+32) of s; bits at negative indices are zero. */
static uint32_t nat_bits32(const uint32_t *s, int64_t nw, int64_t pos) {
  int64_t q = floor_div32(pos);
  int r = (int)(pos - 32 * q);
  uint64_t lo = nat_word(s, nw, q), hi = nat_word(s, nw, q + 1);
  return (uint32_t)((((hi << 32) | lo) >> r) & 0xffffffffu);
}

/* 1 if any bit of s with index < pos is set. */
static int nat_any_below(const uint32_t *s, int64_t nw, int64_t pos) {
  for (int64_t i = 0; i < pos; i++) {
    if (i % 32 == 0 && pos - i >= 32) {
      if (nat_word(s, nw, i / 32)) return 1;
      i += 31;
      continue;
    }
    if ((nat_word(s, nw, i / 32) >> (i % 32)) & 1u) return 1;
  }
  return 0;
}

static int nat_is_zero(const uint32_t *s, int64_t nw) {
  for (int64_t i = 0; i < nw; i++)
    if (s[i]) return 0;
  return 1;
}

/* r[0 .. na+nb) = a * b, schoolbook. */
static void nat_mul(uint32_t *r, const uint32_t *a, int64_t na, const uint32_t *b,
                    int64_t nb) {
  memset(r, 0, sizeof(uint32_t) * (size_t)(na + nb));
  for (int64_t i = 0; i < na; i++) {
    uint64_t carry = 0;
    for (int64_t j = 0; j < nb; j++) {
      uint64_t t = (uint64_t)a[i] * b[j] + r[i + j] + carry;
      r[i + j] = (uint32_t)t;
      carry = t >> 32;
    }
    r[i + nb] = (uint32_t)carry;
  }
}

/* acc += x * 2^sh (acc has nacc words; the sum must fit). */
static void nat_add_shifted(uint32_t *acc, int64_t nacc, const uint32_t *x, int64_t nx,
                            int64_t sh) {
  int64_t top = (sh + 32 * nx) / 32 + 1; /* last word x<<sh can reach */
  uint64_t carry = 0;
  for (int64_t i = sh / 32; i < nacc; i++) {
    uint64_t w = (i <= top) ? nat_bits32(x, nx, 32 * i - sh) : 0u;
    if (i > top && carry == 0) break;
    uint64_t t = (uint64_t)acc[i] + w + carry;
    acc[i] = (uint32_t)t;
    carry = t >> 32;
  }
  if (carry) die("accumulator overflow");
}

static int nat_cmp(const uint32_t *a, const uint32_t *b, int64_t n) {
  for (int64_t i = n - 1; i >= 0; i--) {
    if (a[i] != b[i]) return a[i] > b[i] ? 1 : -1;
  }
  return 0;
}

/* a -= b (a >= b), both n words. */
static void nat_sub(uint32_t *a, const uint32_t *b, int64_t n) {
  int64_t borrow = 0;
  for (int64_t i = 0; i < n; i++) {
    int64_t t = (int64_t)a[i] - (int64_t)b[i] - borrow;
    borrow = t < 0;
    a[i] = (uint32_t)(t + (borrow ? (INT64_C(1) << 32) : 0));
  }
  if (borrow) die("negative difference");
}

/* ------------------------------------------------------------------------ */
/* Rounding: the one place where precision is lost                          */
/* ------------------------------------------------------------------------ */

static void set_zero(num *r, int neg) {
  memset(r, 0, sizeof(*r));
  r->zero = 1;
  r->neg = neg;
  r->e = MPO_EXP_ZERO;
}

/* r = RN_p( (-1)^neg * S * 2^k ) for a natural S > 0: keep the top p bits,
 * round up when the first dropped bit is 1 and either a later dropped bit is
 * 1 or the kept part is odd (ties to even); a carry out of the top renormalises
 * to 2^(p-1) with the exponent raised by one.  The value S*2^k lies in
 * [2^(nb+k-1), 2^(nb+k)), so its exponent in the 0.1xxx convention is nb+k. */
static void round_nat(const uint32_t *S, int64_t nw, int64_t k, int p, int neg, num *r) {
  int W = p / 32;
  int64_t nb = nat_bitlen(S, nw);
  if (nb == 0) die("round_nat of zero");
  int64_t sh = nb - p; /* dropped bits; negative means an exact left shift */
  memset(r, 0, sizeof(*r));
  for (int i = 0; i < W; i++) r->m[i] = nat_bits32(S, nw, sh + 32 * (int64_t)i);
  int64_t e = nb + k;
  if (sh > 0) {
    int rbit = (int)(nat_bits32(S, nw, sh - 1) & 1u);
    int sticky = nat_any_below(S, nw, sh - 1);
    if (rbit && (sticky || (r->m[0] & 1u))) {
      int i = 0;
      while (i < W && ++r->m[i] == 0) i++;
      if (i == W) { /* M was 2^p - 1 and became 2^p */
        r->m[W - 1] = 0x80000000u;
        e += 1;
      }
    }
  }
  if (e >= MPO_EXP_LIMIT || e <= -MPO_EXP_LIMIT) die("exponent out of range");
  r->e = e;
  r->neg = neg;
  r->zero = 0;
}

/* ------------------------------------------------------------------------ */
/* Records                                                                  */
/* ------------------------------------------------------------------------ */

static int rec_load(const uint64_t *rec, int p, num *a) {
  int L = p / 64, W = p / 32;
  int64_t head = (int64_t)rec[0];
  memset(a, 0, sizeof(*a));
  a->neg = (int)(head & 1);
  int64_t e = (head - a->neg) / 2;
  for (int k = 0; k < L; k++) {
    a->m[2 * k] = (uint32_t)(rec[1 + k] & 0xffffffffu);
    a->m[2 * k + 1] = (uint32_t)(rec[1 + k] >> 32);
  }
  if (e == MPO_EXP_ZERO) {
    a->zero = 1;
    a->e = e;
    return nat_is_zero(a->m, W) ? MPO_OK : MPO_ERR_ARG;
  }
  a->e = e;
  if (!(a->m[W - 1] & 0x80000000u)) return MPO_ERR_ARG;
  if (e >= MPO_EXP_LIMIT || e <= -MPO_EXP_LIMIT) return MPO_ERR_ARG;
  return MPO_OK;
}

static void rec_store(const num *a, int p, uint64_t *rec) {
  int L = p / 64;
  int64_t e = a->zero ? MPO_EXP_ZERO : a->e;
  rec[0] = (uint64_t)(e * 2 + a->neg);
  for (int k = 0; k < L; k++)
    rec[1 + k] = (uint64_t)a->m[2 * k] | ((uint64_t)a->m[2 * k + 1] << 32);
}

/* Load record i of a vector, aborting on a malformed record (inputs are
 * validated by the public entry points before the arithmetic starts). */
static void vload(const uint64_t *v, int64_t i, int p, num *a) {
  if (rec_load(v + (size_t)i * (size_t)(p / 64 + 1), p, a) != MPO_OK)
    die("malformed record");
}
static void vstore(uint64_t *v, int64_t i, int p, const num *a) {
  rec_store(a, p, v + (size_t)i * (size_t)(p / 64 + 1));
}

static int vcheck(const uint64_t *v, int64_t n, int p) {
  num a;
  for (int64_t i = 0; i < n; i++)
    if (rec_load(v + (size_t)i * (size_t)(p / 64 + 1), p, &a) != MPO_OK) return MPO_ERR_ARG;
  return MPO_OK;
}

/* ------------------------------------------------------------------------ */
/* Correctly rounded operations                                             */
/* ------------------------------------------------------------------------ */

/* r = RN(a*b).  a = Ma 2^(ea-p), b = Mb 2^(eb-p), so a*b = (Ma Mb) 2^(ea+eb-2p).
 * A zero factor gives a zero whose sign is the xor of the signs. */
static void num_mul(const num *a, const num *b, int p, num *r) {
  if (a->zero || b->zero) {
    set_zero(r, a->neg ^ b->neg);
    return;
  }
  int W = p / 32;
  uint32_t prod[2 * WMAX];
  nat_mul(prod, a->m, W, b->m, W);
  round_nat(prod, 2 * W, a->e + b->e - 2 * (int64_t)p, p, a->neg ^ b->neg, r);
}

/* r = RN(a+b) with IEEE/MPFR signed-zero rules: (+0)+(-0) = +0,
 * (-0)+(-0) = -0, x+(+-0) = x, and an exact cancellation gives +0. */
static void num_add(const num *a, const num *b, int p, num *r) {
  if (a->zero && b->zero) {
    set_zero(r, a->neg & b->neg);
    return;
  }
  if (a->zero) {
    *r = *b;
    return;
  }
  if (b->zero) {
    *r = *a;
    return;
  }
  const num *big = a, *sml = b;
  if (b->e > a->e) {
    big = b;
    sml = a;
  }
  int64_t d = big->e - sml->e;
  if (d >= (int64_t)p + 2) {
    /* |sml| < 2^(sml.e) <= 2^(big.e-p-2) = ulp(big)/4.  Adding it moves big by
     * less than a quarter ulp; below big the spacing is at least ulp(big)/2
     * (half when big is a power of two), so the exact sum rounds to big. */
    *r = *big;
    return;
  }
  int W = p / 32;
  /* Exact sum on the grid 2^(sml.e - p): X = Mbig 2^d, Y = Msml. */
  enum { NX = 3 * WMAX + 4 };
  uint32_t X[NX], Y[NX];
  memset(X, 0, sizeof X);
  memset(Y, 0, sizeof Y);
  nat_add_shifted(X, NX, big->m, W, d);
  memcpy(Y, sml->m, sizeof(uint32_t) * (size_t)W);
  int neg;
  if (big->neg == sml->neg) {
    nat_add_shifted(X, NX, Y, NX, 0);
    neg = big->neg;
  } else {
    int c = nat_cmp(X, Y, NX);
    if (c == 0) {
      set_zero(r, 0);
      return;
    }
    if (c > 0) {
      nat_sub(X, Y, NX);
      neg = big->neg;
    } else {
      nat_sub(Y, X, NX);
      memcpy(X, Y, sizeof X);
      neg = sml->neg;
    }
  }
  round_nat(X, NX, sml->e - (int64_t)p, p, neg, r);
}

static void num_neg(const num *a, num *r) {
  *r = *a;
  r->neg ^= 1;
}

static void num_sub(const num *a, const num *b, int p, num *r) {
  num nb;
  num_neg(b, &nb);
  num_add(a, &nb, p, r);
}

/* r = RN(a/b).  a/b = (N/Mb) 2^(ea-eb-p-2) with N = Ma 2^(p+2).  Binary long
 * division gives Q = floor(N/Mb) and R; Q has at least p+2 bits, so rounding
 * S = 2Q + [R != 0] at scale 2^(ea-eb-p-3) sees the exact round bit and an
 * exact sticky bit, and equals rounding the exact quotient. */
static int num_div(const num *a, const num *b, int p, num *r) {
  if (b->zero) return MPO_ERR_DIVZERO;
  if (a->zero) {
    set_zero(r, a->neg ^ b->neg);
    return MPO_OK;
  }
  int W = p / 32;
  enum { NN = 2 * WMAX + 4 };
  uint32_t N[NN], Q[NN], R[NN], D[NN];
  memset(N, 0, sizeof N);
  memset(Q, 0, sizeof Q);
  memset(R, 0, sizeof R);
  memset(D, 0, sizeof D);
  nat_add_shifted(N, NN, a->m, W, (int64_t)p + 2);
  memcpy(D, b->m, sizeof(uint32_t) * (size_t)W);
  int64_t nb = nat_bitlen(N, NN);
  for (int64_t i = nb - 1; i >= 0; i--) {
    /* R = 2R + bit i of N */
    uint32_t in = (N[i / 32] >> (i % 32)) & 1u;
    for (int64_t j = NN - 1; j > 0; j--) R[j] = (R[j] << 1) | (R[j - 1] >> 31);
    R[0] = (R[0] << 1) | in;
    if (nat_cmp(R, D, NN) >= 0) {
      nat_sub(R, D, NN);
      Q[i / 32] |= 1u << (i % 32);
    }
  }
  uint32_t S[NN];
  memset(S, 0, sizeof S);
  nat_add_shifted(S, NN, Q, NN - 1, 1);
  if (!nat_is_zero(R, NN)) S[0] |= 1u;
  round_nat(S, NN, a->e - b->e - (int64_t)p - 3, p, a->neg ^ b->neg, r);
  return MPO_OK;
}

/* -1, 0, 1; zeros of either sign compare equal. */
static int num_cmp(const num *a, const num *b, int p) {
  int sa = a->zero ? 0 : (a->neg ? -1 : 1);
  int sb = b->zero ? 0 : (b->neg ? -1 : 1);
  if (sa != sb) return sa < sb ? -1 : 1;
  if (sa == 0) return 0;
  int mag;
  if (a->e != b->e)
    mag = a->e > b->e ? 1 : -1;
  else
    mag = nat_cmp(a->m, b->m, p / 32);
  return sa > 0 ? mag : -mag;
}

static int num_from_f64(double d, int p, num *r) {
  if (isnan(d) || isinf(d)) return MPO_ERR_ARG;
  if (d == 0.0) {
    set_zero(r, signbit(d) ? 1 : 0);
    return MPO_OK;
  }
  int ex;
  double f = frexp(fabs(d), &ex);          /* f in [1/2, 1) */
  uint64_t m53 = (uint64_t)ldexp(f, 53);   /* exact integer in [2^52, 2^53) */
  memset(r, 0, sizeof(*r));
  uint32_t w[2] = {(uint32_t)(m53 & 0xffffffffu), (uint32_t)(m53 >> 32)};
  /* M = m53 * 2^(p-53): value M 2^(ex-p) = m53 2^(ex-53) = d */
  for (int i = 0; i < p / 32; i++) r->m[i] = nat_bits32(w, 2, 32 * (int64_t)i - (p - 53));
  r->e = ex;
  r->neg = d < 0;
  r->zero = 0;
  return MPO_OK;
}

static double num_to_f64(const num *a, int p) {
  if (a->zero) return a->neg ? -0.0 : 0.0;
  int W = p / 32;
  uint64_t t = ((uint64_t)a->m[W - 1] << 32) | a->m[W - 2];
  int sticky = !nat_is_zero(a->m, W - 2);
  uint64_t q = t >> 11;
  int rbit = (int)((t >> 10) & 1u);
  int st = ((t & 0x3ffu) != 0) || sticky;
  if (rbit && (st || (q & 1u))) q++;
  double v = ldexp((double)q, (int)((a->e > 4000) ? 4000 : (a->e < -4000 ? -4000 : a->e)) - 53);
  return a->neg ? -v : v;
}

/* ------------------------------------------------------------------------ */
/* Exact sums of products (EXACT SpMV rows, dot products, residuals)         */
/* ------------------------------------------------------------------------ */

/* A term is P * 2^(E - 2p) with P a natural of 2W words: the exact product
 * Ma*Mb (E = ea + eb), or a single value b as Mb 2^p (E = eb). */
typedef struct {
  uint32_t P[2 * WMAX];
  int64_t E;
  int neg;
} term;

typedef struct {
  int p;
  int64_t m; /* terms added */
  int64_t emin, emax;
  term *t;
  int64_t cap;
} termlist;

static void tl_init(termlist *tl, int p) {
  memset(tl, 0, sizeof(*tl));
  tl->p = p;
}
static void tl_free(termlist *tl) { free(tl->t); }
static term *tl_push(termlist *tl) {
  if (tl->m == tl->cap) {
    tl->cap = tl->cap ? 2 * tl->cap : 64;
    tl->t = (term *)realloc(tl->t, sizeof(term) * (size_t)tl->cap);
    if (!tl->t) die("out of memory");
  }
  return &tl->t[tl->m++];
}

/* Add the exact product a*b (skipped when either factor is zero). */
static void tl_add_product(termlist *tl, const num *a, const num *b, int negate) {
  if (a->zero || b->zero) return;
  int W = tl->p / 32;
  term *t = tl_push(tl);
  memset(t->P, 0, sizeof t->P);
  nat_mul(t->P, a->m, W, b->m, W);
  t->E = a->e + b->e;
  t->neg = a->neg ^ b->neg ^ negate;
}

/* Add the single value a (skipped when zero). */
static void tl_add_value(termlist *tl, const num *a, int negate) {
  if (a->zero) return;
  int W = tl->p / 32;
  term *t = tl_push(tl);
  memset(t->P, 0, sizeof t->P);
  for (int i = 0; i < W; i++) t->P[W + i] = a->m[i];
  t->E = a->e;
  t->neg = a->neg ^ negate;
}

/* r = RN(sum of terms), computed exactly.  No terms -> +0, exact zero -> +0.
 * Returns MPO_ERR_SPAN (and r = +0) when max E - min E exceeds the cap. */
static int tl_sum(termlist *tl, num *r) {
  int p = tl->p, W = p / 32;
  if (tl->m == 0) {
    set_zero(r, 0);
    return MPO_OK;
  }
  int64_t emin = tl->t[0].E, emax = tl->t[0].E;
  for (int64_t i = 1; i < tl->m; i++) {
    if (tl->t[i].E < emin) emin = tl->t[i].E;
    if (tl->t[i].E > emax) emax = tl->t[i].E;
  }
  if (emax - emin > MPO_SPAN_CAP) {
    set_zero(r, 0);
    return MPO_ERR_SPAN;
  }
  int64_t nbits = (emax - emin) + 2 * (int64_t)p + 64 + 64;
  int64_t nw = nbits / 32 + 2;
  uint32_t *Pos = (uint32_t *)calloc((size_t)nw, sizeof(uint32_t));
  uint32_t *Neg = (uint32_t *)calloc((size_t)nw, sizeof(uint32_t));
  if (!Pos || !Neg) die("out of memory");
  for (int64_t i = 0; i < tl->m; i++) {
    const term *t = &tl->t[i];
    nat_add_shifted(t->neg ? Neg : Pos, nw, t->P, 2 * W, t->E - emin);
  }
  int c = nat_cmp(Pos, Neg, nw);
  if (c == 0) {
    set_zero(r, 0);
  } else if (c > 0) {
    nat_sub(Pos, Neg, nw);
    round_nat(Pos, nw, emin - 2 * (int64_t)p, p, 0, r);
  } else {
    nat_sub(Neg, Pos, nw);
    round_nat(Neg, nw, emin - 2 * (int64_t)p, p, 1, r);
  }
  free(Pos);
  free(Neg);
  return MPO_OK;
}

/* ------------------------------------------------------------------------ */
/* Public entry points: elementwise                                         */
/* ------------------------------------------------------------------------ */

int mpo_ewise(int p, int op, int64_t n, const uint64_t *a, const uint64_t *b,
              uint64_t *r) {
  if (!prec_ok(p)) return MPO_ERR_PREC;
  if (n < 0 || vcheck(a, n, p) || vcheck(b, n, p)) return MPO_ERR_ARG;
  int st = MPO_OK;
  for (int64_t i = 0; i < n; i++) {
    num x, y, z;
    vload(a, i, p, &x);
    vload(b, i, p, &y);
    switch (op) {
      case MPO_OP_MUL: num_mul(&x, &y, p, &z); break;
      case MPO_OP_ADD: num_add(&x, &y, p, &z); break;
      case MPO_OP_SUB: num_sub(&x, &y, p, &z); break;
      case MPO_OP_DIV:
        if (num_div(&x, &y, p, &z) != MPO_OK) {
          set_zero(&z, 0);
          st = MPO_ERR_DIVZERO;
        }
        break;
      default: return MPO_ERR_ARG;
    }
    vstore(r, i, p, &z);
  }
  return st;
}

int mpo_cmp(int p, const uint64_t *a, const uint64_t *b, int *out) {
  if (!prec_ok(p)) return MPO_ERR_PREC;
  num x, y;
  if (rec_load(a, p, &x) || rec_load(b, p, &y)) return MPO_ERR_ARG;
  *out = num_cmp(&x, &y, p);
  return MPO_OK;
}

int mpo_from_f64(int p, int64_t n, const double *d, uint64_t *out) {
  if (!prec_ok(p)) return MPO_ERR_PREC;
  for (int64_t i = 0; i < n; i++) {
    num x;
    if (num_from_f64(d[i], p, &x) != MPO_OK) return MPO_ERR_ARG;
    vstore(out, i, p, &x);
  }
  return MPO_OK;
}

int mpo_to_f64(int p, int64_t n, const uint64_t *a, double *out) {
  if (!prec_ok(p)) return MPO_ERR_PREC;
  if (vcheck(a, n, p)) return MPO_ERR_ARG;
  for (int64_t i = 0; i < n; i++) {
    num x;
    vload(a, i, p, &x);
    out[i] = num_to_f64(&x, p);
  }
  return MPO_OK;
}

/* ------------------------------------------------------------------------ */
/* Public entry points: sparse matrix and vectors                           */
/* ------------------------------------------------------------------------ */

static int csr_check(int64_t n, const int64_t *rowptr, const int32_t *colidx) {
  if (n < 0 || rowptr[0] != 0) return MPO_ERR_ARG;
  for (int64_t i = 0; i < n; i++) {
    if (rowptr[i + 1] < rowptr[i]) return MPO_ERR_ARG;
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; k++) {
      if (colidx[k] < 0 || colidx[k] >= n) return MPO_ERR_ARG;
      if (k > rowptr[i] && colidx[k] <= colidx[k - 1]) return MPO_ERR_ARG;
    }
  }
  return MPO_OK;
}

/* ORDERED row (the paper's CSR loop, Section 3): y <- +0, then for each stored
 * entry in column order, skipping a zero factor (the zero fast path of
 * Section 2), y <- RN(y + RN(a_k * x_col)). */
static void row_ordered(int p, const int64_t *rowptr, const int32_t *colidx,
                        const uint64_t *vals, const uint64_t *x, int64_t i, num *y) {
  set_zero(y, 0);
  for (int64_t k = rowptr[i]; k < rowptr[i + 1]; k++) {
    num a, xc, t, s;
    vload(vals, k, p, &a);
    vload(x, colidx[k], p, &xc);
    if (a.zero || xc.zero) continue;
    num_mul(&a, &xc, p, &t);
    num_add(y, &t, p, &s);
    *y = s;
  }
}

/* EXACT row: y = RN(sum_k a_k x_col(k)) with the sum formed exactly. */
static int row_exact(int p, const int64_t *rowptr, const int32_t *colidx,
                     const uint64_t *vals, const uint64_t *x, int64_t i, num *y) {
  termlist tl;
  tl_init(&tl, p);
  for (int64_t k = rowptr[i]; k < rowptr[i + 1]; k++) {
    num a, xc;
    vload(vals, k, p, &a);
    vload(x, colidx[k], p, &xc);
    tl_add_product(&tl, &a, &xc, 0);
  }
  int st = tl_sum(&tl, y);
  tl_free(&tl);
  return st;
}

int mpo_spmv_rows(int p, int mode, int64_t n, const int64_t *rowptr,
                  const int32_t *colidx, const uint64_t *vals, const uint64_t *x,
                  uint64_t *y, int64_t r0, int64_t r1) {
  if (!prec_ok(p)) return MPO_ERR_PREC;
  if (mode != MPO_ORDERED && mode != MPO_EXACT) return MPO_ERR_ARG;
  if (csr_check(n, rowptr, colidx)) return MPO_ERR_ARG;
  if (r0 < 0 || r1 > n || r0 > r1) return MPO_ERR_ARG;
  if (vcheck(vals, rowptr[n], p) || vcheck(x, n, p)) return MPO_ERR_ARG;
  int st = MPO_OK;
  for (int64_t i = r0; i < r1; i++) {
    num yi;
    if (mode == MPO_ORDERED) {
      row_ordered(p, rowptr, colidx, vals, x, i, &yi);
    } else if (row_exact(p, rowptr, colidx, vals, x, i, &yi) != MPO_OK) {
      st = MPO_ERR_SPAN;
    }
    vstore(y, i, p, &yi);
  }
  return st;
}

int mpo_spmv(int p, int mode, int64_t n, const int64_t *rowptr,
             const int32_t *colidx, const uint64_t *vals, const uint64_t *x,
             uint64_t *y) {
  return mpo_spmv_rows(p, mode, n, rowptr, colidx, vals, x, y, 0, n);
}

int mpo_transpose(int p, int64_t n, const int64_t *rowptr, const int32_t *colidx,
                  const uint64_t *vals, int64_t *trowptr, int32_t *tcolidx,
                  uint64_t *tvals) {
  if (!prec_ok(p)) return MPO_ERR_PREC;
  if (csr_check(n, rowptr, colidx)) return MPO_ERR_ARG;
  int64_t nnz = rowptr[n];
  size_t rl = (size_t)(p / 64 + 1);
  for (int64_t j = 0; j <= n; j++) trowptr[j] = 0;
  for (int64_t k = 0; k < nnz; k++) trowptr[colidx[k] + 1]++;
  for (int64_t j = 0; j < n; j++) trowptr[j + 1] += trowptr[j];
  int64_t *next = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
  if (!next) die("out of memory");
  memcpy(next, trowptr, sizeof(int64_t) * (size_t)(n + 1));
  for (int64_t i = 0; i < n; i++) { /* rows ascending: the sort is stable */
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; k++) {
      int64_t pos = next[colidx[k]]++;
      tcolidx[pos] = (int32_t)i;
      memcpy(tvals + (size_t)pos * rl, vals + (size_t)k * rl, rl * sizeof(uint64_t));
    }
  }
  free(next);
  return MPO_OK;
}

typedef struct {
  int64_t *rowptr;
  int32_t *colidx;
  uint64_t *vals;
} csr_copy;

static int make_transpose(int p, int64_t n, const int64_t *rowptr, const int32_t *colidx,
                          const uint64_t *vals, csr_copy *t) {
  int64_t nnz = rowptr[n];
  size_t rl = (size_t)(p / 64 + 1);
  t->rowptr = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
  t->colidx = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
  t->vals = (uint64_t *)malloc(sizeof(uint64_t) * rl * (size_t)(nnz > 0 ? nnz : 1));
  if (!t->rowptr || !t->colidx || !t->vals) die("out of memory");
  return mpo_transpose(p, n, rowptr, colidx, vals, t->rowptr, t->colidx, t->vals);
}

static void free_copy(csr_copy *t) {
  free(t->rowptr);
  free(t->colidx);
  free(t->vals);
}

int mpo_spmv_t(int p, int mode, int64_t n, const int64_t *rowptr,
               const int32_t *colidx, const uint64_t *vals, const uint64_t *x,
               uint64_t *y) {
  if (!prec_ok(p)) return MPO_ERR_PREC;
  if (csr_check(n, rowptr, colidx)) return MPO_ERR_ARG;
  csr_copy t;
  int st = make_transpose(p, n, rowptr, colidx, vals, &t);
  if (st == MPO_OK) st = mpo_spmv(p, mode, n, t.rowptr, t.colidx, t.vals, x, y);
  free_copy(&t);
  return st;
}

/* out = RN(sum x_i y_i), exact sum, zero pairs skipped. */
static int dot_num(int p, int64_t n, const uint64_t *x, const uint64_t *y, num *out) {
  termlist tl;
  tl_init(&tl, p);
  for (int64_t i = 0; i < n; i++) {
    num a, b;
    vload(x, i, p, &a);
    vload(y, i, p, &b);
    tl_add_product(&tl, &a, &b, 0);
  }
  int st = tl_sum(&tl, out);
  tl_free(&tl);
  return st;
}

int mpo_dot(int p, int64_t n, const uint64_t *x, const uint64_t *y, uint64_t *out) {
  if (!prec_ok(p)) return MPO_ERR_PREC;
  if (n < 0 || vcheck(x, n, p) || vcheck(y, n, p)) return MPO_ERR_ARG;
  num r;
  int st = dot_num(p, n, x, y, &r);
  rec_store(&r, p, out);
  return st;
}

int mpo_axpy(int p, int64_t n, const uint64_t *alpha, const uint64_t *x, uint64_t *y) {
  if (!prec_ok(p)) return MPO_ERR_PREC;
  num al;
  if (rec_load(alpha, p, &al) || n < 0 || vcheck(x, n, p) || vcheck(y, n, p))
    return MPO_ERR_ARG;
  for (int64_t i = 0; i < n; i++) {
    num xi, yi, t, s;
    vload(x, i, p, &xi);
    vload(y, i, p, &yi);
    num_mul(&al, &xi, p, &t);
    num_add(&yi, &t, p, &s);
    vstore(y, i, p, &s);
  }
  return MPO_OK;
}

/* r_i = RN(b_i - sum_k a_k x_col(k)) as one exact sum. */
static int residual_vec(int p, int64_t n, const int64_t *rowptr, const int32_t *colidx,
                        const uint64_t *vals, const uint64_t *b, const uint64_t *x,
                        uint64_t *r) {
  int st = MPO_OK;
  for (int64_t i = 0; i < n; i++) {
    termlist tl;
    tl_init(&tl, p);
    num bi, ri;
    vload(b, i, p, &bi);
    tl_add_value(&tl, &bi, 0);
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; k++) {
      num a, xc;
      vload(vals, k, p, &a);
      vload(x, colidx[k], p, &xc);
      tl_add_product(&tl, &a, &xc, 1);
    }
    if (tl_sum(&tl, &ri) != MPO_OK) st = MPO_ERR_SPAN;
    tl_free(&tl);
    vstore(r, i, p, &ri);
  }
  return st;
}

int mpo_residual(int p, int64_t n, const int64_t *rowptr, const int32_t *colidx,
                 const uint64_t *vals, const uint64_t *b, const uint64_t *x,
                 uint64_t *r) {
  if (!prec_ok(p)) return MPO_ERR_PREC;
  if (csr_check(n, rowptr, colidx)) return MPO_ERR_ARG;
  if (vcheck(vals, rowptr[n], p) || vcheck(b, n, p) || vcheck(x, n, p)) return MPO_ERR_ARG;
  return residual_vec(p, n, rowptr, colidx, vals, b, x, r);
}

/* ------------------------------------------------------------------------ */
/* Krylov solvers (Fig. 5, left preconditioner K = I)                        */
/* ------------------------------------------------------------------------ */

typedef struct {
  int p, mode;
  int64_t n;
  const int64_t *rowptr;
  const int32_t *colidx;
  const uint64_t *vals;
  size_t rl; /* words per record */
} sysA;

static uint64_t *vnew(const sysA *s) {
  uint64_t *v = (uint64_t *)malloc(sizeof(uint64_t) * s->rl * (size_t)(s->n > 0 ? s->n : 1));
  if (!v) die("out of memory");
  num z;
  set_zero(&z, 0);
  for (int64_t i = 0; i < s->n; i++) vstore(v, i, s->p, &z);
  return v;
}

static void vcopy(const sysA *s, uint64_t *dst, const uint64_t *src) {
  memcpy(dst, src, sizeof(uint64_t) * s->rl * (size_t)s->n);
}

static int matvec(const sysA *s, const int64_t *rowptr, const int32_t *colidx,
                  const uint64_t *vals, const uint64_t *x, uint64_t *y) {
  return mpo_spmv(s->p, s->mode, s->n, rowptr, colidx, vals, x, y);
}

static int sdot(const sysA *s, const uint64_t *x, const uint64_t *y, num *out) {
  return dot_num(s->p, s->n, x, y, out);
}

/* Convergence threshold of the stopping rule (r,r) <= RN(RN(T*(r0,r0)) + A)
 * with T = RN(rtol^2), A = RN(atol^2): the squared form of
 * ||r|| <= rtol ||r0|| (+ atol) used in Section 4. */
static void conv_threshold(int p, double rtol, double atol, const num *rr0, num *thr) {
  num rt, at, T, A, t;
  num_from_f64(rtol, p, &rt);
  num_from_f64(atol, p, &at);
  num_mul(&rt, &rt, p, &T);
  num_mul(&at, &at, p, &A);
  num_mul(&T, rr0, p, &t);
  num_add(&t, &A, p, thr);
}

static int solve_args(int p, int mode, int64_t n, const int64_t *rowptr,
                      const int32_t *colidx, const uint64_t *vals, const uint64_t *b,
                      const uint64_t *x, double rtol, double atol, int64_t maxit) {
  if (!prec_ok(p)) return MPO_ERR_PREC;
  if (mode != MPO_ORDERED && mode != MPO_EXACT) return MPO_ERR_ARG;
  if (csr_check(n, rowptr, colidx)) return MPO_ERR_ARG;
  if (vcheck(vals, rowptr[n], p) || vcheck(b, n, p) || vcheck(x, n, p)) return MPO_ERR_ARG;
  if (!(rtol >= 0) || !(atol >= 0) || isinf(rtol) || isinf(atol) || maxit < 0)
    return MPO_ERR_ARG;
  return MPO_OK;
}

/* BiCG, Fig. 5 left, with K = I (so w = r and w~ = r~).  Readings: the shadow
 * product is z~ = A^T p~ (the figure prints A), the shadow direction update
 * uses r~_{i-1}, the stopping rule is checked once r_i is formed, and a zero
 * divisor (p~, z) is a breakdown like rho = 0. */
int mpo_bicg(int p, int mode, int64_t n, const int64_t *rowptr,
             const int32_t *colidx, const uint64_t *vals, const uint64_t *b,
             uint64_t *x, double rtol, double atol, int64_t maxit,
             int64_t *iters, uint64_t *hist) {
  int st = solve_args(p, mode, n, rowptr, colidx, vals, b, x, rtol, atol, maxit);
  *iters = 0;
  if (st) return st;
  sysA s = {p, mode, n, rowptr, colidx, vals, (size_t)(p / 64 + 1)};
  csr_copy At;
  make_transpose(p, n, rowptr, colidx, vals, &At);
  uint64_t *r = vnew(&s), *rt = vnew(&s), *pv = vnew(&s), *pt = vnew(&s);
  uint64_t *z = vnew(&s), *zt = vnew(&s);
  num rr0, rr, thr, rho, rho_prev, beta, alpha, d;
  st = residual_vec(p, n, rowptr, colidx, vals, b, x, r); /* r0 = b - A x0 */
  if (st) goto done;
  vcopy(&s, rt, r); /* r~0 = r0 */
  sdot(&s, r, r, &rr0);
  conv_threshold(p, rtol, atol, &rr0, &thr);
  if (num_cmp(&rr0, &thr, p) <= 0) {
    st = MPO_OK;
    goto done;
  }
  sdot(&s, rt, r, &rho);
  st = MPO_ERR_NOCONV;
  for (int64_t i = 1; i <= maxit; i++) {
    if (rho.zero) {
      st = MPO_ERR_BREAKDOWN;
      break;
    }
    if (i == 1) {
      vcopy(&s, pv, r);
      vcopy(&s, pt, rt);
    } else {
      num_div(&rho, &rho_prev, p, &beta); /* beta = rho_{i-1} / rho_{i-2} */
      for (int64_t k = 0; k < n; k++) {
        num rk, rtk, pk, ptk, t1, t2;
        vload(r, k, p, &rk);
        vload(rt, k, p, &rtk);
        vload(pv, k, p, &pk);
        vload(pt, k, p, &ptk);
        num_mul(&beta, &pk, p, &t1);
        num_add(&rk, &t1, p, &t2); /* p = r + beta p */
        vstore(pv, k, p, &t2);
        num_mul(&beta, &ptk, p, &t1);
        num_add(&rtk, &t1, p, &t2); /* p~ = r~ + beta p~ */
        vstore(pt, k, p, &t2);
      }
    }
    matvec(&s, rowptr, colidx, vals, pv, z);        /* z = A p */
    matvec(&s, At.rowptr, At.colidx, At.vals, pt, zt); /* z~ = A^T p~ */
    sdot(&s, pt, z, &d);
    if (d.zero) {
      st = MPO_ERR_BREAKDOWN;
      break;
    }
    num_div(&rho, &d, p, &alpha); /* alpha = rho_{i-1} / (p~, z) */
    for (int64_t k = 0; k < n; k++) {
      num xk, pk, rk, zk, rtk, ztk, t1, t2;
      vload(x, k, p, &xk);
      vload(pv, k, p, &pk);
      num_mul(&alpha, &pk, p, &t1);
      num_add(&xk, &t1, p, &t2); /* x = x + alpha p */
      vstore(x, k, p, &t2);
      vload(r, k, p, &rk);
      vload(z, k, p, &zk);
      num_mul(&alpha, &zk, p, &t1);
      num_sub(&rk, &t1, p, &t2); /* r = r - alpha z */
      vstore(r, k, p, &t2);
      vload(rt, k, p, &rtk);
      vload(zt, k, p, &ztk);
      num_mul(&alpha, &ztk, p, &t1);
      num_sub(&rtk, &t1, p, &t2); /* r~ = r~ - alpha z~ */
      vstore(rt, k, p, &t2);
    }
    *iters = i;
    sdot(&s, r, r, &rr);
    if (hist) rec_store(&rr, p, hist + (size_t)(i - 1) * s.rl);
    rho_prev = rho;
    sdot(&s, rt, r, &rho);
    if (num_cmp(&rr, &thr, p) <= 0) {
      st = MPO_OK;
      break;
    }
  }
done:
  free(r);
  free(rt);
  free(pv);
  free(pt);
  free(z);
  free(zt);
  free_copy(&At);
  return st;
}

/* GPBiCG, Fig. 5 right (Zhang's product-type method).  Readings: the figure's
 * "z = zeta r + zeta z - alpha u" is read z = zeta r + eta z - alpha u and its
 * "r = t - eta y - zeta u" is read r = t - eta y - zeta v with v = A t; only
 * these keep the recursively updated r equal to b - A x (at i = 1 the printed
 * form already gives r = t - zeta^2 A r0 instead of t - zeta A t).  At i = 1
 * the general u/z/x/r formulas run with u = z = s = 0 and beta = eta = +0.  The
 * stopping rule is checked once r_i is formed; then zeta = 0 exits.  A zero
 * (r~, q) is a breakdown.  A zero divisor of zeta and eta (mu5 at i = 1, tau
 * later) sets zeta = eta = +0: the iteration then ends with x + alpha p and
 * r = t, which is the exact solution when t = 0 (e.g. A = cI), and otherwise
 * leads to the figure's own zeta = 0 exit after the convergence check. */
int mpo_gpbicg(int p, int mode, int64_t n, const int64_t *rowptr,
               const int32_t *colidx, const uint64_t *vals, const uint64_t *b,
               uint64_t *x, double rtol, double atol, int64_t maxit,
               int64_t *iters, uint64_t *hist) {
  int st = solve_args(p, mode, n, rowptr, colidx, vals, b, x, rtol, atol, maxit);
  *iters = 0;
  if (st) return st;
  sysA s = {p, mode, n, rowptr, colidx, vals, (size_t)(p / 64 + 1)};
  uint64_t *r = vnew(&s), *rt = vnew(&s), *pv = vnew(&s), *q = vnew(&s);
  uint64_t *t = vnew(&s), *v = vnew(&s), *w = vnew(&s), *y = vnew(&s);
  uint64_t *u = vnew(&s), *z = vnew(&s), *sv = vnew(&s);
  num rr0, rr, thr, rho, rho_prev, alpha, beta, zeta, eta, d;
  num mu1, mu2, mu3, mu4, mu5, tau, t1, t2, t3;
  set_zero(&beta, 0);
  set_zero(&eta, 0);
  set_zero(&zeta, 0);
  st = residual_vec(p, n, rowptr, colidx, vals, b, x, r); /* r0 = b - A x0 */
  if (st) goto done;
  vcopy(&s, rt, r); /* r~ = r0 */
  sdot(&s, r, r, &rr0);
  conv_threshold(p, rtol, atol, &rr0, &thr);
  if (num_cmp(&rr0, &thr, p) <= 0) {
    st = MPO_OK;
    goto done;
  }
  sdot(&s, rt, r, &rho);
  st = MPO_ERR_NOCONV;
  for (int64_t i = 1; i <= maxit; i++) {
    if (rho.zero) {
      st = MPO_ERR_BREAKDOWN;
      break;
    }
    if (i == 1) {
      vcopy(&s, pv, r); /* p = r0 */
      matvec(&s, rowptr, colidx, vals, pv, q); /* q = A p */
      sdot(&s, rt, q, &d);
      if (d.zero) {
        st = MPO_ERR_BREAKDOWN;
        break;
      }
      num_div(&rho, &d, p, &alpha);
      for (int64_t k = 0; k < n; k++) {
        num rk, qk, aq;
        vload(r, k, p, &rk);
        vload(q, k, p, &qk);
        num_mul(&alpha, &qk, p, &aq);
        num_sub(&rk, &aq, p, &t1); /* t = r - alpha q */
        vstore(t, k, p, &t1);
        num_sub(&aq, &rk, p, &t2); /* y = alpha q - r */
        vstore(y, k, p, &t2);
      }
      matvec(&s, rowptr, colidx, vals, t, v); /* v = A t */
      sdot(&s, v, t, &mu2);
      sdot(&s, v, v, &mu5);
      if (mu5.zero) /* v = A t = 0: zeta = 0 (see the reading above) */
        set_zero(&zeta, 0);
      else
        num_div(&mu2, &mu5, p, &zeta); /* zeta = mu2 / mu5 */
      set_zero(&eta, 0);
    } else {
      num_div(&rho, &rho_prev, p, &t1);
      num_div(&alpha, &zeta, p, &t2);
      num_mul(&t1, &t2, p, &beta); /* beta = (rho_{i-1}/rho_{i-2})(alpha_{i-1}/zeta) */
      for (int64_t k = 0; k < n; k++) {
        num vk, qk, rk, pk, uk, a1, a2, a3;
        vload(v, k, p, &vk);
        vload(q, k, p, &qk);
        vload(r, k, p, &rk);
        vload(pv, k, p, &pk);
        vload(u, k, p, &uk);
        num_mul(&beta, &qk, p, &a1);
        num_add(&vk, &a1, p, &a2); /* w = v + beta q */
        vstore(w, k, p, &a2);
        num_sub(&pk, &uk, p, &a1);
        num_mul(&beta, &a1, p, &a2);
        num_add(&rk, &a2, p, &a3); /* p = r + beta (p - u) */
        vstore(pv, k, p, &a3);
      }
      matvec(&s, rowptr, colidx, vals, pv, q); /* q = A p */
      sdot(&s, rt, q, &d);
      if (d.zero) {
        st = MPO_ERR_BREAKDOWN;
        break;
      }
      num_div(&rho, &d, p, &alpha); /* alpha = rho_{i-1} / (r~, q) */
      for (int64_t k = 0; k < n; k++) {
        num tk, rk, qk, a1, a2;
        vload(t, k, p, &tk);
        vload(r, k, p, &rk);
        vload(q, k, p, &qk);
        num_sub(&tk, &rk, p, &a1); /* s = t - r */
        vstore(sv, k, p, &a1);
        num_mul(&alpha, &qk, p, &a1);
        num_sub(&rk, &a1, p, &a2); /* t = r - alpha q */
        vstore(t, k, p, &a2);
      }
      matvec(&s, rowptr, colidx, vals, t, v); /* v = A t */
      for (int64_t k = 0; k < n; k++) {
        num sk, wk, qk, a1, a2, a3;
        vload(sv, k, p, &sk);
        vload(w, k, p, &wk);
        vload(q, k, p, &qk);
        num_sub(&wk, &qk, p, &a1);
        num_mul(&alpha, &a1, p, &a2);
        num_sub(&sk, &a2, p, &a3); /* y = s - alpha (w - q) */
        vstore(y, k, p, &a3);
      }
      sdot(&s, y, y, &mu1);
      sdot(&s, v, t, &mu2);
      sdot(&s, y, t, &mu3);
      sdot(&s, v, y, &mu4);
      sdot(&s, v, v, &mu5);
      num_mul(&mu5, &mu1, p, &t1);
      num_mul(&mu4, &mu4, p, &t2);
      num_sub(&t1, &t2, p, &tau); /* tau = mu5 mu1 - mu4 mu4 */
      if (tau.zero) { /* zeta = eta = 0 (see the reading above) */
        set_zero(&zeta, 0);
        set_zero(&eta, 0);
      } else {
        num_mul(&mu1, &mu2, p, &t1);
        num_mul(&mu3, &mu4, p, &t2);
        num_sub(&t1, &t2, p, &t3);
        num_div(&t3, &tau, p, &zeta); /* zeta = (mu1 mu2 - mu3 mu4) / tau */
        num_mul(&mu5, &mu3, p, &t1);
        num_mul(&mu4, &mu2, p, &t2);
        num_sub(&t1, &t2, p, &t3);
        num_div(&t3, &tau, p, &eta); /* eta = (mu5 mu3 - mu4 mu2) / tau */
      }
    }
    for (int64_t k = 0; k < n; k++) {
      num qk, sk, uk, rk, zk, xk, pk, tk, yk, vk, a1, a2, a3, a4;
      vload(q, k, p, &qk);
      vload(sv, k, p, &sk);
      vload(u, k, p, &uk);
      vload(r, k, p, &rk);
      vload(z, k, p, &zk);
      vload(x, k, p, &xk);
      vload(pv, k, p, &pk);
      vload(t, k, p, &tk);
      vload(y, k, p, &yk);
      vload(v, k, p, &vk);
      /* u = zeta q + eta (s + beta u) */
      num_mul(&beta, &uk, p, &a1);
      num_add(&sk, &a1, p, &a2);
      num_mul(&eta, &a2, p, &a3);
      num_mul(&zeta, &qk, p, &a1);
      num_add(&a1, &a3, p, &uk);
      vstore(u, k, p, &uk);
      /* z = zeta r + eta z - alpha u */
      num_mul(&zeta, &rk, p, &a1);
      num_mul(&eta, &zk, p, &a2);
      num_add(&a1, &a2, p, &a3);
      num_mul(&alpha, &uk, p, &a1);
      num_sub(&a3, &a1, p, &zk);
      vstore(z, k, p, &zk);
      /* x = x + alpha p + z */
      num_mul(&alpha, &pk, p, &a1);
      num_add(&xk, &a1, p, &a2);
      num_add(&a2, &zk, p, &a3);
      vstore(x, k, p, &a3);
      /* r = t - eta y - zeta v */
      num_mul(&eta, &yk, p, &a1);
      num_sub(&tk, &a1, p, &a2);
      num_mul(&zeta, &vk, p, &a1);
      num_sub(&a2, &a1, p, &a4);
      vstore(r, k, p, &a4);
    }
    *iters = i;
    sdot(&s, r, r, &rr);
    if (hist) rec_store(&rr, p, hist + (size_t)(i - 1) * s.rl);
    rho_prev = rho;
    sdot(&s, rt, r, &rho);
    if (num_cmp(&rr, &thr, p) <= 0) {
      st = MPO_OK;
      break;
    }
    if (zeta.zero) {
      st = MPO_ERR_BREAKDOWN;
      break;
    }
  }
done:
  free(r);
  free(rt);
  free(pv);
  free(q);
  free(t);
  free(v);
  free(w);
  free(y);
  free(u);
  free(z);
  free(sv);
  return st;
}

/* CGS (Sonneveld's conjugate gradient squared; Section 4 runs it, the paper
 * prints no algorithm, so the textbook form with K = I is taken, Saad,
 * Iterative Methods for Sparse Linear Systems, Alg. 7.6).  With r~ = r0 and
 * rho_{i-1} = (r~, r_{i-1}):
 *   i = 1: u = p = r0;  i > 1: beta = rho_{i-1}/rho_{i-2},
 *   u = r + beta q,  p = u + beta (q + beta p);
 *   v = A p,  alpha = rho_{i-1} / (r~, v),  q = u - alpha v,  w = u + q,
 *   x = x + alpha w,  r = r - alpha A w.
 * Each printed product and sum is rounded, left to right; (r~, v) = 0 and
 * rho = 0 are breakdowns; the stopping rule is checked once r_i is formed
 * (the same order of exits as BiCG). */
int mpo_cgs(int p, int mode, int64_t n, const int64_t *rowptr,
            const int32_t *colidx, const uint64_t *vals, const uint64_t *b,
            uint64_t *x, double rtol, double atol, int64_t maxit,
            int64_t *iters, uint64_t *hist) {
  int st = solve_args(p, mode, n, rowptr, colidx, vals, b, x, rtol, atol, maxit);
  *iters = 0;
  if (st) return st;
  sysA s = {p, mode, n, rowptr, colidx, vals, (size_t)(p / 64 + 1)};
  uint64_t *r = vnew(&s), *rt = vnew(&s), *u = vnew(&s), *pv = vnew(&s);
  uint64_t *q = vnew(&s), *v = vnew(&s), *w = vnew(&s), *aw = vnew(&s);
  num rr0, rr, thr, rho, rho_prev, alpha, beta, d;
  st = residual_vec(p, n, rowptr, colidx, vals, b, x, r); /* r0 = b - A x0 */
  if (st) goto done;
  vcopy(&s, rt, r); /* r~ = r0 */
  sdot(&s, r, r, &rr0);
  conv_threshold(p, rtol, atol, &rr0, &thr);
  if (num_cmp(&rr0, &thr, p) <= 0) {
    st = MPO_OK;
    goto done;
  }
  sdot(&s, rt, r, &rho);
  st = MPO_ERR_NOCONV;
  for (int64_t i = 1; i <= maxit; i++) {
    if (rho.zero) {
      st = MPO_ERR_BREAKDOWN;
      break;
    }
    if (i == 1) {
      vcopy(&s, u, r);
      vcopy(&s, pv, r);
    } else {
      num_div(&rho, &rho_prev, p, &beta); /* beta = rho_{i-1} / rho_{i-2} */
      for (int64_t k = 0; k < n; k++) {
        num rk, qk, pk, a1, a2, a3, uk;
        vload(r, k, p, &rk);
        vload(q, k, p, &qk);
        vload(pv, k, p, &pk);
        num_mul(&beta, &qk, p, &a1);
        num_add(&rk, &a1, p, &uk); /* u = r + beta q */
        vstore(u, k, p, &uk);
        num_mul(&beta, &pk, p, &a1);
        num_add(&qk, &a1, p, &a2);
        num_mul(&beta, &a2, p, &a3);
        num_add(&uk, &a3, p, &a1); /* p = u + beta (q + beta p) */
        vstore(pv, k, p, &a1);
      }
    }
    matvec(&s, rowptr, colidx, vals, pv, v); /* v = A p */
    sdot(&s, rt, v, &d);
    if (d.zero) {
      st = MPO_ERR_BREAKDOWN;
      break;
    }
    num_div(&rho, &d, p, &alpha); /* alpha = rho_{i-1} / (r~, v) */
    for (int64_t k = 0; k < n; k++) {
      num uk, vk, xk, a1, qk, wk;
      vload(u, k, p, &uk);
      vload(v, k, p, &vk);
      num_mul(&alpha, &vk, p, &a1);
      num_sub(&uk, &a1, p, &qk); /* q = u - alpha v */
      vstore(q, k, p, &qk);
      num_add(&uk, &qk, p, &wk); /* w = u + q */
      vstore(w, k, p, &wk);
      vload(x, k, p, &xk);
      num_mul(&alpha, &wk, p, &a1);
      num_add(&xk, &a1, p, &qk); /* x = x + alpha w */
      vstore(x, k, p, &qk);
    }
    matvec(&s, rowptr, colidx, vals, w, aw); /* A w */
    for (int64_t k = 0; k < n; k++) {
      num rk, ak, a1, a2;
      vload(r, k, p, &rk);
      vload(aw, k, p, &ak);
      num_mul(&alpha, &ak, p, &a1);
      num_sub(&rk, &a1, p, &a2); /* r = r - alpha A w */
      vstore(r, k, p, &a2);
    }
    *iters = i;
    sdot(&s, r, r, &rr);
    if (hist) rec_store(&rr, p, hist + (size_t)(i - 1) * s.rl);
    rho_prev = rho;
    sdot(&s, rt, r, &rho);
    if (num_cmp(&rr, &thr, p) <= 0) {
      st = MPO_OK;
      break;
    }
  }
done:
  free(r);
  free(rt);
  free(u);
  free(pv);
  free(q);
  free(v);
  free(w);
  free(aw);
  return st;
}

/* BiCGSTAB (van der Vorst; Section 4 runs it, the paper prints no algorithm,
 * so the textbook form with K = I is taken, Saad, Alg. 7.7).  With r~ = r0:
 *   i = 1: p = r0;  i > 1: beta = (rho_{i-1}/rho_{i-2}) (alpha/omega),
 *   p = r + beta (p - omega v);
 *   v = A p,  alpha = rho_{i-1} / (r~, v),  s = r - alpha v,  t = A s,
 *   omega = (t, s) / (t, t)  (+0 when t = 0),
 *   x = x + alpha p + omega s,  r = s - omega t.
 * Each printed product and sum is rounded, left to right; (r~, v) = 0 and
 * rho = 0 are breakdowns.  Exits after r_i is formed: the stopping rule,
 * then omega = 0 (the next beta would divide by it) as a breakdown; reaching
 * maxit wins over a zero rho found for the next iteration. */
int mpo_bicgstab(int p, int mode, int64_t n, const int64_t *rowptr,
                 const int32_t *colidx, const uint64_t *vals, const uint64_t *b,
                 uint64_t *x, double rtol, double atol, int64_t maxit,
                 int64_t *iters, uint64_t *hist) {
  int st = solve_args(p, mode, n, rowptr, colidx, vals, b, x, rtol, atol, maxit);
  *iters = 0;
  if (st) return st;
  sysA s = {p, mode, n, rowptr, colidx, vals, (size_t)(p / 64 + 1)};
  uint64_t *r = vnew(&s), *rt = vnew(&s), *pv = vnew(&s), *v = vnew(&s);
  uint64_t *sv = vnew(&s), *t = vnew(&s);
  num rr0, rr, thr, rho, rho_prev, alpha, beta, omega, d, tt, ts, t1, t2;
  set_zero(&omega, 0);
  set_zero(&alpha, 0);
  st = residual_vec(p, n, rowptr, colidx, vals, b, x, r); /* r0 = b - A x0 */
  if (st) goto done;
  vcopy(&s, rt, r); /* r~ = r0 */
  sdot(&s, r, r, &rr0);
  conv_threshold(p, rtol, atol, &rr0, &thr);
  if (num_cmp(&rr0, &thr, p) <= 0) {
    st = MPO_OK;
    goto done;
  }
  sdot(&s, rt, r, &rho);
  st = MPO_ERR_NOCONV;
  for (int64_t i = 1; i <= maxit; i++) {
    if (rho.zero) {
      st = MPO_ERR_BREAKDOWN;
      break;
    }
    if (i == 1) {
      vcopy(&s, pv, r);
    } else {
      num_div(&rho, &rho_prev, p, &t1);
      num_div(&alpha, &omega, p, &t2);
      num_mul(&t1, &t2, p, &beta); /* beta = (rho_{i-1}/rho_{i-2}) (alpha/omega) */
      for (int64_t k = 0; k < n; k++) {
        num rk, pk, vk, a1, a2, a3;
        vload(r, k, p, &rk);
        vload(pv, k, p, &pk);
        vload(v, k, p, &vk);
        num_mul(&omega, &vk, p, &a1);
        num_sub(&pk, &a1, p, &a2);
        num_mul(&beta, &a2, p, &a3);
        num_add(&rk, &a3, p, &a1); /* p = r + beta (p - omega v) */
        vstore(pv, k, p, &a1);
      }
    }
    matvec(&s, rowptr, colidx, vals, pv, v); /* v = A p */
    sdot(&s, rt, v, &d);
    if (d.zero) {
      st = MPO_ERR_BREAKDOWN;
      break;
    }
    num_div(&rho, &d, p, &alpha); /* alpha = rho_{i-1} / (r~, v) */
    for (int64_t k = 0; k < n; k++) {
      num rk, vk, a1, sk;
      vload(r, k, p, &rk);
      vload(v, k, p, &vk);
      num_mul(&alpha, &vk, p, &a1);
      num_sub(&rk, &a1, p, &sk); /* s = r - alpha v */
      vstore(sv, k, p, &sk);
    }
    matvec(&s, rowptr, colidx, vals, sv, t); /* t = A s */
    sdot(&s, t, sv, &ts);
    sdot(&s, t, t, &tt);
    if (tt.zero)
      set_zero(&omega, 0);
    else
      num_div(&ts, &tt, p, &omega); /* omega = (t, s) / (t, t) */
    for (int64_t k = 0; k < n; k++) {
      num xk, pk, sk, tk, a1, a2, a3;
      vload(x, k, p, &xk);
      vload(pv, k, p, &pk);
      vload(sv, k, p, &sk);
      vload(t, k, p, &tk);
      num_mul(&alpha, &pk, p, &a1);
      num_add(&xk, &a1, p, &a2);
      num_mul(&omega, &sk, p, &a1);
      num_add(&a2, &a1, p, &a3); /* x = x + alpha p + omega s */
      vstore(x, k, p, &a3);
      num_mul(&omega, &tk, p, &a1);
      num_sub(&sk, &a1, p, &a2); /* r = s - omega t */
      vstore(r, k, p, &a2);
    }
    *iters = i;
    sdot(&s, r, r, &rr);
    if (hist) rec_store(&rr, p, hist + (size_t)(i - 1) * s.rl);
    rho_prev = rho;
    sdot(&s, rt, r, &rho);
    if (num_cmp(&rr, &thr, p) <= 0) {
      st = MPO_OK;
      break;
    }
    if (omega.zero) {
      st = MPO_ERR_BREAKDOWN;
      break;
    }
  }
done:
  free(r);
  free(rt);
  free(pv);
  free(v);
  free(sv);
  free(t);
  return st;
}

/* ------------------------------------------------------------------------ */
/* ILU(0) preconditioning (Section 4's BiCGSTAB+ILU(0) rows; the paper prints
 * no algorithm, the textbook IKJ form is taken, Saad, Alg. 10.4).  The factors
 * share A's pattern: L (unit lower, the entries left of the diagonal) and U
 * (the diagonal and right of it) overwrite a copy of A's values in CSR order.
 * For each row i, for each stored (i, k) with k < i in ascending k:
 *   a_ik = RN(a_ik / a_kk);
 *   for each stored (i, j) with j > k in ascending j, if (k, j) is stored:
 *     a_ij = RN(a_ij - RN(a_ik a_kj)).
 * Every operation is rounded; no product is skipped.  A missing or zero
 * pivot a_kk returns MPO_ERR_DIVZERO. */

static int64_t row_find(const int64_t *rowptr, const int32_t *colidx, int64_t i, int32_t j) {
  for (int64_t k = rowptr[i]; k < rowptr[i + 1]; k++)
    if (colidx[k] == j) return k;
  return -1;
}

int mpo_ilu0(int p, int64_t n, const int64_t *rowptr, const int32_t *colidx,
             const uint64_t *vals, uint64_t *lu) {
  if (!prec_ok(p)) return MPO_ERR_PREC;
  if (csr_check(n, rowptr, colidx)) return MPO_ERR_ARG;
  if (vcheck(vals, rowptr[n], p)) return MPO_ERR_ARG;
  size_t rl = (size_t)(p / 64 + 1);
  memcpy(lu, vals, sizeof(uint64_t) * rl * (size_t)rowptr[n]);
  for (int64_t i = 0; i < n; i++) {
    for (int64_t ik = rowptr[i]; ik < rowptr[i + 1] && colidx[ik] < i; ik++) {
      const int32_t k = colidx[ik];
      const int64_t kk = row_find(rowptr, colidx, k, k);
      if (kk < 0) return MPO_ERR_DIVZERO;
      num akk, aik, q;
      vload(lu, kk, p, &akk);
      if (akk.zero) return MPO_ERR_DIVZERO;
      vload(lu, ik, p, &aik);
      num_div(&aik, &akk, p, &q); /* l_ik = a_ik / u_kk */
      vstore(lu, ik, p, &q);
      for (int64_t ij = ik + 1; ij < rowptr[i + 1]; ij++) {
        const int64_t kj = row_find(rowptr, colidx, k, colidx[ij]);
        if (kj < 0) continue;
        num akj, aij, t, u;
        vload(lu, kj, p, &akj);
        vload(lu, ij, p, &aij);
        num_mul(&q, &akj, p, &t);
        num_sub(&aij, &t, p, &u); /* a_ij = a_ij - l_ik u_kj */
        vstore(lu, ij, p, &u);
      }
    }
  }
  return MPO_OK;
}

/* w = (LU)^{-1} r with the factors of mpo_ilu0: forward, y_i = r_i minus the
 * rounded products l_ik y_k (k < i, ascending), one rounding per step; then
 * backward from the last row, w_i = RN((y_i minus u_ik w_k, k > i
 * ascending) / u_ii).  Returns MPO_ERR_DIVZERO on a zero or missing u_ii. */
static int ilu0_apply(int p, int64_t n, const int64_t *rowptr, const int32_t *colidx,
                      const uint64_t *lu, const uint64_t *r, uint64_t *w) {
  for (int64_t i = 0; i < n; i++) { /* forward, into w */
    num acc, l, y, t, u;
    vload(r, i, p, &acc);
    for (int64_t k = rowptr[i]; k < rowptr[i + 1] && colidx[k] < i; k++) {
      vload(lu, k, p, &l);
      vload(w, colidx[k], p, &y);
      num_mul(&l, &y, p, &t);
      num_sub(&acc, &t, p, &u);
      acc = u;
    }
    vstore(w, i, p, &acc);
  }
  for (int64_t i = n - 1; i >= 0; i--) { /* backward, in place */
    num acc, a, z, t, u, d;
    int64_t dk = -1;
    vload(w, i, p, &acc);
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; k++) {
      if (colidx[k] == i) dk = k;
      if (colidx[k] <= i) continue;
      vload(lu, k, p, &a);
      vload(w, colidx[k], p, &z);
      num_mul(&a, &z, p, &t);
      num_sub(&acc, &t, p, &u);
      acc = u;
    }
    if (dk < 0) return MPO_ERR_DIVZERO;
    vload(lu, dk, p, &d);
    if (d.zero) return MPO_ERR_DIVZERO;
    num_div(&acc, &d, p, &u);
    vstore(w, i, p, &u);
  }
  return MPO_OK;
}

int mpo_ilu0_apply(int p, int64_t n, const int64_t *rowptr, const int32_t *colidx,
                   const uint64_t *lu, const uint64_t *r, uint64_t *w) {
  if (!prec_ok(p)) return MPO_ERR_PREC;
  if (csr_check(n, rowptr, colidx)) return MPO_ERR_ARG;
  if (vcheck(lu, rowptr[n], p) || vcheck(r, n, p)) return MPO_ERR_ARG;
  return ilu0_apply(p, n, rowptr, colidx, lu, r, w);
}

/* BiCGSTAB with ILU(0) as a right preconditioner M = LU (the preconditioned
 * BiCGSTAB of Barrett et al., Templates for the Solution of Linear Systems):
 * as mpo_bicgstab with p^ = M^{-1} p and s^ = M^{-1} s,
 *   v = A p^,  t = A s^,  x = x + alpha p^ + omega s^;
 * r stays the residual b - A x of the unpreconditioned system, so the
 * stopping rule is unchanged.  A zero pivot of the factorization returns
 * MPO_ERR_DIVZERO before the first iteration.  Kept beside the paper's left
 * form (mpo_bicgstab_ilu0) as an option. */
int mpo_bicgstab_ilu0_right(int p, int mode, int64_t n, const int64_t *rowptr,
                      const int32_t *colidx, const uint64_t *vals, const uint64_t *b,
                      uint64_t *x, double rtol, double atol, int64_t maxit,
                      int64_t *iters, uint64_t *hist) {
  int st = solve_args(p, mode, n, rowptr, colidx, vals, b, x, rtol, atol, maxit);
  *iters = 0;
  if (st) return st;
  sysA s = {p, mode, n, rowptr, colidx, vals, (size_t)(p / 64 + 1)};
  uint64_t *lu = (uint64_t *)malloc(sizeof(uint64_t) * s.rl * (size_t)(rowptr[n] > 0 ? rowptr[n] : 1));
  if (!lu) die("out of memory");
  uint64_t *r = vnew(&s), *rt = vnew(&s), *pv = vnew(&s), *ph = vnew(&s), *v = vnew(&s);
  uint64_t *sv = vnew(&s), *sh = vnew(&s), *t = vnew(&s);
  num rr0, rr, thr, rho, rho_prev, alpha, beta, omega, d, tt, ts, t1, t2;
  set_zero(&omega, 0);
  set_zero(&alpha, 0);
  st = mpo_ilu0(p, n, rowptr, colidx, vals, lu);
  if (st) goto done;
  st = residual_vec(p, n, rowptr, colidx, vals, b, x, r); /* r0 = b - A x0 */
  if (st) goto done;
  vcopy(&s, rt, r);
  sdot(&s, r, r, &rr0);
  conv_threshold(p, rtol, atol, &rr0, &thr);
  if (num_cmp(&rr0, &thr, p) <= 0) {
    st = MPO_OK;
    goto done;
  }
  sdot(&s, rt, r, &rho);
  st = MPO_ERR_NOCONV;
  for (int64_t i = 1; i <= maxit; i++) {
    if (rho.zero) {
      st = MPO_ERR_BREAKDOWN;
      break;
    }
    if (i == 1) {
      vcopy(&s, pv, r);
    } else {
      num_div(&rho, &rho_prev, p, &t1);
      num_div(&alpha, &omega, p, &t2);
      num_mul(&t1, &t2, p, &beta);
      for (int64_t k = 0; k < n; k++) {
        num rk, pk, vk, a1, a2, a3;
        vload(r, k, p, &rk);
        vload(pv, k, p, &pk);
        vload(v, k, p, &vk);
        num_mul(&omega, &vk, p, &a1);
        num_sub(&pk, &a1, p, &a2);
        num_mul(&beta, &a2, p, &a3);
        num_add(&rk, &a3, p, &a1); /* p = r + beta (p - omega v) */
        vstore(pv, k, p, &a1);
      }
    }
    int ast = ilu0_apply(p, n, rowptr, colidx, lu, pv, ph); /* p^ */
    if (ast != MPO_OK) {
      st = ast;
      break;
    }
    matvec(&s, rowptr, colidx, vals, ph, v); /* v = A p^ */
    sdot(&s, rt, v, &d);
    if (d.zero) {
      st = MPO_ERR_BREAKDOWN;
      break;
    }
    num_div(&rho, &d, p, &alpha);
    for (int64_t k = 0; k < n; k++) {
      num rk, vk, a1, sk;
      vload(r, k, p, &rk);
      vload(v, k, p, &vk);
      num_mul(&alpha, &vk, p, &a1);
      num_sub(&rk, &a1, p, &sk); /* s = r - alpha v */
      vstore(sv, k, p, &sk);
    }
    ast = ilu0_apply(p, n, rowptr, colidx, lu, sv, sh); /* s^ */
    if (ast != MPO_OK) {
      st = ast;
      break;
    }
    matvec(&s, rowptr, colidx, vals, sh, t); /* t = A s^ */
    sdot(&s, t, sv, &ts);
    sdot(&s, t, t, &tt);
    if (tt.zero)
      set_zero(&omega, 0);
    else
      num_div(&ts, &tt, p, &omega);
    for (int64_t k = 0; k < n; k++) {
      num xk, pk, sk, shk, tk, a1, a2, a3;
      vload(x, k, p, &xk);
      vload(ph, k, p, &pk);
      vload(sh, k, p, &shk);
      vload(sv, k, p, &sk);
      vload(t, k, p, &tk);
      num_mul(&alpha, &pk, p, &a1);
      num_add(&xk, &a1, p, &a2);
      num_mul(&omega, &shk, p, &a1);
      num_add(&a2, &a1, p, &a3); /* x = x + alpha p^ + omega s^ */
      vstore(x, k, p, &a3);
      num_mul(&omega, &tk, p, &a1);
      num_sub(&sk, &a1, p, &a2); /* r = s - omega t */
      vstore(r, k, p, &a2);
    }
    *iters = i;
    sdot(&s, r, r, &rr);
    if (hist) rec_store(&rr, p, hist + (size_t)(i - 1) * s.rl);
    rho_prev = rho;
    sdot(&s, rt, r, &rho);
    if (num_cmp(&rr, &thr, p) <= 0) {
      st = MPO_OK;
      break;
    }
    if (omega.zero) {
      st = MPO_ERR_BREAKDOWN;
      break;
    }
  }
done:
  free(lu);
  free(r);
  free(rt);
  free(pv);
  free(ph);
  free(v);
  free(sv);
  free(sh);
  free(t);
  return st;
}

/* BiCGSTAB with ILU(0) as the left preconditioner K = LU, the paper's
 * preconditioned method (Section 4.2, Table 3; Fig. 5 calls K the matrix for
 * left preconditioning and applies it by solving K w = r).  The method is BiCGSTAB (as mpo_bicgstab, the same op
 * order) run on the preconditioned system K^{-1} A x = K^{-1} b, so every
 * residual it carries is a preconditioned one:
 *   r^_0 = K^{-1} (b - A x_0)  (the exact residual, rounded once, then K^{-1}),
 *   r~ = r^_0, rho = (r~, r^),
 *   p = r^ (i = 1), else p = RN(r^ + RN(beta RN(p - RN(omega v)))),
 *   v = K^{-1} (A p), alpha = RN(rho / (r~, v)), s = RN(r^ - RN(alpha v)),
 *   t = K^{-1} (A s), omega = RN((t, s) / (t, t)) (+0 when (t, t) = 0),
 *   x = RN(RN(x + RN(alpha p)) + RN(omega s)), r^ = RN(s - RN(omega t)).
 * The stopping rule and the history take the recursive preconditioned
 * residual: (r^, r^) <= RN(RN(rtol^2) (r^_0, r^_0)) + RN(atol^2).  The true
 * residual b - A x is not formed during the iteration.  Exits as
 * mpo_bicgstab; a zero pivot returns MPO_ERR_DIVZERO before iteration 1. */
int mpo_bicgstab_ilu0(int p, int mode, int64_t n, const int64_t *rowptr,
                      const int32_t *colidx, const uint64_t *vals, const uint64_t *b,
                      uint64_t *x, double rtol, double atol, int64_t maxit,
                      int64_t *iters, uint64_t *hist) {
  int st = solve_args(p, mode, n, rowptr, colidx, vals, b, x, rtol, atol, maxit);
  *iters = 0;
  if (st) return st;
  sysA s = {p, mode, n, rowptr, colidx, vals, (size_t)(p / 64 + 1)};
  uint64_t *lu = (uint64_t *)malloc(sizeof(uint64_t) * s.rl * (size_t)(rowptr[n] > 0 ? rowptr[n] : 1));
  if (!lu) die("out of memory");
  uint64_t *r = vnew(&s), *rt = vnew(&s), *pv = vnew(&s), *v = vnew(&s);
  uint64_t *sv = vnew(&s), *t = vnew(&s), *q = vnew(&s);
  num rr0, rr, thr, rho, rho_prev, alpha, beta, omega, d, tt, ts, t1, t2;
  set_zero(&omega, 0);
  set_zero(&alpha, 0);
  st = mpo_ilu0(p, n, rowptr, colidx, vals, lu);
  if (st) goto done;
  st = residual_vec(p, n, rowptr, colidx, vals, b, x, q); /* b - A x0 */
  if (st) goto done;
  st = ilu0_apply(p, n, rowptr, colidx, lu, q, r); /* r^0 = K^{-1} (b - A x0) */
  if (st) goto done;
  vcopy(&s, rt, r);
  sdot(&s, r, r, &rr0);
  conv_threshold(p, rtol, atol, &rr0, &thr);
  if (num_cmp(&rr0, &thr, p) <= 0) {
    st = MPO_OK;
    goto done;
  }
  sdot(&s, rt, r, &rho);
  st = MPO_ERR_NOCONV;
  for (int64_t i = 1; i <= maxit; i++) {
    if (rho.zero) {
      st = MPO_ERR_BREAKDOWN;
      break;
    }
    if (i == 1) {
      vcopy(&s, pv, r);
    } else {
      num_div(&rho, &rho_prev, p, &t1);
      num_div(&alpha, &omega, p, &t2);
      num_mul(&t1, &t2, p, &beta);
      for (int64_t k = 0; k < n; k++) {
        num rk, pk, vk, a1, a2, a3;
        vload(r, k, p, &rk);
        vload(pv, k, p, &pk);
        vload(v, k, p, &vk);
        num_mul(&omega, &vk, p, &a1);
        num_sub(&pk, &a1, p, &a2);
        num_mul(&beta, &a2, p, &a3);
        num_add(&rk, &a3, p, &a1); /* p = r^ + beta (p - omega v) */
        vstore(pv, k, p, &a1);
      }
    }
    matvec(&s, rowptr, colidx, vals, pv, q); /* A p */
    int ast = ilu0_apply(p, n, rowptr, colidx, lu, q, v); /* v = K^{-1} A p */
    if (ast != MPO_OK) {
      st = ast;
      break;
    }
    sdot(&s, rt, v, &d);
    if (d.zero) {
      st = MPO_ERR_BREAKDOWN;
      break;
    }
    num_div(&rho, &d, p, &alpha);
    for (int64_t k = 0; k < n; k++) {
      num rk, vk, a1, sk;
      vload(r, k, p, &rk);
      vload(v, k, p, &vk);
      num_mul(&alpha, &vk, p, &a1);
      num_sub(&rk, &a1, p, &sk); /* s = r^ - alpha v */
      vstore(sv, k, p, &sk);
    }
    matvec(&s, rowptr, colidx, vals, sv, q); /* A s */
    ast = ilu0_apply(p, n, rowptr, colidx, lu, q, t); /* t = K^{-1} A s */
    if (ast != MPO_OK) {
      st = ast;
      break;
    }
    sdot(&s, t, sv, &ts);
    sdot(&s, t, t, &tt);
    if (tt.zero)
      set_zero(&omega, 0);
    else
      num_div(&ts, &tt, p, &omega);
    for (int64_t k = 0; k < n; k++) {
      num xk, pk, sk, tk, a1, a2, a3;
      vload(x, k, p, &xk);
      vload(pv, k, p, &pk);
      vload(sv, k, p, &sk);
      vload(t, k, p, &tk);
      num_mul(&alpha, &pk, p, &a1);
      num_add(&xk, &a1, p, &a2);
      num_mul(&omega, &sk, p, &a1);
      num_add(&a2, &a1, p, &a3); /* x = x + alpha p + omega s */
      vstore(x, k, p, &a3);
      num_mul(&omega, &tk, p, &a1);
      num_sub(&sk, &a1, p, &a2); /* r^ = s - omega t */
      vstore(r, k, p, &a2);
    }
    *iters = i;
    sdot(&s, r, r, &rr);
    if (hist) rec_store(&rr, p, hist + (size_t)(i - 1) * s.rl);
    rho_prev = rho;
    sdot(&s, rt, r, &rho);
    if (num_cmp(&rr, &thr, p) <= 0) {
      st = MPO_OK;
      break;
    }
    if (omega.zero) {
      st = MPO_ERR_BREAKDOWN;
      break;
    }
  }
done:
  free(lu);
  free(r);
  free(rt);
  free(pv);
  free(v);
  free(sv);
  free(t);
  free(q);
  return st;
}
