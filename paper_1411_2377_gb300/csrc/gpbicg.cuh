// gpbicg.cuh -- GPBiCG's vector updates for one element (Fig. 5 right, in
// the evaluation order the oracle follows), shared by the single solver
// (solvers.cu) and the batched solver (batch.cu).
#pragma once
#include "mpdev.cuh"

namespace mpk {

struct Vecs {
  uint64_t* v[12];
  int64_t ld;
  int64_t n;
};

// The update steps below load every operand of an element before they
// compute and store: a store to one vector cannot then hold back a load from
// another (the compiler must assume they may alias), so the loads' latency
// overlaps instead of adding up along the element's chain of operations.

// GPBiCG, i >= 2, element i: w = v + beta q;  p = r + beta (p - u)
template <int W>
__device__ __forceinline__ void gp_wp_elem(int64_t i, const Num<W>& beta, const uint64_t* v,
                                           const uint64_t* q, const uint64_t* r, uint64_t* p,
                                           const uint64_t* u, uint64_t* w, int64_t ld) {
  Num<W> qi, vi, pi, ui, ri, a, b, c;
  load<W>(qi, q, ld, i);
  load<W>(vi, v, ld, i);
  load<W>(pi, p, ld, i);
  load<W>(ui, u, ld, i);
  load<W>(ri, r, ld, i);
  mul_rn_fast<W>(beta, qi, b);
  add_rn<W>(vi, b, c);
  store<W>(c, w, ld, i);
  sub_rn<W>(pi, ui, c);
  mul_rn_fast<W>(beta, c, a);
  add_rn<W>(ri, a, c);
  store<W>(c, p, ld, i);
}

// GPBiCG, i >= 2, element i: s = t - r;  t = r - alpha q;  y = s - alpha (w - q)
template <int W>
__device__ __forceinline__ void gp_sty_elem(int64_t i, const Num<W>& alpha, const uint64_t* r,
                                            const uint64_t* q, const uint64_t* w, uint64_t* s,
                                            uint64_t* t, uint64_t* y, int64_t ld) {
  Num<W> ti, ri, qi, wi, a, c, sv;
  load<W>(ti, t, ld, i);
  load<W>(ri, r, ld, i);
  load<W>(qi, q, ld, i);
  load<W>(wi, w, ld, i);
  sub_rn<W>(ti, ri, sv);
  store<W>(sv, s, ld, i);
  mul_rn_fast<W>(alpha, qi, c);
  sub_rn<W>(ri, c, a);
  store<W>(a, t, ld, i);
  sub_rn<W>(wi, qi, c);
  mul_rn_fast<W>(alpha, c, a);
  sub_rn<W>(sv, a, c);
  store<W>(c, y, ld, i);
}

// GPBiCG, element i: u = zeta q + eta (s + beta u);  z = zeta r + eta z - alpha u;
//                    x = x + alpha p + z;            r = t - eta y - zeta v
// V.v: 0 q, 1 s, 2 u, 3 r, 4 z, 5 p, 6 t, 7 y, 8 v
template <int W>
__device__ __forceinline__ void gp_uzxr_elem(int64_t i, const Num<W>& beta, const Num<W>& eta,
                                             const Num<W>& zeta, const Num<W>& alpha,
                                             const Vecs& V, uint64_t* x, int64_t ldx) {
  const int64_t ld = V.ld;
  Num<W> qi, si, ui, ri, zi, pi, xi, yi, ti, vi, a, b, c, un, zn;
  load<W>(ui, V.v[2], ld, i);
  load<W>(si, V.v[1], ld, i);
  load<W>(qi, V.v[0], ld, i);
  load<W>(ri, V.v[3], ld, i);
  load<W>(zi, V.v[4], ld, i);
  load<W>(pi, V.v[5], ld, i);
  load<W>(xi, x, ldx, i);
  load<W>(yi, V.v[7], ld, i);
  load<W>(ti, V.v[6], ld, i);
  load<W>(vi, V.v[8], ld, i);
  mul_rn_fast<W>(beta, ui, b);
  add_rn<W>(si, b, c);
  mul_rn_fast<W>(eta, c, b);
  mul_rn_fast<W>(zeta, qi, c);
  add_rn<W>(c, b, un);
  store<W>(un, V.v[2], ld, i);
  mul_rn_fast<W>(zeta, ri, b);  // zeta r
  mul_rn_fast<W>(eta, zi, c);   // eta z
  add_rn<W>(b, c, a);
  mul_rn_fast<W>(alpha, un, b);
  sub_rn<W>(a, b, zn);
  store<W>(zn, V.v[4], ld, i);
  mul_rn_fast<W>(alpha, pi, b);  // alpha p
  add_rn<W>(xi, b, c);
  add_rn<W>(c, zn, a);
  store<W>(a, x, ldx, i);
  mul_rn_fast<W>(eta, yi, b);  // eta y
  sub_rn<W>(ti, b, c);
  mul_rn_fast<W>(zeta, vi, b);  // zeta v
  sub_rn<W>(c, b, a);
  store<W>(a, V.v[3], ld, i);
}

}  // namespace mpk
