// solvers.cu -- device-resident BiCG and GPBiCG (Fig. 5, K = I), and CGS and
// BiCGSTAB (the other product-type methods of Section 4, textbook forms).
//
// Every step of an iteration is a kernel on the caller's stream: the SpMVs,
// the exact dot products (fused where they share operands; two kernels per
// group, dot.cuh), and fused vector updates that evaluate the figure's
// formulas with each product and sum rounded, left to right.  The scalar
// recurrences (alpha, zeta and eta, omega, the stopping rule and the next
// beta; p-bit divisions included) run on one thread at the end of the dot
// group whose results they take, in that group's finalize kernel, so no
// launch carries a scalar step alone.  A device state word ("done") gates
// every kernel: once a scalar step decides convergence, breakdown or the
// iteration limit, later launches return at once, so the host can run
// several iterations between polls and the result does not depend on the
// poll interval.  From the second iteration on, one iteration is captured
// once as a CUDA graph and replayed.
//
// Readings of Fig. 5 (shared with the oracle):
//  * GPBiCG uses z = zeta r + eta z - alpha u and r = t - eta y - zeta A t
//    (Zhang's method); the printed "zeta z" and "zeta u" break r = b - A x.
//  * At i = 1 the general u/z/x/r updates run with u = z = s = 0 and
//    beta = eta = +0; y = alpha q - r and zeta = mu2/mu5.
//  * A zero divisor of zeta/eta (mu5 at i = 1, tau later) gives
//    zeta = eta = +0; a zero (r~, q) or (p~, z) is a breakdown.
//  * The stopping rule (r,r) <= RN(RN(rtol^2)(r0,r0)) + RN(atol^2) is checked
//    once r_i is formed; GPBiCG then exits on zeta = 0.  Reaching maxit wins
//    over a zero rho found for the next iteration.
//  * BiCG: z~ = A^T p~ and p~_i = r~_{i-1} + beta p~_{i-1}.
#include <cmath>
#include <cstring>
#include <vector>

#include "dot.cuh"
#include "gpbicg.cuh"
#include "internal.h"
#include "mpdev.cuh"

// The file is compiled once per word count W = p/32 (MPK_W = 4, 8, 16, 32:
// the kernels and solve_entry<W>) and once with MPK_W = 0 (argument checks
// and the C entry points), so that the precisions build in parallel.
#ifndef MPK_W
#define MPK_W 0
#endif

namespace mpk {

struct SolveCall {
  mp_csr A;
  mp_vec b, x;
  mp_solve_opts o;
  cudaStream_t st;
  const mp_ilu_s* pre;  // ILU(0) preconditioner K (BiCGSTAB), or null
  int pre_left;         // 1: K applied on the left (Section 4.2), 0: on the right
  // BiCG: a second stream and two events, for A^T p~ beside A p
  cudaStream_t st2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

template <int W>
mp_status solve_entry(int method, const SolveCall& c, mp_solve_info* info);

}  // namespace mpk

#if MPK_W != 0
namespace mpk {
namespace {

struct SState {
  int done;    // gate for every kernel of the solve
  int status;  // MP_OK, MP_ERR_BREAKDOWN, MP_ERR_NOCONV, MP_ERR_TIMEOUT
  long long iters;
  long long maxit;
  cudaGraphConditionalHandle loop;  // the device-side iteration loop (has_loop)
  int has_loop;
  int pad;
  unsigned long long t0;        // device time (ns) at the set-up
  unsigned long long limit_ns;  // 0: no time limit
};

enum Scal {
  RHO, RHO_NEW, RHO_PREV, ALPHA, BETA, ZETA, ETA, DEN, MU1, MU2, MU3, MU4, MU5, RR, RR0, THR,
  OMEGA, TS, TT, NSCAL
};

// Solvers of the library (the template argument of the driver).
enum Method { kBiCG = 0, kGPBiCG = 1, kCGS = 2, kBiCGSTAB = 3 };

// Scalar slots are read through L2 (the post-steps below read slots that other
// blocks of the same kernel wrote).
template <int W>
__device__ __forceinline__ void ld_s(Num<W>& a, const uint64_t* S, int j) {
  const uint64_t* p = S + (size_t)j * (W / 2 + 1);
  unpack_head(__ldcg(p), a.e, a.s);
#pragma unroll
  for (int k = 0; k < W / 2; ++k) {
    const uint64_t l = __ldcg(p + 1 + k);
    a.m[2 * k] = (uint32_t)l;
    a.m[2 * k + 1] = (uint32_t)(l >> 32);
  }
}
template <int W>
__device__ __forceinline__ void st_s(const Num<W>& a, uint64_t* S, int j) {
  store<W>(a, S + (size_t)j * (W / 2 + 1), 1, 0);
}

// Ends the solve: every later kernel returns at once, and the device-side
// loop that replays the iteration stops after the current pass.
__device__ __forceinline__ void finish(SState* st, int status) {
  st->status = status;
  st->done = 1;
  if (st->has_loop) cudaGraphSetConditional(st->loop, 0u);
}


// ---------------------------------------------------------------------------
// Scalar steps.  Each runs on one thread right after the dot products it
// consumes: the last block of those dots' finalize kernel calls it (dot.cuh),
// so an iteration launches no scalar kernel of its own.
// ---------------------------------------------------------------------------

// thr = RN(RN(T*(r0,r0)) + A) with T = RN(rtol^2), A = RN(atol^2); exits
// before the first iteration when (r0,r0) <= thr or rho = 0.
template <int W>
__device__ void s_setup(SState* st, uint64_t* S, double rtol, double atol) {
  Num<W> rt, at, T, A, t, thr, rr0, rho, z;
  from_f64<W>(rtol, rt);
  from_f64<W>(atol, at);
  mul_rn_fast<W>(rt, rt, T);
  mul_rn_fast<W>(at, at, A);
  ld_s<W>(rr0, S, RR0);
  mul_rn_fast<W>(T, rr0, t);
  add_rn<W>(t, A, thr);
  st_s<W>(thr, S, THR);
  set_zero(z, 0u);
  st_s<W>(z, S, BETA);
  st_s<W>(z, S, ETA);
  st_s<W>(z, S, ZETA);
  ld_s<W>(rho, S, RHO);
  st->iters = 0;
  st->status = MP_OK;
  st->done = 0;
  st->t0 = device_ns();
  if (cmp<W>(rr0, thr) <= 0) {
    finish(st, MP_OK);
  } else if (st->maxit <= 0) {
    finish(st, MP_ERR_NOCONV);
  } else if (zero_e(rho.e)) {
    finish(st, MP_ERR_BREAKDOWN);
  }
}

// alpha = RN(rho / DEN); DEN = 0 is a breakdown.
template <int W>
__device__ void s_alpha(SState* st, uint64_t* S) {
  if (st->done) return;
  Num<W> rho, d, a;
  ld_s<W>(d, S, DEN);
  if (zero_e(d.e)) {
    finish(st, MP_ERR_BREAKDOWN);
    return;
  }
  ld_s<W>(rho, S, RHO);
  div_rn<W>(rho, d, a);
  st_s<W>(a, S, ALPHA);
}

// GPBiCG i = 1: zeta = mu2/mu5 (mu5 = 0 -> 0), eta = 0.
template <int W>
__device__ void s_zeta1(SState* st, uint64_t* S) {
  if (st->done) return;
  Num<W> m2, m5, z;
  ld_s<W>(m2, S, MU2);
  ld_s<W>(m5, S, MU5);
  if (zero_e(m5.e))
    set_zero(z, 0u);
  else
    div_rn<W>(m2, m5, z);
  st_s<W>(z, S, ZETA);
  set_zero(z, 0u);
  st_s<W>(z, S, ETA);
}

// tau = mu5 mu1 - mu4 mu4; zeta = (mu1 mu2 - mu3 mu4)/tau;
// eta = (mu5 mu3 - mu4 mu2)/tau; tau = 0 -> zeta = eta = 0.  Lanes 0-2 of
// the warp form tau and the two numerators at once (one code path, the
// operands chosen by lane), then lanes 1 and 2 divide; each value takes the
// same rounded operations as one thread computing them in turn.
template <int W>
__device__ void s_zeta(SState* st, uint64_t* S, int lane) {
  __shared__ Num<W> part[3];  // tau, zeta's numerator, eta's numerator
  if (st->done) return;
  if (lane < 3) {
    const int i1 = lane == 0 ? MU5 : (lane == 1 ? MU1 : MU5);
    const int j1 = lane == 0 ? MU1 : (lane == 1 ? MU2 : MU3);
    const int i2 = lane == 0 ? MU4 : (lane == 1 ? MU3 : MU4);
    const int j2 = lane == 0 ? MU4 : (lane == 1 ? MU4 : MU2);
    Num<W> x1, y1, x2, y2, a, b, c;
    ld_s<W>(x1, S, i1);
    ld_s<W>(y1, S, j1);
    ld_s<W>(x2, S, i2);
    ld_s<W>(y2, S, j2);
    mul_rn_fast<W>(x1, y1, a);
    mul_rn_fast<W>(x2, y2, b);
    sub_rn<W>(a, b, c);
    part[lane] = c;
  }
  __syncwarp();
  if (lane < 3) {
    const Num<W> tau = part[0];
    Num<W> z;
    if (zero_e(tau.e)) {
      if (lane == 0) {
        set_zero(z, 0u);
        st_s<W>(z, S, ZETA);
        st_s<W>(z, S, ETA);
      }
    } else if (lane > 0) {
      const Num<W> num = part[lane];
      div_rn<W>(num, tau, z);
      st_s<W>(z, S, lane == 1 ? ZETA : ETA);
    }
  }
}

// BiCGSTAB: omega = RN(TS / TT), +0 when TT = (t, t) = 0.
template <int W>
__device__ void s_omega(SState* st, uint64_t* S) {
  if (st->done) return;
  Num<W> ts, tt, om;
  ld_s<W>(tt, S, TT);
  if (zero_e(tt.e)) {
    set_zero(om, 0u);
  } else {
    ld_s<W>(ts, S, TS);
    div_rn<W>(ts, tt, om);
  }
  st_s<W>(om, S, OMEGA);
}

// End of an iteration: count it, record (r,r), shift rho, decide the exit.
// ZX: the scalar whose zero ends the iteration after the convergence test
// (GPBiCG's zeta, BiCGSTAB's omega), -1 none.  A time limit, when set, ends
// the solve (MP_ERR_TIMEOUT) once an iteration finishes past it.  When the
// solve goes on, the next iteration's beta = RN(rho_i/rho_{i-1}) (BiCG,
// CGS) or RN(RN(rho_i/rho_{i-1}) * RN(alpha/d)) with d = zeta (GPBiCG) or
// omega (BiCGSTAB) (BDIV names d's slot, -1 none) is formed here: its inputs
// are final at this point, and the next iteration then starts with its
// vector update.  Lanes 0 and 1 start beta's two divisions from the slots
// the check shifts into place (rho_i = RHO_NEW, rho_{i-1} = RHO) while lane 0
// decides the exit; beta is stored only when the solve goes on.
template <int W, int ZX, int BDIV>
__device__ void s_check(SState* st, uint64_t* S, uint64_t* hist, int64_t hist_ld,
                        int64_t hist_n, int lane) {
  __shared__ Num<W> q[2];
  if (st->done) return;
  if (lane == 0 || (lane == 1 && BDIV >= 0)) {
    Num<W> num, den, r;
    ld_s<W>(num, S, lane == 0 ? RHO_NEW : ALPHA);
    ld_s<W>(den, S, lane == 0 ? RHO : (BDIV >= 0 ? BDIV : RHO));
    if (zero_e(den.e))
      set_zero(r, 0u);  // the solve ends in this check (a zero rho or d): beta is not used
    else
      div_rn<W>(num, den, r);
    q[lane] = r;
  }
  __syncwarp();
  if (lane != 0) return;
  Num<W> rr, thr, rho, rn, z;
  st->iters += 1;
  ld_s<W>(rr, S, RR);
  if (hist && st->iters <= hist_n) store<W>(rr, hist, hist_ld, st->iters - 1);
  ld_s<W>(rho, S, RHO);
  ld_s<W>(rn, S, RHO_NEW);
  st_s<W>(rho, S, RHO_PREV);
  st_s<W>(rn, S, RHO);
  ld_s<W>(thr, S, THR);
  ld_s<W>(z, S, ZX >= 0 ? ZX : ZETA);
  if (cmp<W>(rr, thr) <= 0) {
    finish(st, MP_OK);
  } else if (ZX >= 0 && zero_e(z.e)) {
    finish(st, MP_ERR_BREAKDOWN);
  } else if (st->iters >= st->maxit) {
    finish(st, MP_ERR_NOCONV);
  } else if (zero_e(rn.e)) {
    finish(st, MP_ERR_BREAKDOWN);
  } else if (st->limit_ns != 0 && device_ns() - st->t0 > st->limit_ns) {
    finish(st, MP_ERR_TIMEOUT);
  } else if (BDIV >= 0) {
    Num<W> b;
    mul_rn_fast<W>(q[0], q[1], b);
    st_s<W>(b, S, BETA);
  } else {
    st_s<W>(q[0], S, BETA);
  }
}

// The steps as the dot finalize's post-step functors (called by the 32 lanes
// of one warp; the one-thread steps run on lane 0).
template <int W>
struct PostSetup {
  SState* st;
  uint64_t* S;
  double rtol, atol;
  __device__ void operator()(int lane) const {
    if (lane == 0) s_setup<W>(st, S, rtol, atol);
  }
};
template <int W>
struct PostAlpha {
  SState* st;
  uint64_t* S;
  __device__ void operator()(int lane) const {
    if (lane == 0) s_alpha<W>(st, S);
  }
};
template <int W, bool FIRST>
struct PostZeta {
  SState* st;
  uint64_t* S;
  __device__ void operator()(int lane) const {
    if (FIRST) {
      if (lane == 0) s_zeta1<W>(st, S);
    } else {
      s_zeta<W>(st, S, lane);
    }
  }
};
template <int W>
struct PostOmega {
  SState* st;
  uint64_t* S;
  __device__ void operator()(int lane) const {
    if (lane == 0) s_omega<W>(st, S);
  }
};
template <int W, int ZX, int BDIV>
struct PostCheck {
  SState* st;
  uint64_t* S;
  uint64_t* hist;
  int64_t hist_ld, hist_n;
  __device__ void operator()(int lane) const {
    s_check<W, ZX, BDIV>(st, S, hist, hist_ld, hist_n, lane);
  }
};

// ---------------------------------------------------------------------------
// Vector kernels (gated)
// ---------------------------------------------------------------------------


#define GRID_LOOP(i, n) \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

template <int W>
__global__ void set_zero_kernel(uint64_t* a, int64_t ld, int64_t n) {
  GRID_LOOP(i, n) {
    Num<W> z;
    set_zero(z, 0u);
    store<W>(z, a, ld, i);
  }
}

template <int W>
__global__ void copy_kernel(const SState* st, const uint64_t* __restrict__ src, int64_t lds,
                            uint64_t* __restrict__ dst, int64_t ldd, int64_t n) {
  pdl_begin();
  if (st && st->done) return;
  GRID_LOOP(i, n) {
    for (int k = 0; k <= W / 2; ++k) dst[k * ldd + i] = src[k * lds + i];
  }
}

template <int W>
__global__ void gp_wp(const SState* st, const uint64_t* __restrict__ S, const uint64_t* v,
                      const uint64_t* q, const uint64_t* r, uint64_t* p, const uint64_t* u,
                      uint64_t* w, int64_t ld, int64_t n) {
  pdl_begin();
  if (st->done) return;
  Num<W> beta;
  ld_s<W>(beta, S, BETA);
  GRID_LOOP(i, n) gp_wp_elem<W>(i, beta, v, q, r, p, u, w, ld);
}

// GPBiCG, i = 1: t = r - alpha q;  y = alpha q - r
template <int W>
__global__ void gp_ty1(const SState* st, const uint64_t* __restrict__ S, const uint64_t* r,
                       const uint64_t* q, uint64_t* t, uint64_t* y, int64_t ld, int64_t n) {
  pdl_begin();
  if (st->done) return;
  Num<W> alpha;
  ld_s<W>(alpha, S, ALPHA);
  GRID_LOOP(i, n) {
    Num<W> a, aq, c;
    load<W>(a, q, ld, i);
    mul_rn_fast<W>(alpha, a, aq);
    load<W>(a, r, ld, i);
    sub_rn<W>(a, aq, c);
    store<W>(c, t, ld, i);
    sub_rn<W>(aq, a, c);
    store<W>(c, y, ld, i);
  }
}

template <int W>
__global__ void gp_sty(const SState* st, const uint64_t* __restrict__ S, const uint64_t* r,
                       const uint64_t* q, const uint64_t* w, uint64_t* s, uint64_t* t,
                       uint64_t* y, int64_t ld, int64_t n) {
  pdl_begin();
  if (st->done) return;
  Num<W> alpha;
  ld_s<W>(alpha, S, ALPHA);
  GRID_LOOP(i, n) gp_sty_elem<W>(i, alpha, r, q, w, s, t, y, ld);
}

template <int W>
__global__ void gp_uzxr(const SState* st, const uint64_t* __restrict__ S, const Vecs V,
                        uint64_t* x, int64_t ldx) {
  pdl_begin();
  if (st->done) return;
  Num<W> beta, eta, zeta, alpha;
  ld_s<W>(beta, S, BETA);
  ld_s<W>(eta, S, ETA);
  ld_s<W>(zeta, S, ZETA);
  ld_s<W>(alpha, S, ALPHA);
  GRID_LOOP(i, V.n) gp_uzxr_elem<W>(i, beta, eta, zeta, alpha, V, x, ldx);
}

// BiCG, i >= 2: p = r + beta p;  p~ = r~ + beta p~
template <int W>
__global__ void bi_p(const SState* st, const uint64_t* __restrict__ S, const uint64_t* r,
                     const uint64_t* rt, uint64_t* p, uint64_t* pt, int64_t ld, int64_t n) {
  pdl_begin();
  if (st->done) return;
  GRID_LOOP(i, n) {
    Num<W> beta, pi, ri, pti, rti, b, c;
    ld_s<W>(beta, S, BETA);
    load<W>(pi, p, ld, i);
    load<W>(ri, r, ld, i);
    load<W>(pti, pt, ld, i);
    load<W>(rti, rt, ld, i);
    mul_rn_fast<W>(beta, pi, b);
    add_rn<W>(ri, b, c);
    store<W>(c, p, ld, i);
    mul_rn_fast<W>(beta, pti, b);
    add_rn<W>(rti, b, c);
    store<W>(c, pt, ld, i);
  }
}

// BiCG: x = x + alpha p;  r = r - alpha z;  r~ = r~ - alpha z~
template <int W>
__global__ void bi_xr(const SState* st, const uint64_t* __restrict__ S, const uint64_t* p,
                      const uint64_t* z, const uint64_t* zt, uint64_t* r, uint64_t* rt,
                      uint64_t* x, int64_t ldx, int64_t ld, int64_t n) {
  pdl_begin();
  if (st->done) return;
  GRID_LOOP(i, n) {
    Num<W> alpha, pi, xi, zi, ri, zti, rti, b, c;
    ld_s<W>(alpha, S, ALPHA);
    load<W>(pi, p, ld, i);
    load<W>(xi, x, ldx, i);
    load<W>(zi, z, ld, i);
    load<W>(ri, r, ld, i);
    load<W>(zti, zt, ld, i);
    load<W>(rti, rt, ld, i);
    mul_rn_fast<W>(alpha, pi, b);
    add_rn<W>(xi, b, c);
    store<W>(c, x, ldx, i);
    mul_rn_fast<W>(alpha, zi, b);
    sub_rn<W>(ri, b, c);
    store<W>(c, r, ld, i);
    mul_rn_fast<W>(alpha, zti, b);
    sub_rn<W>(rti, b, c);
    store<W>(c, rt, ld, i);
  }
}

// CGS, i >= 2: u = r + beta q;  p = u + beta (q + beta p)
template <int W>
__global__ void cgs_up(const SState* st, const uint64_t* __restrict__ S, const uint64_t* r,
                       const uint64_t* q, uint64_t* u, uint64_t* p, int64_t ld, int64_t n) {
  pdl_begin();
  if (st->done) return;
  GRID_LOOP(i, n) {
    Num<W> beta, qv, ri, pi, a, b, un;
    ld_s<W>(beta, S, BETA);
    load<W>(qv, q, ld, i);
    load<W>(ri, r, ld, i);
    load<W>(pi, p, ld, i);
    mul_rn_fast<W>(beta, qv, a);
    add_rn<W>(ri, a, un);
    store<W>(un, u, ld, i);
    mul_rn_fast<W>(beta, pi, b);
    add_rn<W>(qv, b, a);
    mul_rn_fast<W>(beta, a, b);
    add_rn<W>(un, b, a);
    store<W>(a, p, ld, i);
  }
}

// CGS: q = u - alpha v;  w = u + q;  x = x + alpha w
template <int W>
__global__ void cgs_qwx(const SState* st, const uint64_t* __restrict__ S, const uint64_t* u,
                        const uint64_t* v, uint64_t* q, uint64_t* w, uint64_t* x, int64_t ldx,
                        int64_t ld, int64_t n) {
  pdl_begin();
  if (st->done) return;
  GRID_LOOP(i, n) {
    Num<W> alpha, uv, vi, xi, b, qv, wv;
    ld_s<W>(alpha, S, ALPHA);
    load<W>(uv, u, ld, i);
    load<W>(vi, v, ld, i);
    load<W>(xi, x, ldx, i);
    mul_rn_fast<W>(alpha, vi, b);
    sub_rn<W>(uv, b, qv);
    store<W>(qv, q, ld, i);
    add_rn<W>(uv, qv, wv);
    store<W>(wv, w, ld, i);
    mul_rn_fast<W>(alpha, wv, b);
    add_rn<W>(xi, b, uv);
    store<W>(uv, x, ldx, i);
  }
}

// r = r - SCAL * a  (CGS: alpha A w)
template <int W, int SCAL>
__global__ void r_minus(const SState* st, const uint64_t* __restrict__ S, const uint64_t* a,
                        uint64_t* r, int64_t ld, int64_t n) {
  pdl_begin();
  if (st->done) return;
  GRID_LOOP(i, n) {
    Num<W> sc, av, b, rv, c;
    ld_s<W>(sc, S, SCAL);
    load<W>(av, a, ld, i);
    mul_rn_fast<W>(sc, av, b);
    load<W>(rv, r, ld, i);
    sub_rn<W>(rv, b, c);
    store<W>(c, r, ld, i);
  }
}

// BiCGSTAB, i >= 2: p = r + beta (p - omega v)
template <int W>
__global__ void bs_p(const SState* st, const uint64_t* __restrict__ S, const uint64_t* r,
                     const uint64_t* v, uint64_t* p, int64_t ld, int64_t n) {
  pdl_begin();
  if (st->done) return;
  GRID_LOOP(i, n) {
    Num<W> beta, omega, a, b, c;
    ld_s<W>(beta, S, BETA);
    ld_s<W>(omega, S, OMEGA);
    load<W>(a, v, ld, i);
    mul_rn_fast<W>(omega, a, b);
    load<W>(a, p, ld, i);
    sub_rn<W>(a, b, c);
    mul_rn_fast<W>(beta, c, a);
    load<W>(b, r, ld, i);
    add_rn<W>(b, a, c);
    store<W>(c, p, ld, i);
  }
}

// BiCGSTAB: s = r - alpha v
template <int W>
__global__ void bs_s(const SState* st, const uint64_t* __restrict__ S, const uint64_t* r,
                     const uint64_t* v, uint64_t* s, int64_t ld, int64_t n) {
  pdl_begin();
  if (st->done) return;
  GRID_LOOP(i, n) {
    Num<W> alpha, a, b, c;
    ld_s<W>(alpha, S, ALPHA);
    load<W>(a, v, ld, i);
    mul_rn_fast<W>(alpha, a, b);
    load<W>(a, r, ld, i);
    sub_rn<W>(a, b, c);
    store<W>(c, s, ld, i);
  }
}

// BiCGSTAB: x = x + alpha p + omega s;  r = s - omega t (with a right
// preconditioner, x takes p^ = M^{-1} p and s^ = M^{-1} s: px, sx)
template <int W>
__global__ void bs_xr(const SState* st, const uint64_t* __restrict__ S, const uint64_t* px,
                      const uint64_t* sx, const uint64_t* s, const uint64_t* t, uint64_t* r,
                      uint64_t* x, int64_t ldx, int64_t ld, int64_t n) {
  pdl_begin();
  if (st->done) return;
  GRID_LOOP(i, n) {
    Num<W> alpha, omega, pxi, xi, sxi, si, ti, a, b, c;
    ld_s<W>(alpha, S, ALPHA);
    ld_s<W>(omega, S, OMEGA);
    load<W>(pxi, px, ld, i);
    load<W>(xi, x, ldx, i);
    load<W>(sxi, sx, ld, i);
    load<W>(si, s, ld, i);
    load<W>(ti, t, ld, i);
    mul_rn_fast<W>(alpha, pxi, b);
    add_rn<W>(xi, b, c);
    mul_rn_fast<W>(omega, sxi, b);
    add_rn<W>(c, b, a);
    store<W>(a, x, ldx, i);
    mul_rn_fast<W>(omega, ti, b);
    sub_rn<W>(si, b, c);
    store<W>(c, r, ld, i);
  }
}

int ew_grid(int64_t n) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t b = (n + 127) / 128;
  const int64_t lim = (int64_t)(sms > 0 ? sms : 1) * 8;
  if (b > lim) b = lim;
  return (int)(b < 1 ? 1 : b);
}

// ---------------------------------------------------------------------------
// Host driver
// ---------------------------------------------------------------------------

struct Work {
  int prec = 0, L = 0;
  int64_t n = 0, ld = 0;
  uint64_t* vecs = nullptr;  // nvec vectors of (L+1)*ld words
  uint64_t* S = nullptr;     // NSCAL scalars of L+1 words
  SState* st = nullptr;
  int* status = nullptr;     // the device status word (span errors of the dots)
  void* dscratch = nullptr;
  int nvec = 0;
  uint64_t* vec(int k) const { return vecs + (size_t)k * (L + 1) * ld; }
  uint64_t* scal(int j) const { return S + (size_t)j * (L + 1); }
};

mp_status alloc_work(Work& w, int prec, int64_t n, int nvec, cudaStream_t st) {
  w.prec = prec;
  w.L = prec / 64;
  w.n = n;
  w.ld = n > 0 ? n : 1;
  w.nvec = nvec;
  const size_t vb = (size_t)nvec * (w.L + 1) * w.ld * 8;
  const size_t sb = (size_t)NSCAL * (w.L + 1) * 8;
  const size_t db = dot_scratch_bytes(prec, 5);
  w.status = status_word();
  if (!w.status) return set_error(MP_ERR_CUDA, "status word unavailable");
  // what was allocated before a failure is released by free_work
  cudaError_t e = work_malloc((void**)&w.vecs, vb, st);
  if (e == cudaSuccess) e = work_malloc((void**)&w.S, sb, st);
  if (e == cudaSuccess) e = work_malloc((void**)&w.st, sizeof(SState), st);
  if (e == cudaSuccess) e = work_malloc(&w.dscratch, db, st);
  if (e != cudaSuccess) return cuda_error(e, "solver work memory");
  return init_dot_scratch(w.dscratch, st);
}

void free_work(Work& w, cudaStream_t st) {
  cudaFreeAsync(w.vecs, st);
  cudaFreeAsync(w.S, st);
  cudaFreeAsync(w.st, st);
  cudaFreeAsync(w.dscratch, st);
  w = Work{};
}

// One or two dots (a0.b0 -> slot o0, a1.b1 -> slot o1) followed by `post`.
template <int W, class Post>
mp_status dot2(const Work& w, const uint64_t* a0, const uint64_t* b0, int o0, const uint64_t* a1,
               const uint64_t* b1, int o1, cudaStream_t st, const int* gate, Post post) {
  DotDev d{};
  d.k = a1 ? 2 : 1;
  d.n = w.n;
  d.x[0] = a0;
  d.y[0] = b0;
  d.x[1] = a1;
  d.y[1] = b1;
  for (int j = 0; j < 5; ++j) {
    d.ldx[j] = d.ldy[j] = w.ld;
    d.out_ld[j] = 1;
  }
  d.out[0] = w.scal(o0);
  d.out[1] = a1 ? w.scal(o1) : nullptr;
  return dot_launch<W, Post>(d, w.dscratch, dot_blocks<W>(w.n), w.status, gate, st, post);
}

// The end-of-iteration dots (r, r) and (r~, r) with the convergence check.
template <int W, int ZX, int BDIV>
mp_status check_dots(const Work& w, const SolveCall& c, uint64_t* r, uint64_t* rt, cudaStream_t st,
                     const int* gate) {
  const PostCheck<W, ZX, BDIV> post{w.st, w.S, c.o.history.data, c.o.history.ld,
                                    c.o.history.data ? c.o.history.n : 0};
  return dot2<W>(w, r, r, RR, rt, r, RHO_NEW, st, gate, post);
}

// The operator of the solve (A, or A^T for an adjoint solve) and its transpose.
const Sell& op_a(const SolveCall& c) { return c.o.transpose ? c.A->AT : c.A->A; }
const Sell& op_at(const SolveCall& c) { return c.o.transpose ? c.A->A : c.A->AT; }

// One iteration body for i >= 2 (captured into a graph) or i = 1.
template <int W>
mp_status gp_iteration(const Work& w, const SolveCall& c, bool first) {
  enum { R, RT, P, Q, T, V, WV, Y, U, Z, SV };
  const int64_t n = w.n, ld = w.ld;
  const int* gate = &w.st->done;
  cudaStream_t st = c.st;
  const int g = ew_grid(n);
  mp_status r;
  if (first) {
    launch_pdl(copy_kernel<W>, g, 128, 0, st, w.st, w.vec(R), ld, w.vec(P), ld, n);
    count_launch();
  } else {  // beta was formed by the previous iteration's check
    launch_pdl(gp_wp<W>, g, 128, 0, st, w.st, w.S, w.vec(V), w.vec(Q), w.vec(R), w.vec(P), w.vec(U),
                                w.vec(WV), ld, n);
    count_launch();
  }
  if ((r = launch_spmv(c.A, op_a(c),c.o.mode, w.vec(P), ld, w.vec(Q), ld, nullptr, 0, gate, st)) != MP_OK)
    return r;
  if ((r = dot2<W>(w, w.vec(RT), w.vec(Q), DEN, nullptr, nullptr, 0, st, gate,
                   PostAlpha<W>{w.st, w.S})) != MP_OK)
    return r;
  if (first) {
    launch_pdl(gp_ty1<W>, g, 128, 0, st, w.st, w.S, w.vec(R), w.vec(Q), w.vec(T), w.vec(Y), ld, n);
  } else {
    launch_pdl(gp_sty<W>, g, 128, 0, st, w.st, w.S, w.vec(R), w.vec(Q), w.vec(WV), w.vec(SV), w.vec(T),
                                 w.vec(Y), ld, n);
  }
  count_launch();
  if ((r = launch_spmv(c.A, op_a(c),c.o.mode, w.vec(T), ld, w.vec(V), ld, nullptr, 0, gate, st)) != MP_OK)
    return r;
  DotDev d{};
  d.n = n;
  for (int j = 0; j < 5; ++j) {
    d.ldx[j] = d.ldy[j] = ld;
    d.out_ld[j] = 1;
  }
  if (first) {
    d.k = 2;
    d.x[0] = w.vec(V); d.y[0] = w.vec(T); d.out[0] = w.scal(MU2);
    d.x[1] = w.vec(V); d.y[1] = w.vec(V); d.out[1] = w.scal(MU5);
  } else {
    d.k = 5;
    d.x[0] = w.vec(Y); d.y[0] = w.vec(Y); d.out[0] = w.scal(MU1);
    d.x[1] = w.vec(V); d.y[1] = w.vec(T); d.out[1] = w.scal(MU2);
    d.x[2] = w.vec(Y); d.y[2] = w.vec(T); d.out[2] = w.scal(MU3);
    d.x[3] = w.vec(V); d.y[3] = w.vec(Y); d.out[3] = w.scal(MU4);
    d.x[4] = w.vec(V); d.y[4] = w.vec(V); d.out[4] = w.scal(MU5);
  }
  r = first ? dot_launch<W>(d, w.dscratch, dot_blocks<W>(n), w.status, gate, st,
                            PostZeta<W, true>{w.st, w.S})
            : dot_launch<W>(d, w.dscratch, dot_blocks<W>(n), w.status, gate, st,
                            PostZeta<W, false>{w.st, w.S});
  if (r != MP_OK) return r;
  Vecs V9{};
  V9.v[0] = w.vec(Q); V9.v[1] = w.vec(SV); V9.v[2] = w.vec(U); V9.v[3] = w.vec(R);
  V9.v[4] = w.vec(Z); V9.v[5] = w.vec(P); V9.v[6] = w.vec(T); V9.v[7] = w.vec(Y);
  V9.v[8] = w.vec(V);
  V9.ld = ld;
  V9.n = n;
  launch_pdl(gp_uzxr<W>, g, 128, 0, st, w.st, w.S, V9, c.x.data, c.x.ld);
  count_launch();
  if ((r = check_dots<W, ZETA, ZETA>(w, c, w.vec(R), w.vec(RT), st, gate)) != MP_OK) return r;
  return launch_check("gpbicg iteration");
}

template <int W>
mp_status bi_iteration(const Work& w, const SolveCall& c, bool first) {
  enum { R, RT, P, PT, Z, ZT };
  const int64_t n = w.n, ld = w.ld;
  const int* gate = &w.st->done;
  cudaStream_t st = c.st;
  const int g = ew_grid(n);
  mp_status r;
  if (first) {
    launch_pdl(copy_kernel<W>, g, 128, 0, st, w.st, w.vec(R), ld, w.vec(P), ld, n);
    launch_pdl(copy_kernel<W>, g, 128, 0, st, w.st, w.vec(RT), ld, w.vec(PT), ld, n);
    count_launch(2);
  } else {  // beta was formed by the previous iteration's check
    launch_pdl(bi_p<W>, g, 128, 0, st, w.st, w.S, w.vec(R), w.vec(RT), w.vec(P), w.vec(PT), ld, n);
    count_launch();
  }
  // z~ = A^T p~ does not depend on z = A p: it runs on the second stream
  // (forked after the p update, joined before the x, r updates that use it),
  // beside z = A p and the (p~, z) dot and alpha on the first
  cudaError_t ce = cudaEventRecord(c.ev_fork, st);
  if (ce == cudaSuccess) ce = cudaStreamWaitEvent(c.st2, c.ev_fork, 0);
  if (ce != cudaSuccess) return cuda_error(ce, "forking A^T p~");
  if ((r = launch_spmv(c.A, op_at(c), c.o.mode, w.vec(PT), ld, w.vec(ZT), ld, nullptr, 0, gate,
                       c.st2)) != MP_OK)
    return r;
  if ((ce = cudaEventRecord(c.ev_join, c.st2)) != cudaSuccess) return cuda_error(ce, "joining A^T p~");
  if ((r = launch_spmv(c.A, op_a(c), c.o.mode, w.vec(P), ld, w.vec(Z), ld, nullptr, 0, gate, st)) != MP_OK)
    return r;
  if ((r = dot2<W>(w, w.vec(PT), w.vec(Z), DEN, nullptr, nullptr, 0, st, gate,
                   PostAlpha<W>{w.st, w.S})) != MP_OK)
    return r;
  if ((ce = cudaStreamWaitEvent(st, c.ev_join, 0)) != cudaSuccess)
    return cuda_error(ce, "joining A^T p~");
  launch_pdl(bi_xr<W>, g, 128, 0, st, w.st, w.S, w.vec(P), w.vec(Z), w.vec(ZT), w.vec(R), w.vec(RT),
                              c.x.data, c.x.ld, ld, n);
  count_launch();
  if ((r = check_dots<W, -1, -1>(w, c, w.vec(R), w.vec(RT), st, gate)) != MP_OK) return r;
  return launch_check("bicg iteration");
}

template <int W>
mp_status cgs_iteration(const Work& w, const SolveCall& c, bool first) {
  enum { R, RT, U, P, Q, V, WV, AW };
  const int64_t n = w.n, ld = w.ld;
  const int* gate = &w.st->done;
  cudaStream_t st = c.st;
  const int g = ew_grid(n);
  mp_status r;
  if (first) {
    launch_pdl(copy_kernel<W>, g, 128, 0, st, w.st, w.vec(R), ld, w.vec(U), ld, n);
    launch_pdl(copy_kernel<W>, g, 128, 0, st, w.st, w.vec(R), ld, w.vec(P), ld, n);
    count_launch(2);
  } else {  // beta was formed by the previous iteration's check
    launch_pdl(cgs_up<W>, g, 128, 0, st, w.st, w.S, w.vec(R), w.vec(Q), w.vec(U), w.vec(P), ld, n);
    count_launch();
  }
  if ((r = launch_spmv(c.A, op_a(c), c.o.mode, w.vec(P), ld, w.vec(V), ld, nullptr, 0, gate, st)) != MP_OK)
    return r;
  if ((r = dot2<W>(w, w.vec(RT), w.vec(V), DEN, nullptr, nullptr, 0, st, gate,
                   PostAlpha<W>{w.st, w.S})) != MP_OK)
    return r;
  launch_pdl(cgs_qwx<W>, g, 128, 0, st, w.st, w.S, w.vec(U), w.vec(V), w.vec(Q), w.vec(WV), c.x.data,
                                c.x.ld, ld, n);
  count_launch();
  if ((r = launch_spmv(c.A, op_a(c), c.o.mode, w.vec(WV), ld, w.vec(AW), ld, nullptr, 0, gate, st)) != MP_OK)
    return r;
  launch_pdl(r_minus<W, ALPHA>, g, 128, 0, st, w.st, w.S, w.vec(AW), w.vec(R), ld, n);
  count_launch();
  if ((r = check_dots<W, -1, -1>(w, c, w.vec(R), w.vec(RT), st, gate)) != MP_OK) return r;
  return launch_check("cgs iteration");
}

template <int W>
mp_status bicgstab_iteration(const Work& w, const SolveCall& c, bool first) {
  enum { R, RT, P, V, SV, T, PH, SH };
  const int64_t n = w.n, ld = w.ld;
  const int* gate = &w.st->done;
  cudaStream_t st = c.st;
  const int g = ew_grid(n);
  mp_status r;
  if (first) {
    launch_pdl(copy_kernel<W>, g, 128, 0, st, w.st, w.vec(R), ld, w.vec(P), ld, n);
    count_launch();
  } else {  // beta was formed by the previous iteration's check
    launch_pdl(bs_p<W>, g, 128, 0, st, w.st, w.S, w.vec(R), w.vec(V), w.vec(P), ld, n);
    count_launch();
  }
  // right preconditioning: v = A K^{-1} p, t = A K^{-1} s (x takes K^{-1} p
  // and K^{-1} s); left: v = K^{-1} A p, t = K^{-1} A s (PH and SH hold A p
  // and A s), and r is the preconditioned residual K^{-1}(b - A x)
  const bool left = c.pre && c.pre_left;
  const uint64_t* pv = w.vec(P);
  if (c.pre && !left) {
    if ((r = launch_ilu0_apply(c.pre, w.vec(P), ld, w.vec(PH), ld, gate, st)) != MP_OK) return r;
    pv = w.vec(PH);
  }
  if ((r = launch_spmv(c.A, op_a(c), c.o.mode, pv, ld, left ? w.vec(PH) : w.vec(V), ld, nullptr,
                       0, gate, st)) != MP_OK)
    return r;
  if (left && (r = launch_ilu0_apply(c.pre, w.vec(PH), ld, w.vec(V), ld, gate, st)) != MP_OK)
    return r;
  if ((r = dot2<W>(w, w.vec(RT), w.vec(V), DEN, nullptr, nullptr, 0, st, gate,
                   PostAlpha<W>{w.st, w.S})) != MP_OK)
    return r;
  launch_pdl(bs_s<W>, g, 128, 0, st, w.st, w.S, w.vec(R), w.vec(V), w.vec(SV), ld, n);
  count_launch();
  const uint64_t* sv = w.vec(SV);
  if (c.pre && !left) {
    if ((r = launch_ilu0_apply(c.pre, w.vec(SV), ld, w.vec(SH), ld, gate, st)) != MP_OK) return r;
    sv = w.vec(SH);
  }
  if ((r = launch_spmv(c.A, op_a(c), c.o.mode, sv, ld, left ? w.vec(SH) : w.vec(T), ld, nullptr,
                       0, gate, st)) != MP_OK)
    return r;
  if (left && (r = launch_ilu0_apply(c.pre, w.vec(SH), ld, w.vec(T), ld, gate, st)) != MP_OK)
    return r;
  if ((r = dot2<W>(w, w.vec(T), w.vec(SV), TS, w.vec(T), w.vec(T), TT, st, gate,
                   PostOmega<W>{w.st, w.S})) != MP_OK)
    return r;
  launch_pdl(bs_xr<W>, g, 128, 0, st, w.st, w.S, pv, sv, w.vec(SV), w.vec(T), w.vec(R), c.x.data,
                              c.x.ld, ld, n);
  count_launch();
  if ((r = check_dots<W, OMEGA, OMEGA>(w, c, w.vec(R), w.vec(RT), st, gate)) != MP_OK) return r;
  return launch_check("bicgstab iteration");
}

template <int W, int M>
mp_status solve_w(const SolveCall& cu, mp_solve_info* info) {
  // The solve runs on a private non-blocking stream fenced to the caller's
  // stream by events (the legacy default stream cannot be captured).
  cudaStream_t st = nullptr;
  cudaEvent_t fence = nullptr;
  mp_status r = private_stream_open(cu.st, &st, &fence);
  if (r != MP_OK) return r;
  SolveCall c = cu;
  c.st = st;
  const int64_t n = c.A->n;
  if (M == kBiCG) {
    cudaError_t ces = cudaStreamCreateWithFlags(&c.st2, cudaStreamNonBlocking);
    if (ces == cudaSuccess) ces = cudaEventCreateWithFlags(&c.ev_fork, cudaEventDisableTiming);
    if (ces == cudaSuccess) ces = cudaEventCreateWithFlags(&c.ev_join, cudaEventDisableTiming);
    if (ces != cudaSuccess) {
      if (c.ev_fork) cudaEventDestroy(c.ev_fork);
      if (c.st2) cudaStreamDestroy(c.st2);
      private_stream_close(cu.st, st, fence);
      return cuda_error(ces, "solver stream set-up");
    }
  }
  Work w;
  const int kVecs = M == kGPBiCG ? 11 : (M == kCGS || c.pre ? 8 : 6);
  r = alloc_work(w, c.A->prec, n, kVecs, st);
  if (r != MP_OK) {  // the work space, the streams and events go before returning
    free_work(w, st);
    if (c.st2) {
      cudaEventDestroy(c.ev_fork);
      cudaEventDestroy(c.ev_join);
      cudaStreamDestroy(c.st2);
    }
    private_stream_close(cu.st, st, fence);
    return r;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, st);
  SState init{};
  init.done = 1;
  init.status = MP_OK;
  init.maxit = c.o.maxit;
  init.limit_ns = (unsigned long long)c.o.time_limit_ms * 1000000ull;
  const int64_t ld = w.ld;
  const int g = ew_grid(n);
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  SState hs{};
  auto body = [&](bool first) {
    switch (M) {
      case kGPBiCG: return gp_iteration<W>(w, c, first);
      case kCGS: return cgs_iteration<W>(w, c, first);
      case kBiCGSTAB: return bicgstab_iteration<W>(w, c, first);
      default: return bi_iteration<W>(w, c, first);
    }
  };
  do {
    cudaError_t ce0 = cudaMemcpyAsync(w.st, &init, sizeof init, cudaMemcpyHostToDevice, st);
    if (ce0 != cudaSuccess) { r = cuda_error(ce0, "state upload"); break; }
    for (int k = 0; k < w.nvec; ++k) {
      set_zero_kernel<W><<<g, 128, 0, st>>>(w.vec(k), ld, n);
      count_launch();
    }
    // r0 = b - A x0 (exact residual), r~ = r0, (r0, r0) and rho_0 = (r~, r0);
    // with a left preconditioner r0 = K^{-1}(b - A x0), the residual formed
    // in the last work vector first
    const bool left = c.pre && c.pre_left;
    uint64_t* r0 = left ? w.vec(w.nvec - 1) : w.vec(0);
    if ((r = launch_spmv(c.A, op_a(c), MP_EXACT, c.x.data, c.x.ld, r0, ld, c.b.data, c.b.ld,
                         nullptr, st)) != MP_OK)
      break;
    if (left && (r = launch_ilu0_apply(c.pre, r0, ld, w.vec(0), ld, nullptr, st)) != MP_OK) break;
    launch_pdl(copy_kernel<W>, g, 128, 0, st, nullptr, w.vec(0), ld, w.vec(1), ld, n);
    count_launch();
    if ((r = dot2<W>(w, w.vec(0), w.vec(0), RR0, w.vec(1), w.vec(0), RHO, st, nullptr,
                     PostSetup<W>{w.st, w.S, c.o.rtol, c.o.atol})) != MP_OK)
      break;
    if ((r = launch_check("solver setup")) != MP_OK) break;
    // first iteration (not captured)
    if ((r = body(true)) != MP_OK) break;
    cudaError_t cer = injected_fault("solver poll");
    if (cer == cudaSuccess) cer = cudaMemcpyAsync(&hs, w.st, sizeof hs, cudaMemcpyDeviceToHost, st);
    if (cer == cudaSuccess) cer = cudaStreamSynchronize(st);
    if (cer != cudaSuccess) { r = cuda_error(cer, "reading the solver state"); break; }
    if (hs.done) break;
    // The remaining iterations run on the device in one graph launch: a
    // conditional while node whose body is one captured iteration.  finish()
    // clears the loop's condition wherever the solve ends (the stopping rule,
    // a breakdown, maxit, the time limit), so no host poll is needed.
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
    if (ce != cudaSuccess) { r = cuda_error(ce, "building the iteration loop"); break; }
    cudaGraph_t bodyg = cp.conditional.phGraph_out[0];
    const int one = 1;
    ce = cudaMemcpyAsync(&w.st->loop, &loop, sizeof loop, cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(&w.st->has_loop, &one, sizeof one, cudaMemcpyHostToDevice, st);
    if (ce != cudaSuccess) { r = cuda_error(ce, "loop handle upload"); break; }
    ce = cudaStreamBeginCaptureToGraph(st, bodyg, nullptr, nullptr, 0,
                                       cudaStreamCaptureModeRelaxed);
    if (ce != cudaSuccess) { r = cuda_error(ce, "cudaStreamBeginCaptureToGraph"); break; }
    const int64_t before = mp_launch_count(0);
    mp_status rb = body(false);
    const int64_t per_iter = mp_launch_count(0) - before;
    count_launch(-(int)per_iter);  // the capture itself launched nothing
    ce = cudaStreamEndCapture(st, &bodyg);
    if (rb != MP_OK) { r = rb; break; }
    if (ce != cudaSuccess) { r = cuda_error(ce, "cudaStreamEndCapture"); break; }
    ce = cudaGraphInstantiate(&exec, graph, 0);
    if (ce != cudaSuccess) { r = cuda_error(ce, "cudaGraphInstantiate"); break; }
    const long long it0 = hs.iters;
    ce = cudaGraphLaunch(exec, st);
    if (ce != cudaSuccess) { r = cuda_error(ce, "cudaGraphLaunch"); break; }
    ce = injected_fault("solver poll");
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&hs, w.st, sizeof hs, cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) { r = cuda_error(ce, "reading the solver state"); break; }
    count_launch((int)(per_iter * (hs.iters - it0)));
  } while (false);
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  cudaEventRecord(e1, st);
  if (r == MP_OK) {
    cudaError_t ce = cudaMemcpyAsync(&hs, w.st, sizeof hs, cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) r = cuda_error(ce, "reading the solver state");
  }
  if (info) {
    memset(info, 0, sizeof *info);
    float ms = 0.f;
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    info->ms = ms;
    info->iters = hs.iters;
    info->status = hs.status;
    double h[2] = {0, 0};
    // relres from (r,r) and (r0,r0): converted on the device, read back.
    double* dd = nullptr;
    if (r == MP_OK && cudaMallocAsync((void**)&dd, 2 * sizeof(double), st) == cudaSuccess) {
      mp_vec v1{1, c.A->prec, 1, w.scal(RR)}, v2{1, c.A->prec, 1, w.scal(RR0)};
      if (hs.iters == 0) v1 = v2;
      mp_vec_to_f64(v1, dd, st);
      mp_vec_to_f64(v2, dd + 1, st);
      cudaMemcpyAsync(h, dd, sizeof h, cudaMemcpyDeviceToHost, st);
      cudaFreeAsync(dd, st);
      cudaStreamSynchronize(st);
      info->relres = (h[1] > 0) ? sqrt(h[0] / h[1]) : 0.0;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  free_work(w, st);
  if (c.st2) {
    cudaStreamSynchronize(c.st2);
    cudaEventDestroy(c.ev_fork);
    cudaEventDestroy(c.ev_join);
    cudaStreamDestroy(c.st2);
  }
  private_stream_close(cu.st, st, fence);
  if (r != MP_OK) return r;
  return static_cast<mp_status>(hs.status);
}

}  // namespace

template <int W>
mp_status solve_entry(int method, const SolveCall& c, mp_solve_info* info) {
  switch (method) {
    case kGPBiCG: return solve_w<W, kGPBiCG>(c, info);
    case kCGS: return solve_w<W, kCGS>(c, info);
    case kBiCGSTAB: return solve_w<W, kBiCGSTAB>(c, info);
    default: return solve_w<W, kBiCG>(c, info);
  }
}
template mp_status solve_entry<MPK_W>(int, const SolveCall&, mp_solve_info*);

}  // namespace mpk

#else  // MPK_W == 0

namespace mpk {
namespace {

mp_status solve(int method, mp_csr A, mp_vec b, mp_vec x, const mp_solve_opts* opts,
                mp_solve_info* info, void* stream, const mp_ilu_s* pre = nullptr,
                int pre_left = 1) {
  if (!A) return set_error(MP_ERR_ARG, "matrix is null");
  if (!opts) return set_error(MP_ERR_ARG, "opts is null");
  mp_status r;
  if ((r = check_vec(b, A->n, A->prec, "b")) != MP_OK) return r;
  if ((r = check_vec(x, A->n, A->prec, "x")) != MP_OK) return r;
  if (A->n > 0 && b.data == x.data) return set_error(MP_ERR_ARG, "b and x must not alias");
  if (!(opts->rtol >= 0) || !(opts->atol >= 0) || !isfinite(opts->rtol) || !isfinite(opts->atol))
    return set_error(MP_ERR_ARG, "rtol/atol must be finite and >= 0");
  if (opts->maxit < 0) return set_error(MP_ERR_ARG, "maxit < 0");
  if (opts->mode != MP_ORDERED && opts->mode != MP_EXACT)
    return set_error(MP_ERR_ARG, "mode %d", opts->mode);
  if (opts->history.data) {
    if ((r = check_vec(opts->history, opts->history.n, A->prec, "history")) != MP_OK) return r;
  }
  if (method == 0 && !A->has_t) return set_error(MP_ERR_ARG, "BiCG needs MP_CSR_TRANSPOSE");
  if (opts->transpose != 0 && opts->transpose != 1)
    return set_error(MP_ERR_ARG, "transpose must be 0 or 1");
  if (opts->transpose && !A->has_t)
    return set_error(MP_ERR_ARG, "a solve with A^T needs MP_CSR_TRANSPOSE");
  if (opts->time_limit_ms < 0) return set_error(MP_ERR_ARG, "time_limit_ms < 0");
  if (!status_word()) return set_error(MP_ERR_CUDA, "status word unavailable");
  if (pre && (pre->n != A->n || pre->prec != A->prec || opts->transpose))
    return set_error(MP_ERR_ARG, "preconditioner does not match the matrix (or a transposed solve)");
  if (prec_big(A->prec)) {
    if (opts->time_limit_ms != 0)
      return set_error(MP_ERR_ARG, "time_limit_ms: only the solvers at p <= 1024 take a limit");
    return solve_big(method, A, b, x, opts, info, static_cast<cudaStream_t>(stream), pre,
                     pre_left);
  }
  SolveCall c{A, b, x, *opts, static_cast<cudaStream_t>(stream), pre, pre_left};
  return dispatch_w(A->prec, [&](auto w) {
    constexpr int W = decltype(w)::value;
    return solve_entry<W>(method, c, info);
  });
}

}  // namespace
}  // namespace mpk

extern "C" {

mp_status mp_bicg(mp_csr A, mp_vec b, mp_vec x, const mp_solve_opts* opts, mp_solve_info* info,
                  void* stream) {
  return mpk::solve(0, A, b, x, opts, info, stream);
}

mp_status mp_gpbicg(mp_csr A, mp_vec b, mp_vec x, const mp_solve_opts* opts, mp_solve_info* info,
                    void* stream) {
  return mpk::solve(1, A, b, x, opts, info, stream);
}

mp_status mp_cgs(mp_csr A, mp_vec b, mp_vec x, const mp_solve_opts* opts, mp_solve_info* info,
                 void* stream) {
  return mpk::solve(2, A, b, x, opts, info, stream);
}

mp_status mp_bicgstab(mp_csr A, mp_vec b, mp_vec x, const mp_solve_opts* opts,
                      mp_solve_info* info, void* stream) {
  return mpk::solve(3, A, b, x, opts, info, stream);
}

mp_status mp_bicgstab_ilu0(mp_csr A, mp_ilu M, mp_vec b, mp_vec x, const mp_solve_opts* opts,
                           mp_solve_info* info, void* stream) {
  if (!M) return mpk::set_error(MP_ERR_ARG, "preconditioner is null");
  return mpk::solve(3, A, b, x, opts, info, stream, M, 1);
}

mp_status mp_bicgstab_ilu0_right(mp_csr A, mp_ilu M, mp_vec b, mp_vec x,
                                 const mp_solve_opts* opts, mp_solve_info* info, void* stream) {
  if (!M) return mpk::set_error(MP_ERR_ARG, "preconditioner is null");
  return mpk::solve(3, A, b, x, opts, info, stream, M, 0);
}

}  // extern "C"

#endif  // MPK_W
