// refine.cu -- mixed-precision iterative refinement of A x = b (not in the
// paper): the p-bit solve of Section 4 with the inner work moved to FP64.
//
// Outer step (p bits):  r = RN_row(b - A x), each row one exact sum rounded
// once (the EXACT residual kernel).  E = the largest exponent of r; the
// FP64 right-hand side is rhat_i = 2^-E_i * double(r_i * 2^-E), where 2^-E_i
// equilibrates row i of the FP64 copy of A (E_i = the largest exponent in
// row i; powers of two, so the scaling itself is exact).
// Inner step (FP64):    GPBiCG on (D A) d = D rhat with FP64 CSR kernels on
// the same sliced layout as the p-bit matrix (D A is what the FP64 copy
// stores), stopped at a relative residual inner_rtol.
// Update (p bits):      x_i = RN(x_i + 2^E d_i)  (d_i converted exactly).
// The loop stops when max|2^E d| <= rtol * max|x| (the correction no longer
// changes x at the requested relative level) or after max_outer steps.
// FP64 appears only in the inner solve and its inner products; FP64 dot
// products sum per-block partials in a fixed order, so runs are repeatable.
#include <climits>
#include <cmath>
#include <cstring>

#include "internal.h"
#include "mpdev.cuh"

namespace mpk {
namespace {

constexpr int kT = 128;

struct SellV {
  int64_t nchunks, nslots;
  const int64_t* __restrict__ chunk_off;
  const int32_t* __restrict__ row_of;
  const int32_t* __restrict__ row_len;
  const int32_t* __restrict__ col;
};

SellV sview(const Sell& S) {
  return SellV{S.nchunks, S.nslots, S.chunk_off, S.row_of, S.row_len, S.col};
}

#define ROW_PROLOGUE                                                         \
  const int lane = threadIdx.x & 31;                                         \
  const int64_t chunk = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; \
  if (chunk >= S.nchunks) return;                                            \
  const int64_t slot = chunk * 32 + lane;                                    \
  const int32_t row = S.row_of[slot];                                        \
  if (row < 0) return;                                                       \
  const int32_t len = S.row_len[slot];                                       \
  const int64_t base = S.chunk_off[chunk] + lane;

// FP64 copy of A: a64[k] = double(2^-E_i a_k), rowscale[i] = 2^-E_i.
template <int W>
__global__ void build_f64_kernel(const SellV S, const uint64_t* __restrict__ val,
                                 double* __restrict__ a64, double* __restrict__ rowscale,
                                 int equilibrate) {
  ROW_PROLOGUE
  int64_t E = 0;
  if (equilibrate) {
    int64_t mx = LLONG_MIN;
    for (int32_t j = 0; j < len; ++j) {
      int64_t e;
      uint32_t s;
      unpack_head(val[base + (int64_t)j * 32], e, s);
      if (!zero_e(e)) mx = max(mx, e);
    }
    if (mx != LLONG_MIN) E = mx < -1000 ? -1000 : (mx > 1000 ? 1000 : mx);
  }
  rowscale[row] = ldexp(1.0, (int)-E);
  for (int32_t j = 0; j < len; ++j) {
    const int64_t k = base + (int64_t)j * 32;
    Num<W> a;
    load<W>(a, val, S.nslots, k);
    if (!zero_e(a.e)) a.e -= E;
    a64[k] = to_f64<W>(a);
  }
}

__global__ void spmv64_kernel(const SellV S, const double* __restrict__ a64,
                              const double* __restrict__ x, double* __restrict__ y,
                              const int* __restrict__ gate) {
  if (gate && *gate) return;
  ROW_PROLOGUE
  double acc = 0.0;
  for (int32_t j = 0; j < len; ++j) {
    const int64_t k = base + (int64_t)j * 32;
    acc = fma(a64[k], x[S.col[k]], acc);
  }
  y[row] = acc;
}

// y = D x (row scaling of a right-hand side)
__global__ void scale64_kernel(const double* __restrict__ d, const double* __restrict__ x,
                               double* __restrict__ y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = d[i] * x[i];
}

// ---- deterministic FP64 dot products (k <= 5 pairs) -----------------------

struct Dot64 {
  int k;
  int64_t n;
  const double* x[5];
  const double* y[5];
  double* out[5];
};

constexpr int kDotBlocks = 256;

__global__ void __launch_bounds__(256) dot64_partial_kernel(const Dot64 a, double* partial,
                                                            const int* gate) {
  __shared__ double red[256];
  if (gate && *gate) return;
  for (int j = 0; j < a.k; ++j) {
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n;
         i += (int64_t)gridDim.x * blockDim.x)
      s = fma(a.x[j][i], a.y[j][i], s);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) partial[j * kDotBlocks + blockIdx.x] = red[0];
    __syncthreads();
  }
}

__global__ void dot64_final_kernel(const Dot64 a, const double* partial, const int* gate) {
  if (gate && *gate) return;
  const int j = threadIdx.x;
  if (j >= a.k) return;
  double s = 0.0;
  for (int b = 0; b < kDotBlocks; ++b) s += partial[j * kDotBlocks + b];
  *a.out[j] = s;
}

// ---- FP64 GPBiCG (Zhang's method, the same reading as the p-bit solver) ---

struct St64 {
  int done, status;
  long long iters, maxit;
};

enum S64 { RHO, RHO_NEW, RHO_PREV, ALPHA, BETA, ZETA, ETA, DEN, MU1, MU2, MU3, MU4, MU5, RR, RR0, THR,
           NS64 };

__global__ void g64_setup(St64* st, double* S, double rtol) {
  S[THR] = rtol * rtol * S[RR0];
  S[BETA] = S[ETA] = S[ZETA] = 0.0;
  st->iters = 0;
  st->status = MP_OK;
  st->done = 0;
  if (S[RR0] <= S[THR])
    st->done = 1;
  else if (st->maxit <= 0) {
    st->status = MP_ERR_NOCONV;
    st->done = 1;
  } else if (S[RHO] == 0.0) {
    st->status = MP_ERR_BREAKDOWN;
    st->done = 1;
  }
}

__global__ void g64_alpha(St64* st, double* S) {
  if (st->done) return;
  if (S[DEN] == 0.0) {
    st->status = MP_ERR_BREAKDOWN;
    st->done = 1;
    return;
  }
  S[ALPHA] = S[RHO] / S[DEN];
}

__global__ void g64_zeta(St64* st, double* S, int first) {
  if (st->done) return;
  if (first) {
    S[ZETA] = S[MU5] != 0.0 ? S[MU2] / S[MU5] : 0.0;
    S[ETA] = 0.0;
    return;
  }
  const double tau = S[MU5] * S[MU1] - S[MU4] * S[MU4];
  if (tau == 0.0) {
    S[ZETA] = S[ETA] = 0.0;
    return;
  }
  S[ZETA] = (S[MU1] * S[MU2] - S[MU3] * S[MU4]) / tau;
  S[ETA] = (S[MU5] * S[MU3] - S[MU4] * S[MU2]) / tau;
}

__global__ void g64_beta(St64* st, double* S) {
  if (st->done) return;
  S[BETA] = (S[RHO] / S[RHO_PREV]) * (S[ALPHA] / S[ZETA]);
}

__global__ void g64_check(St64* st, double* S) {
  if (st->done) return;
  st->iters += 1;
  S[RHO_PREV] = S[RHO];
  S[RHO] = S[RHO_NEW];
  if (S[RR] <= S[THR]) {
    st->done = 1;
  } else if (S[ZETA] == 0.0) {
    st->status = MP_ERR_BREAKDOWN;
    st->done = 1;
  } else if (st->iters >= st->maxit) {
    st->status = MP_ERR_NOCONV;
    st->done = 1;
  } else if (S[RHO] == 0.0) {
    st->status = MP_ERR_BREAKDOWN;
    st->done = 1;
  }
}

#define GATED_LOOP(i, n)      \
  if (st->done) return;       \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// i >= 2: w = v + beta q; p = r + beta (p - u)
__global__ void g64_wp(const St64* st, const double* S, const double* v, const double* q,
                       const double* r, double* p, const double* u, double* w, int64_t n) {
  const double beta = S[BETA];
  GATED_LOOP(i, n) {
    w[i] = v[i] + beta * q[i];
    p[i] = r[i] + beta * (p[i] - u[i]);
  }
}

// i = 1: t = r - alpha q; y = alpha q - r.  i >= 2 also s = t - r and
// y = s - alpha (w - q).
__global__ void g64_sty(const St64* st, const double* S, const double* r, const double* q,
                        const double* w, double* s, double* t, double* y, int64_t n, int first) {
  const double alpha = S[ALPHA];
  GATED_LOOP(i, n) {
    if (first) {
      t[i] = r[i] - alpha * q[i];
      y[i] = alpha * q[i] - r[i];
    } else {
      const double sv = t[i] - r[i];
      s[i] = sv;
      t[i] = r[i] - alpha * q[i];
      y[i] = sv - alpha * (w[i] - q[i]);
    }
  }
}

// u = zeta q + eta (s + beta u); z = zeta r + eta z - alpha u;
// x = x + alpha p + z; r = t - eta y - zeta v
__global__ void g64_uzxr(const St64* st, const double* S, const double* q, const double* s,
                         double* u, double* r, double* z, const double* p, const double* t,
                         const double* y, const double* v, double* x, int64_t n) {
  const double alpha = S[ALPHA], beta = S[BETA], zeta = S[ZETA], eta = S[ETA];
  GATED_LOOP(i, n) {
    const double un = zeta * q[i] + eta * (s[i] + beta * u[i]);
    u[i] = un;
    const double zn = zeta * r[i] + eta * z[i] - alpha * un;
    z[i] = zn;
    x[i] = x[i] + alpha * p[i] + zn;
    r[i] = t[i] - eta * y[i] - zeta * v[i];
  }
}

__global__ void fill64_kernel(double* a, int64_t n, double v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    a[i] = v;
}

__global__ void copy64_kernel(const double* a, double* b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = a[i];
}

// ---- p-bit <-> FP64 glue ----------------------------------------------------

template <int W>
__global__ void max_exp_kernel(const uint64_t* __restrict__ r, int64_t n, long long* emax) {
  long long m = LLONG_MIN;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t e;
    uint32_t s;
    unpack_head(r[i], e, s);
    if (!zero_e(e)) m = max(m, (long long)e);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m != LLONG_MIN) atomicMax(emax, m);
}

// rhat_i = rowscale_i * double(r_i 2^-E)
template <int W>
__global__ void rhs_to_f64_kernel(const uint64_t* __restrict__ r, int64_t ldr, int64_t n,
                                  const long long* emax, const double* __restrict__ rowscale,
                                  double* __restrict__ rhat) {
  const long long E = *emax;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    Num<W> v;
    load<W>(v, r, ldr, i);
    if (!zero_e(v.e)) v.e -= E;
    rhat[i] = rowscale[i] * to_f64<W>(v);
  }
}

// x_i = RN(x_i + 2^E d_i); records max|2^-Ecorr| stats as doubles (bits of
// nonnegative doubles order like integers).
template <int W>
__global__ void correct_kernel(uint64_t* __restrict__ x, int64_t ldx, int64_t n,
                               const double* __restrict__ d, const long long* emax,
                               unsigned long long* dmax_bits, unsigned long long* xmax_bits) {
  const long long E = *emax;
  unsigned long long dm = 0, xm = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    Num<W> c, xv, s;
    from_f64<W>(d[i], c);
    if (!zero_e(c.e)) c.e += E;
    load<W>(xv, x, ldx, i);
    add_rn<W>(xv, c, s);
    store<W>(s, x, ldx, i);
    const double ca = fabs(to_f64<W>(c)), xa = fabs(to_f64<W>(s));
    dm = max(dm, (unsigned long long)__double_as_longlong(ca));
    xm = max(xm, (unsigned long long)__double_as_longlong(xa));
  }
  atomicMax(dmax_bits, dm);
  atomicMax(xmax_bits, xm);
}

__global__ void reset_words(long long* emax, unsigned long long* a, unsigned long long* b) {
  *emax = LLONG_MIN;
  *a = 0;
  *b = 0;
}

int grid_n(int64_t n) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t b = (n + 255) / 256;
  const int64_t lim = (int64_t)(sms > 0 ? sms : 1) * 8;
  return (int)(b < 1 ? 1 : (b > lim ? lim : b));
}

// ---- the FP64 inner solver ----------------------------------------------------

struct Inner {
  int64_t n = 0;
  double* v = nullptr;  // 12 vectors of n
  double* S = nullptr;
  double* partial = nullptr;
  St64* st = nullptr;
  double* vec(int k) const { return v + (size_t)k * n; }
};

enum IV { IR, IRT, IP, IQ, IT, IV_, IW, IY, IU, IZ, IS, IX };

mp_status inner_dots(const Inner& w, int k, const double* const* xs, const double* const* ys,
                     const int* outs, cudaStream_t st, const int* gate) {
  Dot64 d{};
  d.k = k;
  d.n = w.n;
  for (int j = 0; j < k; ++j) {
    d.x[j] = xs[j];
    d.y[j] = ys[j];
    d.out[j] = w.S + outs[j];
  }
  dot64_partial_kernel<<<kDotBlocks, 256, 0, st>>>(d, w.partial, gate);
  dot64_final_kernel<<<1, 32, 0, st>>>(d, w.partial, gate);
  count_launch(2);
  return launch_check("dot64");
}

mp_status inner_iteration(const Inner& w, const mp_csr_s* M, bool first, cudaStream_t st) {
  const int64_t n = w.n;
  const int* gate = &w.st->done;
  const SellV SV = sview(M->A);
  const int rb = (int)((M->A.nchunks * 32 + kT - 1) / kT);
  const int g = grid_n(n);
  if (first) {
    copy64_kernel<<<g, 256, 0, st>>>(w.vec(IR), w.vec(IP), n);
    count_launch();
  } else {
    g64_beta<<<1, 1, 0, st>>>(w.st, w.S);
    g64_wp<<<g, 256, 0, st>>>(w.st, w.S, w.vec(IV_), w.vec(IQ), w.vec(IR), w.vec(IP), w.vec(IU),
                              w.vec(IW), n);
    count_launch(2);
  }
  spmv64_kernel<<<rb, kT, 0, st>>>(SV, M->a64, w.vec(IP), w.vec(IQ), gate);
  count_launch();
  mp_status r;
  {
    const double* xs[1] = {w.vec(IRT)};
    const double* ys[1] = {w.vec(IQ)};
    const int outs[1] = {DEN};
    if ((r = inner_dots(w, 1, xs, ys, outs, st, gate)) != MP_OK) return r;
  }
  g64_alpha<<<1, 1, 0, st>>>(w.st, w.S);
  g64_sty<<<g, 256, 0, st>>>(w.st, w.S, w.vec(IR), w.vec(IQ), w.vec(IW), w.vec(IS), w.vec(IT),
                             w.vec(IY), n, first ? 1 : 0);
  spmv64_kernel<<<rb, kT, 0, st>>>(SV, M->a64, w.vec(IT), w.vec(IV_), gate);
  count_launch(3);
  {
    const double* xs[5] = {w.vec(IY), w.vec(IV_), w.vec(IY), w.vec(IV_), w.vec(IV_)};
    const double* ys[5] = {w.vec(IY), w.vec(IT), w.vec(IT), w.vec(IY), w.vec(IV_)};
    const int outs[5] = {MU1, MU2, MU3, MU4, MU5};
    if ((r = inner_dots(w, 5, xs, ys, outs, st, gate)) != MP_OK) return r;
  }
  g64_zeta<<<1, 1, 0, st>>>(w.st, w.S, first ? 1 : 0);
  g64_uzxr<<<g, 256, 0, st>>>(w.st, w.S, w.vec(IQ), w.vec(IS), w.vec(IU), w.vec(IR), w.vec(IZ),
                              w.vec(IP), w.vec(IT), w.vec(IY), w.vec(IV_), w.vec(IX), n);
  count_launch(2);
  {
    const double* xs[2] = {w.vec(IR), w.vec(IRT)};
    const double* ys[2] = {w.vec(IR), w.vec(IR)};
    const int outs[2] = {RR, RHO_NEW};
    if ((r = inner_dots(w, 2, xs, ys, outs, st, gate)) != MP_OK) return r;
  }
  g64_check<<<1, 1, 0, st>>>(w.st, w.S);
  count_launch();
  return launch_check("fp64 gpbicg iteration");
}

// Solves (D A) d = rhs (rhs in w.vec(IR) on entry, d in w.vec(IX) on exit).
mp_status inner_solve(Inner& w, const mp_csr_s* M, double rtol, int64_t maxit, int poll,
                      cudaStream_t st, St64& hs) {
  const int64_t n = w.n;
  const int g = grid_n(n);
  St64 init{1, MP_OK, 0, maxit};
  MPK_CUDA(cudaMemcpyAsync(w.st, &init, sizeof init, cudaMemcpyHostToDevice, st));
  for (int k : {IP, IQ, IT, IV_, IW, IY, IU, IZ, IS, IX}) {
    fill64_kernel<<<g, 256, 0, st>>>(w.vec(k), n, 0.0);
    count_launch();
  }
  copy64_kernel<<<g, 256, 0, st>>>(w.vec(IR), w.vec(IRT), n);
  count_launch();
  mp_status r;
  {
    const double* xs[2] = {w.vec(IR), w.vec(IRT)};
    const double* ys[2] = {w.vec(IR), w.vec(IR)};
    const int outs[2] = {RR0, RHO};
    if ((r = inner_dots(w, 2, xs, ys, outs, st, nullptr)) != MP_OK) return r;
  }
  g64_setup<<<1, 1, 0, st>>>(w.st, w.S, rtol);
  count_launch();
  if ((r = inner_iteration(w, M, true, st)) != MP_OK) return r;
  MPK_CUDA(cudaMemcpyAsync(&hs, w.st, sizeof hs, cudaMemcpyDeviceToHost, st));
  MPK_CUDA(cudaStreamSynchronize(st));
  if (hs.done) return MP_OK;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  MPK_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
  const int64_t before = mp_launch_count(0);
  r = inner_iteration(w, M, false, st);
  const int64_t per = mp_launch_count(0) - before;
  cudaError_t ce = cudaStreamEndCapture(st, &graph);
  if (r != MP_OK || ce != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return r != MP_OK ? r : cuda_error(ce, "cudaStreamEndCapture");
  }
  count_launch(-(int)per);
  ce = cudaGraphInstantiate(&exec, graph, 0);
  if (ce != cudaSuccess) {
    cudaGraphDestroy(graph);
    return cuda_error(ce, "cudaGraphInstantiate");
  }
  while (true) {
    for (int k = 0; k < poll && ce == cudaSuccess; ++k) {
      ce = cudaGraphLaunch(exec, st);
      count_launch((int)per);
    }
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&hs, w.st, sizeof hs, cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess || hs.done) break;
  }
  cudaGraphExecDestroy(exec);
  cudaGraphDestroy(graph);
  if (ce != cudaSuccess) return cuda_error(ce, "fp64 inner solve");
  return MP_OK;
}

mp_status build_f64(mp_csr_s* M, int equilibrate, cudaStream_t st) {
  if (M->a64) return MP_OK;
  // both buffers or neither: a64 set marks the copy as built
  double *a64 = nullptr, *rowscale = nullptr;
  cudaError_t e = cudaMalloc((void**)&a64, sizeof(double) * (size_t)(M->A.nslots > 0 ? M->A.nslots : 1));
  if (e == cudaSuccess)
    e = cudaMalloc((void**)&rowscale, sizeof(double) * (size_t)(M->n > 0 ? M->n : 1));
  if (e != cudaSuccess) {
    cudaFree(a64);
    return cuda_error(e, "FP64 copy of the matrix");
  }
  M->a64 = a64;
  M->rowscale = rowscale;
  M->bytes += 8 * (M->A.nslots + M->n);
  if (M->A.nchunks == 0) return MP_OK;
  const int rb = (int)((M->A.nchunks * 32 + kT - 1) / kT);
  const SellV SV = sview(M->A);
  return dispatch_w(M->prec, [&](auto w) {
    constexpr int W = decltype(w)::value;
    build_f64_kernel<W><<<rb, kT, 0, st>>>(SV, M->A.val, M->a64, M->rowscale, equilibrate);
    count_launch();
    return launch_check("build_f64_kernel");
  });
}

template <int W>
mp_status refine_w(mp_csr_s* M, const mp_vec& b, const mp_vec& x, const mp_refine_opts& o,
                   mp_refine_info* info, cudaStream_t st) {
  const int64_t n = M->n;
  mp_status r = build_f64(M, o.equilibrate, st);
  if (r != MP_OK) return r;
  Inner w;
  w.n = n > 0 ? n : 1;
  const int L = W / 2;
  uint64_t* rbuf = nullptr;   // p-bit residual
  uint64_t* sc = nullptr;     // p-bit scalars: (r,r), (b,b)
  long long* words = nullptr; // emax, dmax bits, xmax bits
  void* dscr = nullptr;
  // a failed allocation skips the solve; the cleanup below frees what was taken
  const size_t db = dot_scratch_bytes(M->prec, 2);
  cudaError_t ca = work_malloc((void**)&w.v, sizeof(double) * 12 * (size_t)w.n, st);
  if (ca == cudaSuccess) ca = work_malloc((void**)&w.S, sizeof(double) * NS64, st);
  if (ca == cudaSuccess) ca = work_malloc((void**)&w.partial, sizeof(double) * 5 * kDotBlocks, st);
  if (ca == cudaSuccess) ca = work_malloc((void**)&w.st, sizeof(St64), st);
  if (ca == cudaSuccess) ca = work_malloc((void**)&rbuf, sizeof(uint64_t) * (L + 1) * (size_t)w.n, st);
  if (ca == cudaSuccess) ca = work_malloc((void**)&sc, sizeof(uint64_t) * 2 * (L + 1), st);
  if (ca == cudaSuccess) ca = work_malloc((void**)&words, sizeof(long long) * 3, st);
  if (ca == cudaSuccess) ca = work_malloc(&dscr, db, st);
  r = ca != cudaSuccess ? cuda_error(ca, "refinement work memory") : init_dot_scratch(dscr, st);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, st);
  const int g = grid_n(n);
  mp_refine_info out{};
  out.status = MP_ERR_NOCONV;
  double bb = 0.0;
  for (int64_t it = 0; r == MP_OK && it <= o.max_outer; ++it) {
    // r = RN_row(b - A x) (exact rows), (r,r) and (b,b) at p bits
    if ((r = launch_spmv(M, M->A, MP_EXACT, x.data, x.ld, rbuf, w.n, b.data, b.ld, nullptr, st)) != MP_OK)
      break;
    DotArgs d;
    d.k = 2;
    d.n = n;
    d.x[0] = rbuf; d.y[0] = rbuf; d.ldx[0] = d.ldy[0] = w.n; d.out[0] = sc; d.out_ld[0] = 1;
    d.x[1] = b.data; d.y[1] = b.data; d.ldx[1] = d.ldy[1] = b.ld; d.out[1] = sc + (L + 1); d.out_ld[1] = 1;
    if ((r = launch_dot(M->prec, d, dscr, nullptr, st)) != MP_OK) break;
    double rr_bb[2] = {0, 0};
    {
      double* dd = w.S;  // reuse two scalar slots as a staging area
      mp_vec v1{1, M->prec, 1, sc}, v2{1, M->prec, 1, sc + (L + 1)};
      mp_vec_to_f64(v1, dd + MU1, st);
      mp_vec_to_f64(v2, dd + MU2, st);
      cudaMemcpyAsync(rr_bb, dd + MU1, sizeof rr_bb, cudaMemcpyDeviceToHost, st);
      cudaError_t ce = cudaStreamSynchronize(st);
      if (ce != cudaSuccess) { r = cuda_error(ce, "refine residual"); break; }
    }
    bb = rr_bb[1];
    out.relres = bb > 0 ? sqrt(rr_bb[0] / bb) : 0.0;
    if (rr_bb[0] == 0.0 || it == o.max_outer) {
      if (rr_bb[0] == 0.0) out.status = MP_OK;
      break;
    }
    // FP64 right-hand side D (r 2^-E), inner solve, p-bit update
    reset_words<<<1, 1, 0, st>>>(words, (unsigned long long*)words + 1, (unsigned long long*)words + 2);
    max_exp_kernel<W><<<g, 256, 0, st>>>(rbuf, n, words);
    rhs_to_f64_kernel<W><<<g, 256, 0, st>>>(rbuf, w.n, n, words, M->rowscale, w.vec(IR));
    count_launch(3);
    St64 hs{};
    if ((r = inner_solve(w, M, o.inner_rtol, o.inner_maxit, o.poll_every > 0 ? o.poll_every : 8, st,
                         hs)) != MP_OK)
      break;
    out.inner_iters += hs.iters;
    correct_kernel<W><<<g, 256, 0, st>>>(x.data, x.ld, n, w.vec(IX), words,
                                         (unsigned long long*)words + 1,
                                         (unsigned long long*)words + 2);
    count_launch();
    unsigned long long bits[2] = {0, 0};
    cudaMemcpyAsync(bits, words + 1, sizeof bits, cudaMemcpyDeviceToHost, st);
    cudaError_t ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) { r = cuda_error(ce, "refine correction"); break; }
    double dm, xm;
    memcpy(&dm, &bits[0], 8);
    memcpy(&xm, &bits[1], 8);
    out.outer = it + 1;
    out.correction = xm > 0 ? dm / xm : dm;
    if (out.correction <= o.rtol) {
      out.status = MP_OK;
      // final residual of the returned x
      if ((r = launch_spmv(M, M->A, MP_EXACT, x.data, x.ld, rbuf, w.n, b.data, b.ld, nullptr, st)) != MP_OK)
        break;
      if ((r = launch_dot(M->prec, d, dscr, nullptr, st)) != MP_OK) break;
      mp_vec v1{1, M->prec, 1, sc};
      mp_vec_to_f64(v1, w.S + MU1, st);
      double rr = 0;
      cudaMemcpyAsync(&rr, w.S + MU1, sizeof rr, cudaMemcpyDeviceToHost, st);
      cudaStreamSynchronize(st);
      out.relres = bb > 0 ? sqrt(rr / bb) : 0.0;
      break;
    }
  }
  cudaEventRecord(e1, st);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  out.ms = ms;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFreeAsync(w.v, st);
  cudaFreeAsync(w.S, st);
  cudaFreeAsync(w.partial, st);
  cudaFreeAsync(w.st, st);
  cudaFreeAsync(rbuf, st);
  cudaFreeAsync(sc, st);
  cudaFreeAsync(words, st);
  cudaFreeAsync(dscr, st);
  cudaStreamSynchronize(st);
  if (info) *info = out;
  if (r != MP_OK) return r;
  return static_cast<mp_status>(out.status);
}

}  // namespace
}  // namespace mpk

using namespace mpk;

extern "C" {

mp_status mp_refine(mp_csr A, mp_vec b, mp_vec x, const mp_refine_opts* opts, mp_refine_info* info,
                    void* stream) {
  if (!A) return set_error(MP_ERR_ARG, "matrix is null");
  if (!opts) return set_error(MP_ERR_ARG, "opts is null");
  if (!prec_ok(A->prec)) return set_error(MP_ERR_PREC, "refinement at p = %d: p <= 1024", A->prec);
  mp_status r;
  if ((r = check_vec(b, A->n, A->prec, "b")) != MP_OK) return r;
  if ((r = check_vec(x, A->n, A->prec, "x")) != MP_OK) return r;
  if (A->n > 0 && b.data == x.data) return set_error(MP_ERR_ARG, "b and x must not alias");
  if (!(opts->rtol >= 0) || !(opts->inner_rtol > 0) || opts->max_outer < 0 || opts->inner_maxit < 1)
    return set_error(MP_ERR_ARG, "invalid refinement options");
  if (!status_word()) return set_error(MP_ERR_CUDA, "status word unavailable");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // private stream fenced to the caller's (the inner solve captures graphs)
  cudaStream_t ps = nullptr;
  cudaEvent_t fence = nullptr;
  if ((r = private_stream_open(st, &ps, &fence)) != MP_OK) return r;
  r = dispatch_w(A->prec, [&](auto w) {
    constexpr int W = decltype(w)::value;
    return refine_w<W>(A, b, x, *opts, info, ps);
  });
  private_stream_close(st, ps, fence);
  return r;
}

}  // extern "C"
