// bigp_solve.cu -- BiCG and GPBiCG (Fig. 5, K = I), CGS and BiCGSTAB (the
// other product-type methods of Tables 1-2, textbook forms) at p = 2048,
// 4096, 8192, the precisions at which the paper's solves converge; BiCGSTAB
// also with ILU(0) (bigp_ilu.cu) as the left preconditioner of Section 4.2
// and Table 3, or as a right one.
//
// Same readings and operation order as the p <= 1024 drivers: r0 = RN(b - A x0)
// row by row exactly, r~ = r0, exact inner products, every vector update
// rounded left to right, the stopping rule (r,r) <= RN(RN(rtol^2) (r0,r0)) +
// RN(atol^2) checked once r_i is formed, breakdown on rho = 0 or a zero
// (r~, q) / (p~, z), GPBiCG's zeta = eta = +0 on a zero divisor and its exit on
// zeta = 0.  The pieces are the warp-per-value kernels: products and the
// residual (bigp.cu), exact dots, one generic update kernel
//   out_k = RN(+-a_k + RN(alpha * (+-b_k)))   (a, alpha optional),
// and a one-warp scalar kernel that runs a short program of p-bit scalar
// operations (mul, add, sub, correctly rounded division, compare, tests that
// set the solver's gate).  Every kernel returns at once when the gate is set,
// so iterations launched after a stop change nothing; the host reads the
// state every poll_every iterations.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "bigp.cuh"

namespace mpk {
namespace {

using namespace bigp;

struct BState {
  int gate;    // set on convergence or breakdown: every later kernel returns at once
  int status;  // MP_OK, MP_ERR_BREAKDOWN, MP_ERR_NOCONV
  long long iters;
};

// ---- vector update ---------------------------------------------------------------

enum { kNegA = 1, kNegB = 2 };

// out_k = RN(sa a_k + RN(alpha sb b_k)); alpha == nullptr: the second term is
// sb b_k itself; a == nullptr: out_k is the second term alone.  Both inputs of
// element k are read before out_k is written, so out may be a or b.
template <int W>
__global__ void __launch_bounds__(kBigThreads) lin_kernel(uint64_t* out, const uint64_t* a,
                                                          const uint64_t* b,
                                                          const uint64_t* alpha, int64_t ld,
                                                          int64_t n, int flags,
                                                          const int* __restrict__ gate) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (*gate) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const WarpMem m = carve<W>(smem, warp, false);
  int64_t eal = EXP_ZERO;
  uint32_t sal = 0u;
  if (alpha) {
    unpack_head(alpha[0], eal, sal);
    if (!zero_e(eal)) wload<W>(m.A, alpha, 1, 0, lane);
  }
  const uint32_t na = (flags & kNegA) ? 1u : 0u, nb = (flags & kNegB) ? 1u : 0u;
  for (int64_t i = (int64_t)blockIdx.x * kBigWarps + warp; i < n;
       i += (int64_t)gridDim.x * kBigWarps) {
    int64_t eb, ea = EXP_ZERO;
    uint32_t sb, sa = 0u;
    unpack_head(b[i], eb, sb);
    sb ^= nb;
    if (a) {
      unpack_head(a[i], ea, sa);
      sa ^= na;
    }
    // second term t = RN(alpha * b') or b'
    int64_t te = EXP_ZERO;
    uint32_t ts;
    if (alpha) {
      ts = sal ^ sb;
      if (!zero_e(eal) && !zero_e(eb)) {
        wload<W>(m.X, b, ld, i, lane);
        __syncwarp();
        te = wmul_rn<W>(m.A, m.X, eal + eb, m, m.T, lane);
      }
    } else {
      ts = sb;
      te = eb;
      if (!zero_e(eb)) wload<W>(m.T, b, ld, i, lane);
    }
    if (a && !zero_e(ea)) wload<W>(m.Y, a, ld, i, lane);
    __syncwarp();  // every lane has read element i before it is written
    if (!a) {
      wstore<W>(m.T, te, ts, out, ld, i, lane);
    } else if (zero_e(ea) && zero_e(te)) {
      wstore<W>(m.T, EXP_ZERO, sa & ts, out, ld, i, lane);
    } else if (zero_e(te)) {
      wstore<W>(m.Y, ea, sa, out, ld, i, lane);
    } else if (zero_e(ea)) {
      wstore<W>(m.T, te, ts, out, ld, i, lane);
    } else {
      wadd<W>(m.Y, ea, sa, m.T, te, ts, m.cnt, lane);
      wstore<W>(m.Y, ea, sa, out, ld, i, lane);
    }
    __syncwarp();
  }
}

// +0 in every element (heads and limbs).
__global__ void zero_vec_kernel(uint64_t* v, int64_t ld, int64_t n, int L) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    v[i] = pack_head(EXP_ZERO, 0u);
    for (int k = 1; k <= L; ++k) v[(int64_t)k * ld + i] = 0;
  }
}

// Every scalar slot (head + L limbs, record-major) to +0.
__global__ void init_slots_kernel(uint64_t* S, int nslot, int L) {
  for (int i = threadIdx.x; i < nslot * (L + 1); i += blockDim.x)
    S[i] = (i % (L + 1) == 0) ? pack_head(EXP_ZERO, 0u) : 0ull;
}

__global__ void init_span_kernel(long long* e) {
  if (threadIdx.x < 5) {
    e[threadIdx.x] = LLONG_MAX;
    e[5 + threadIdx.x] = LLONG_MIN;
  }
}

// ---- scalar unit ---------------------------------------------------------------------

// Scalars live in slots of L+1 words (head, limbs) at S + slot (L+1).
enum SCode : int8_t {
  kMul,    // d = RN(a b)
  kAdd,    // d = RN(a + b)
  kSub,    // d = RN(a - b)
  kDiv,    // d = RN(a / b), b nonzero
  kDivZ,   // d = b == 0 ? +0 : RN(a / b)
  kZero,   // d = +0
  kCopy,   // d = a
  kF64,    // d = the double f[imm], exactly
  kBrkZ,   // a == 0: stop with MP_ERR_BREAKDOWN
  kDoneLe, // a <= b: stop with MP_OK
  kIter,   // iters = imm
  kHist,   // history[imm] = a
  kIfNz,   // a != 0: skip the next imm operations
  kSkip,   // skip the next imm operations
};

struct SOp {
  int8_t code, d, a, b;
  int32_t imm;
};

constexpr int kMaxOps = 24;

struct SProg {
  SOp op[kMaxOps];
  int n;
  double f[2];
};

// -1, 0, 1 as a - b (zeros of either sign equal), mantissas in shared memory.
template <int W>
__device__ int wcmp(const uint32_t* Ma, int64_t ea, uint32_t sa, const uint32_t* Mb, int64_t eb,
                    uint32_t sb, int lane) {
  const int ga = zero_e(ea) ? 0 : (sa ? -1 : 1), gb = zero_e(eb) ? 0 : (sb ? -1 : 1);
  if (ga != gb) return ga < gb ? -1 : 1;
  if (ga == 0) return 0;
  int mag;
  if (ea != eb) {
    mag = ea > eb ? 1 : -1;
  } else {
    constexpr int per = W / 32;
    int d = 0;
    for (int k = lane * per + per - 1; k >= lane * per; --k) {
      if (Ma[k] != Mb[k]) {
        d = Ma[k] > Mb[k] ? 1 : -1;
        break;
      }
    }
    const unsigned dm = __ballot_sync(kFull, d != 0);
    mag = dm ? __shfl_sync(kFull, d, 31 - __clz(dm)) : 0;
  }
  return ga > 0 ? mag : -mag;
}

// The p-bit value of a double (exact): 53-bit mantissa in the top limb.
template <int W>
__device__ void wfrom_f64(double v, uint32_t* M, int64_t& e, uint32_t& s, int lane) {
  s = signbit(v) ? 1u : 0u;
  e = EXP_ZERO;
  uint64_t top = 0;
  if (v != 0.0) {
    int ex = 0;
    const double f = frexp(fabs(v), &ex);
    top = (uint64_t)ldexp(f, 53) << 11;
    e = ex;
  }
  for (int k = lane; k < W; k += 32) M[k] = 0u;
  __syncwarp();
  if (lane == 0) {
    M[W - 2] = (uint32_t)top;
    M[W - 1] = (uint32_t)(top >> 32);
  }
  __syncwarp();
}

// One warp runs the program; stops at the first op after the gate is set.
template <int W>
__global__ void __launch_bounds__(32) sprog_kernel(uint64_t* S, BState* st, SProg prog,
                                                   uint64_t* hist, int64_t hist_ld) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (st->gate) return;
  constexpr int L = W / 2, REC = L + 1;
  const int lane = threadIdx.x & 31;
  const WarpMem m = carve<W>(smem, 0, false);
  unsigned char* extra = smem + BigMem<W>::bytes(false);
  int64_t* SW = reinterpret_cast<int64_t*>(extra);            // [W + 5]
  uint32_t* Qw = reinterpret_cast<uint32_t*>(SW + (W + 6));   // [W + 4]
  uint32_t* Uw = Qw + (W + 4);                                // [2W + 2]
  for (int pc = 0; pc < prog.n; ++pc) {
    const SOp o = prog.op[pc];
    uint64_t* dst = S + (int64_t)o.d * REC;
    const uint64_t* pa = S + (int64_t)o.a * REC;
    const uint64_t* pb = S + (int64_t)o.b * REC;
    int64_t ea = EXP_ZERO, eb = EXP_ZERO;
    uint32_t sa = 0u, sb = 0u;
    unpack_head(pa[0], ea, sa);
    unpack_head(pb[0], eb, sb);
    __syncwarp();
    switch (o.code) {
      case kMul: {
        int64_t e = EXP_ZERO;
        if (!zero_e(ea) && !zero_e(eb)) {
          wload<W>(m.A, pa, 1, 0, lane);
          wload<W>(m.X, pb, 1, 0, lane);
          __syncwarp();
          e = wmul_rn<W>(m.A, m.X, ea + eb, m, m.T, lane);
        }
        wstore<W>(m.T, e, sa ^ sb, dst, 1, 0, lane);
        break;
      }
      case kAdd:
      case kSub: {
        if (o.code == kSub) sb ^= 1u;
        if (zero_e(ea) && zero_e(eb)) {
          wstore<W>(m.Y, EXP_ZERO, sa & sb, dst, 1, 0, lane);
        } else if (zero_e(eb)) {
          wload<W>(m.Y, pa, 1, 0, lane);
          __syncwarp();
          wstore<W>(m.Y, ea, sa, dst, 1, 0, lane);
        } else if (zero_e(ea)) {
          wload<W>(m.T, pb, 1, 0, lane);
          __syncwarp();
          wstore<W>(m.T, eb, sb, dst, 1, 0, lane);
        } else {
          wload<W>(m.Y, pa, 1, 0, lane);
          wload<W>(m.T, pb, 1, 0, lane);
          __syncwarp();
          wadd<W>(m.Y, ea, sa, m.T, eb, sb, m.cnt, lane);
          wstore<W>(m.Y, ea, sa, dst, 1, 0, lane);
        }
        break;
      }
      case kDiv:
      case kDivZ: {
        int64_t e = EXP_ZERO;
        uint32_t s = sa ^ sb;
        if (zero_e(eb)) {
          s = 0u;  // kDivZ: +0 (kDiv is only issued after a zero test of b)
        } else if (!zero_e(ea)) {
          wload<W>(m.A, pa, 1, 0, lane);
          wload<W>(m.X, pb, 1, 0, lane);
          __syncwarp();
          e = wdiv<W>(m.A, ea, m.X, eb, Uw, m.cnt, Qw, SW, m.T, lane);
        }
        wstore<W>(m.T, e, s, dst, 1, 0, lane);
        break;
      }
      case kZero:
        wstore<W>(m.T, EXP_ZERO, 0u, dst, 1, 0, lane);
        break;
      case kCopy:
        for (int k = lane; k < REC; k += 32) dst[k] = pa[k];
        break;
      case kF64: {
        int64_t e;
        uint32_t s;
        wfrom_f64<W>(prog.f[o.imm], m.T, e, s, lane);
        wstore<W>(m.T, e, s, dst, 1, 0, lane);
        break;
      }
      case kBrkZ:
        if (zero_e(ea) && lane == 0) {
          st->status = MP_ERR_BREAKDOWN;
          st->gate = 1;
        }
        break;
      case kDoneLe: {
        if (!zero_e(ea)) wload<W>(m.A, pa, 1, 0, lane);
        if (!zero_e(eb)) wload<W>(m.X, pb, 1, 0, lane);
        __syncwarp();
        if (wcmp<W>(m.A, ea, sa, m.X, eb, sb, lane) <= 0 && lane == 0) {
          st->status = MP_OK;
          st->gate = 1;
        }
        break;
      }
      case kIter:
        if (lane == 0) st->iters = o.imm;
        break;
      case kHist:
        if (hist)
          for (int k = lane; k < REC; k += 32) hist[(int64_t)k * hist_ld + o.imm] = pa[k];
        break;
      case kIfNz:
        if (!zero_e(ea)) pc += o.imm;
        break;
      case kSkip:
        pc += o.imm;
        break;
    }
    __syncwarp();
    if (__shfl_sync(kFull, st->gate, 0)) break;
  }
}

// ---- host driver -----------------------------------------------------------------


enum Slot {
  RHO, RHO_PREV, ALPHA, BETA, ZETA, ETA, DEN, MU1, MU2, MU3, MU4, MU5, TAU, RR, RR0, THR, T1, T2,
  T3, OMEGA, TS, TT, NSLOT
};

struct Prog {
  SProg p{};
  Prog& add(SCode c, int d = 0, int a = 0, int b = 0, int imm = 0) {
    p.op[p.n++] = SOp{(int8_t)c, (int8_t)d, (int8_t)a, (int8_t)b, imm};
    return *this;
  }
};

template <int W>
struct Solver {
  const mp_csr_s* A;
  const Sell* SA;
  const Sell* SAT;
  int mode;
  int64_t n, ld;
  cudaStream_t st;
  uint64_t* S = nullptr;  // scalar slots
  BState* bs = nullptr;
  void* dscr = nullptr;
  uint64_t* hist = nullptr;
  int64_t hist_ld = 0;
  int* gate() const { return &bs->gate; }
  uint64_t* slot(int j) const { return S + (size_t)j * (W / 2 + 1); }

  mp_status lin(uint64_t* out, const uint64_t* a, const uint64_t* b, int alpha_slot, int flags) {
    const size_t sm = (size_t)kBigWarps * BigMem<W>::bytes(false);
    int grid = 0;
    mp_status r;
    if ((r = big_grid(lin_kernel<W>, sm, n, &grid)) != MP_OK) return r;
    const uint64_t* al = alpha_slot < 0 ? nullptr : slot(alpha_slot);
    lin_kernel<W><<<grid, kBigThreads, sm, st>>>(out, a, b, al,
                                                 ld, n, flags, gate());
    count_launch();
    return launch_check("lin_kernel");
  }
  mp_status spmv(const Sell& M, const uint64_t* x, uint64_t* y) {
    return launch_spmv_big(A, M, mode, x, ld, y, ld, nullptr, 0, gate(), st);
  }
  mp_status dot(const uint64_t* x, const uint64_t* y, int s) {
    return launch_dot_big(A->prec, x, ld, y, ld, n, slot(s), 1, dscr, gate(), st);
  }
  mp_status run(const Prog& pr) {
    const size_t sm =
        BigMem<W>::bytes(false) + 8 * (size_t)(W + 6) + 4 * (size_t)(W + 4) +
        4 * (size_t)(2 * W + 2);
    MPK_CUDA(cudaFuncSetAttribute(sprog_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sm));
    sprog_kernel<W><<<1, 32, sm, st>>>(S, bs, pr.p, hist, hist_ld);
    count_launch();
    return launch_check("sprog_kernel");
  }
};

// Host-side double of a scalar record (for the information block only).
double rec_to_double(const uint64_t* rec, int L) {
  const int64_t h = (int64_t)rec[0];
  const int64_t e = h >> 1;
  if (e == EXP_ZERO) return 0.0;
  const double m = (double)(rec[L] >> 11) * 0x1p-53;
  const int ec = (int)std::max<int64_t>(-4000, std::min<int64_t>(4000, e));
  return ((h & 1) ? -1.0 : 1.0) * std::ldexp(m, ec);
}

template <int W>
mp_status solve_big_w(int method, mp_csr A, mp_vec b, mp_vec x, const mp_solve_opts* o,
                      mp_solve_info* info, cudaStream_t st, const mp_ilu_s* pre, int pre_left) {
  constexpr int L = W / 2;
  const int64_t n = A->n;
  Solver<W> s;
  s.A = A;
  s.SA = o->transpose ? &A->AT : &A->A;
  s.SAT = o->transpose ? &A->A : &A->AT;
  s.mode = o->mode;
  s.n = n;
  s.ld = n > 0 ? n : 1;
  s.st = st;
  s.hist = o->history.data;
  s.hist_ld = o->history.ld;
  static const int kVecs[4] = {7, 13, 10, 8};  // BiCG, GPBiCG, CGS, BiCGSTAB
  // the last one holds the iterate; an ILU(0) preconditioner adds two
  const int nvec = kVecs[method] + (pre ? 2 : 0);
  const bool left = pre && pre_left;
  const size_t vbytes = sizeof(uint64_t) * (L + 1) * (size_t)s.ld;
  uint64_t* V = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  // BiCG: a second stream and two events, for A^T p~ beside A p
  cudaStream_t st2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  BState hs{0, MP_ERR_NOCONV, 0};
  mp_status r = MP_OK;
  // a failing CUDA call ends the solve through the cleanup below
  auto ok = [&](cudaError_t e, const char* what) {
    return e == cudaSuccess ? MP_OK : cuda_error(e, what);
  };
  do {
    if (method == 0) {
      r = ok(cudaStreamCreateWithFlags(&st2, cudaStreamNonBlocking), "cudaStreamCreate");
      if (r == MP_OK) r = ok(cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming), "cudaEventCreate");
      if (r == MP_OK) r = ok(cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming), "cudaEventCreate");
      if (r != MP_OK) break;
    }
    if ((r = ok(cudaMalloc((void**)&V, vbytes * nvec), "cudaMalloc")) != MP_OK) break;
    r = ok(cudaMalloc((void**)&s.S, sizeof(uint64_t) * (L + 1) * NSLOT),
           "cudaMalloc");
    if (r != MP_OK) break;
    if ((r = ok(cudaMalloc((void**)&s.bs, sizeof(BState)), "cudaMalloc")) != MP_OK) break;
    if ((r = ok(cudaMalloc(&s.dscr, dot_big_scratch_bytes(A->prec)), "cudaMalloc")) != MP_OK) break;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);
    r = ok(cudaMemcpyAsync(s.bs, &hs, sizeof hs, cudaMemcpyHostToDevice, st),
           "cudaMemcpyAsync");
    if (r != MP_OK) break;
    init_span_kernel<<<1, 32, 0, st>>>(static_cast<long long*>(s.dscr));
    init_slots_kernel<<<1, 256, 0, st>>>(s.S, NSLOT, L);
    count_launch(2);
    auto vec = [&](int k) { return V + (size_t)k * (L + 1) * s.ld; };
    for (int k = 0; k < nvec; ++k) {  // every work vector starts as +0 (GPBiCG's u = z = s = 0)
      const int zg = (int)std::min<int64_t>((s.ld + 255) / 256, 1024);
      zero_vec_kernel<<<zg, 256, 0, st>>>(vec(k), s.ld, s.ld, L);
      count_launch();
    }
    auto copy = [&](uint64_t* dst, int64_t ldd, const uint64_t* src, int64_t lds) -> mp_status {
      if (n == 0) return MP_OK;
      MPK_CUDA(cudaMemcpy2DAsync(dst, ldd * 8, src, lds * 8, n * 8, L + 1,
                                 cudaMemcpyDeviceToDevice, st));
      return MP_OK;
    };
    uint64_t *rv = vec(0), *rt = vec(1), *pv = vec(2), *xw = vec(nvec - 1);
    if ((r = copy(xw, s.ld, x.data, x.ld)) != MP_OK) break;  // the iterate, ld = n
    // r0 = RN(b - A x0) row by row exactly, r~ = r0; with a left
    // preconditioner r0 = K^{-1} RN(b - A x0), the residual formed in vec(7)
    uint64_t* r0 = left ? vec(7) : rv;
    if ((r = launch_spmv_big(A, *s.SA, MP_EXACT, x.data, x.ld, r0, s.ld, b.data, b.ld, s.gate(),
                             st)) != MP_OK)
      break;
    if (left && (r = launch_ilu0_apply(pre, r0, s.ld, rv, s.ld, s.gate(), st)) != MP_OK) break;
    if ((r = copy(rt, s.ld, rv, s.ld)) != MP_OK) break;
    if ((r = s.dot(rv, rv, RR0)) != MP_OK) break;
    {
      Prog pr;
      pr.p.f[0] = o->rtol;
      pr.p.f[1] = o->atol;
      pr.add(kF64, T1, 0, 0, 0).add(kF64, T2, 0, 0, 1).add(kMul, T1, T1, T1).add(kMul, T2, T2, T2);
      pr.add(kMul, T3, T1, RR0).add(kAdd, THR, T3, T2).add(kDoneLe, 0, RR0, THR);
      if ((r = s.run(pr)) != MP_OK) break;
    }
    if ((r = s.dot(rt, rv, RHO)) != MP_OK) break;
    const int poll = o->poll_every > 0 ? o->poll_every : 1;
    for (int64_t i = 1; i <= o->maxit && r == MP_OK; ++i) {
      if (method == 0) {  // BiCG
        uint64_t *pt = vec(3), *z = vec(4), *zt = vec(5);
        Prog p0;
        p0.add(kBrkZ, 0, RHO);
        if (i > 1) p0.add(kDiv, BETA, RHO, RHO_PREV);
        if ((r = s.run(p0)) != MP_OK) break;
        if (i == 1) {
          if ((r = copy(pv, s.ld, rv, s.ld)) != MP_OK) break;
          if ((r = copy(pt, s.ld, rt, s.ld)) != MP_OK) break;
        } else {
          if ((r = s.lin(pv, rv, pv, BETA, 0)) != MP_OK) break;  // p = r + beta p
          if ((r = s.lin(pt, rt, pt, BETA, 0)) != MP_OK) break;  // p~ = r~ + beta p~
        }
        // z~ = A^T p~ on the second stream, beside z = A p, the (p~, z) dot
        // and alpha; joined before r~ takes it
        if ((r = ok(cudaEventRecord(ev_fork, st), "cudaEventRecord")) != MP_OK) break;
        if ((r = ok(cudaStreamWaitEvent(st2, ev_fork, 0), "cudaStreamWaitEvent")) != MP_OK) break;
        if ((r = launch_spmv_big(A, *s.SAT, s.mode, pt, s.ld, zt, s.ld, nullptr, 0, s.gate(),
                                 st2)) != MP_OK)
          break;  // z~ = A^T p~
        if ((r = ok(cudaEventRecord(ev_join, st2), "cudaEventRecord")) != MP_OK) break;
        if ((r = s.spmv(*s.SA, pv, z)) != MP_OK) break;    // z = A p
        if ((r = s.dot(pt, z, DEN)) != MP_OK) break;
        Prog p1;
        p1.add(kBrkZ, 0, DEN).add(kDiv, ALPHA, RHO, DEN);
        if ((r = s.run(p1)) != MP_OK) break;
        if ((r = s.lin(xw, xw, pv, ALPHA, 0)) != MP_OK) break;      // x = x + alpha p
        if ((r = s.lin(rv, rv, z, ALPHA, kNegB)) != MP_OK) break;   // r = r - alpha z
        if ((r = ok(cudaStreamWaitEvent(st, ev_join, 0), "cudaStreamWaitEvent")) != MP_OK) break;
        if ((r = s.lin(rt, rt, zt, ALPHA, kNegB)) != MP_OK) break;  // r~ = r~ - alpha z~
      } else if (method == 2) {  // CGS (textbook form, the oracle's reading)
        uint64_t *u = vec(3), *q = vec(4), *v = vec(5), *w = vec(6), *aw = vec(7), *tmp = vec(8);
        Prog p0;
        p0.add(kBrkZ, 0, RHO);
        if (i > 1) p0.add(kDiv, BETA, RHO, RHO_PREV);
        if ((r = s.run(p0)) != MP_OK) break;
        if (i == 1) {
          if ((r = copy(u, s.ld, rv, s.ld)) != MP_OK) break;
          if ((r = copy(pv, s.ld, rv, s.ld)) != MP_OK) break;
        } else {
          if ((r = s.lin(u, rv, q, BETA, 0)) != MP_OK) break;     // u = r + beta q
          if ((r = s.lin(tmp, q, pv, BETA, 0)) != MP_OK) break;   // q + beta p
          if ((r = s.lin(pv, u, tmp, BETA, 0)) != MP_OK) break;   // p = u + beta (q + beta p)
        }
        if ((r = s.spmv(*s.SA, pv, v)) != MP_OK) break;  // v = A p
        if ((r = s.dot(rt, v, DEN)) != MP_OK) break;
        Prog p1;
        p1.add(kBrkZ, 0, DEN).add(kDiv, ALPHA, RHO, DEN);
        if ((r = s.run(p1)) != MP_OK) break;
        if ((r = s.lin(q, u, v, ALPHA, kNegB)) != MP_OK) break;  // q = u - alpha v
        if ((r = s.lin(w, u, q, -1, 0)) != MP_OK) break;         // w = u + q
        if ((r = s.lin(xw, xw, w, ALPHA, 0)) != MP_OK) break;    // x = x + alpha w
        if ((r = s.spmv(*s.SA, w, aw)) != MP_OK) break;          // A w
        if ((r = s.lin(rv, rv, aw, ALPHA, kNegB)) != MP_OK) break;  // r = r - alpha A w
      } else if (method == 3) {  // BiCGSTAB (textbook form, the oracle's reading)
        uint64_t *v = vec(3), *sv = vec(4), *t = vec(5), *tmp = vec(6);
        // ILU(0): right, v = A K^{-1} p and t = A K^{-1} s with x taking
        // K^{-1} p and K^{-1} s; left, v = K^{-1} A p and t = K^{-1} A s
        // (vec(7) and vec(8) hold K^{-1} p, K^{-1} s or A p, A s)
        uint64_t *ph = pre ? vec(7) : nullptr, *sh = pre ? vec(8) : nullptr;
        Prog p0;
        p0.add(kBrkZ, 0, RHO);
        if (i > 1)
          p0.add(kDiv, T1, RHO, RHO_PREV).add(kDiv, T2, ALPHA, OMEGA).add(kMul, BETA, T1, T2);
        if ((r = s.run(p0)) != MP_OK) break;
        if (i == 1) {
          if ((r = copy(pv, s.ld, rv, s.ld)) != MP_OK) break;
        } else {
          if ((r = s.lin(tmp, pv, v, OMEGA, kNegB)) != MP_OK) break;  // p - omega v
          if ((r = s.lin(pv, rv, tmp, BETA, 0)) != MP_OK) break;      // p = r + beta (p - omega v)
        }
        const uint64_t* pu = pv;  // what x takes alpha times
        if (pre && !left) {
          if ((r = launch_ilu0_apply(pre, pv, s.ld, ph, s.ld, s.gate(), st)) != MP_OK) break;
          pu = ph;
        }
        if ((r = s.spmv(*s.SA, pu, left ? ph : v)) != MP_OK) break;  // v = A p
        if (left && (r = launch_ilu0_apply(pre, ph, s.ld, v, s.ld, s.gate(), st)) != MP_OK) break;
        if ((r = s.dot(rt, v, DEN)) != MP_OK) break;
        Prog p1;
        p1.add(kBrkZ, 0, DEN).add(kDiv, ALPHA, RHO, DEN);
        if ((r = s.run(p1)) != MP_OK) break;
        if ((r = s.lin(sv, rv, v, ALPHA, kNegB)) != MP_OK) break;  // s = r - alpha v
        const uint64_t* su = sv;  // what x takes omega times
        if (pre && !left) {
          if ((r = launch_ilu0_apply(pre, sv, s.ld, sh, s.ld, s.gate(), st)) != MP_OK) break;
          su = sh;
        }
        if ((r = s.spmv(*s.SA, su, left ? sh : t)) != MP_OK) break;  // t = A s
        if (left && (r = launch_ilu0_apply(pre, sh, s.ld, t, s.ld, s.gate(), st)) != MP_OK) break;
        if ((r = s.dot(t, sv, TS)) != MP_OK) break;
        if ((r = s.dot(t, t, TT)) != MP_OK) break;
        Prog p2;
        p2.add(kDivZ, OMEGA, TS, TT);  // omega = (t, s) / (t, t), +0 when t = 0
        if ((r = s.run(p2)) != MP_OK) break;
        if ((r = s.lin(xw, xw, pu, ALPHA, 0)) != MP_OK) break;     // x + alpha p
        if ((r = s.lin(xw, xw, su, OMEGA, 0)) != MP_OK) break;     // ... + omega s
        if ((r = s.lin(rv, sv, t, OMEGA, kNegB)) != MP_OK) break;  // r = s - omega t
      } else {  // GPBiCG
        uint64_t *q = vec(3), *t = vec(4), *v = vec(5), *w = vec(6), *y = vec(7), *u = vec(8),
                 *z = vec(9), *sv = vec(10), *tmp = vec(11);
        Prog p0;
        p0.add(kBrkZ, 0, RHO);
        if (i > 1)
          p0.add(kDiv, T1, RHO, RHO_PREV).add(kDiv, T2, ALPHA, ZETA).add(kMul, BETA, T1, T2);
        if ((r = s.run(p0)) != MP_OK) break;
        if (i == 1) {
          if ((r = copy(pv, s.ld, rv, s.ld)) != MP_OK) break;
        } else {
          if ((r = s.lin(w, v, q, BETA, 0)) != MP_OK) break;        // w = v + beta q
          if ((r = s.lin(tmp, pv, u, -1, kNegB)) != MP_OK) break;   // p - u
          if ((r = s.lin(pv, rv, tmp, BETA, 0)) != MP_OK) break;    // p = r + beta (p - u)
        }
        if ((r = s.spmv(*s.SA, pv, q)) != MP_OK) break;  // q = A p
        if ((r = s.dot(rt, q, DEN)) != MP_OK) break;
        Prog p1;
        p1.add(kBrkZ, 0, DEN).add(kDiv, ALPHA, RHO, DEN);
        if ((r = s.run(p1)) != MP_OK) break;
        if (i == 1) {
          if ((r = s.lin(t, rv, q, ALPHA, kNegB)) != MP_OK) break;  // t = r - alpha q
          if ((r = s.lin(y, rv, q, ALPHA, kNegA)) != MP_OK) break;  // y = alpha q - r
          if ((r = s.spmv(*s.SA, t, v)) != MP_OK) break;            // v = A t
          if ((r = s.dot(v, t, MU2)) != MP_OK) break;
          if ((r = s.dot(v, v, MU5)) != MP_OK) break;
          Prog p2;
          p2.add(kDivZ, ZETA, MU2, MU5).add(kZero, ETA);
          if ((r = s.run(p2)) != MP_OK) break;
        } else {
          if ((r = s.lin(sv, t, rv, -1, kNegB)) != MP_OK) break;     // s = t - r
          if ((r = s.lin(t, rv, q, ALPHA, kNegB)) != MP_OK) break;   // t = r - alpha q
          if ((r = s.spmv(*s.SA, t, v)) != MP_OK) break;             // v = A t
          if ((r = s.lin(tmp, w, q, -1, kNegB)) != MP_OK) break;     // w - q
          if ((r = s.lin(y, sv, tmp, ALPHA, kNegB)) != MP_OK) break; // y = s - alpha (w - q)
          if ((r = s.dot(y, y, MU1)) != MP_OK) break;
          if ((r = s.dot(v, t, MU2)) != MP_OK) break;
          if ((r = s.dot(y, t, MU3)) != MP_OK) break;
          if ((r = s.dot(v, y, MU4)) != MP_OK) break;
          if ((r = s.dot(v, v, MU5)) != MP_OK) break;
          Prog p2;
          p2.add(kMul, T1, MU5, MU1).add(kMul, T2, MU4, MU4).add(kSub, TAU, T1, T2);
          p2.add(kIfNz, 0, TAU, 0, 3).add(kZero, ZETA).add(kZero, ETA).add(kSkip, 0, 0, 0, 8);
          p2.add(kMul, T1, MU1, MU2).add(kMul, T2, MU3, MU4).add(kSub, T3, T1, T2);
          p2.add(kDiv, ZETA, T3, TAU);
          p2.add(kMul, T1, MU5, MU3).add(kMul, T2, MU4, MU2).add(kSub, T3, T1, T2);
          p2.add(kDiv, ETA, T3, TAU);
          if ((r = s.run(p2)) != MP_OK) break;
        }
        // u = zeta q + eta (s + beta u)
        if ((r = s.lin(tmp, sv, u, BETA, 0)) != MP_OK) break;
        if ((r = s.lin(tmp, nullptr, tmp, ETA, 0)) != MP_OK) break;
        if ((r = s.lin(u, tmp, q, ZETA, 0)) != MP_OK) break;
        // z = zeta r + eta z - alpha u
        if ((r = s.lin(tmp, nullptr, z, ETA, 0)) != MP_OK) break;
        if ((r = s.lin(tmp, tmp, rv, ZETA, 0)) != MP_OK) break;
        if ((r = s.lin(z, tmp, u, ALPHA, kNegB)) != MP_OK) break;
        // x = x + alpha p + z
        if ((r = s.lin(xw, xw, pv, ALPHA, 0)) != MP_OK) break;
        if ((r = s.lin(xw, xw, z, -1, 0)) != MP_OK) break;
        // r = t - eta y - zeta v
        if ((r = s.lin(tmp, t, y, ETA, kNegB)) != MP_OK) break;
        if ((r = s.lin(rv, tmp, v, ZETA, kNegB)) != MP_OK) break;
      }
      Prog p3;
      p3.add(kIter, 0, 0, 0, (int32_t)i).add(kCopy, RHO_PREV, RHO);
      if ((r = s.run(p3)) != MP_OK) break;
      if ((r = s.dot(rv, rv, RR)) != MP_OK) break;
      if ((r = s.dot(rt, rv, RHO)) != MP_OK) break;
      Prog p4;
      if (s.hist && i - 1 < o->history.n) p4.add(kHist, 0, RR, 0, (int32_t)(i - 1));
      p4.add(kDoneLe, 0, RR, THR);
      if (method == 1) p4.add(kBrkZ, 0, ZETA);
      if (method == 3) p4.add(kBrkZ, 0, OMEGA);
      if ((r = s.run(p4)) != MP_OK) break;
      if (i % poll == 0 || i == o->maxit) {
        r = ok(cudaMemcpyAsync(&hs, s.bs, sizeof hs, cudaMemcpyDeviceToHost, st),
               "cudaMemcpyAsync");
        if (r != MP_OK) break;
        if ((r = ok(cudaStreamSynchronize(st), "cudaStreamSynchronize")) != MP_OK) break;
        if (hs.gate) break;
      }
    }
    if (r != MP_OK) break;
    if ((r = copy(x.data, x.ld, xw, s.ld)) != MP_OK) break;  // x holds the last iterate
    cudaEventRecord(e1, st);
    r = ok(cudaMemcpyAsync(&hs, s.bs, sizeof hs, cudaMemcpyDeviceToHost, st),
           "cudaMemcpyAsync");
    if (r != MP_OK) break;
    if ((r = ok(cudaStreamSynchronize(st), "cudaStreamSynchronize")) != MP_OK) break;
    if (info) {
      memset(info, 0, sizeof *info);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      info->ms = ms;
      info->iters = hs.iters;
      info->status = hs.status;
      std::vector<uint64_t> h(2 * (L + 1));
      if ((r = ok(cudaMemcpy(h.data(), s.slot(hs.iters == 0 ? RR0 : RR), 8 * (L + 1),
                          cudaMemcpyDeviceToHost), "cudaMemcpy")) != MP_OK) break;
      r = ok(cudaMemcpy(h.data() + L + 1, s.slot(RR0), 8 * (L + 1), cudaMemcpyDeviceToHost),
             "cudaMemcpy");
      if (r != MP_OK) break;
      const double a = rec_to_double(h.data(), L), c = rec_to_double(h.data() + L + 1, L);
      info->relres = c > 0 ? std::sqrt(a / c) : 0.0;
    }
  } while (false);
  cudaStreamSynchronize(st);
  if (st2) {
    cudaStreamSynchronize(st2);
    cudaStreamDestroy(st2);
  }
  if (ev_fork) cudaEventDestroy(ev_fork);
  if (ev_join) cudaEventDestroy(ev_join);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(V);
  cudaFree(s.S);
  cudaFree(s.bs);
  cudaFree(s.dscr);
  if (r != MP_OK) return r;
  return static_cast<mp_status>(hs.status);
}

}  // namespace

mp_status solve_big(int method, mp_csr A, mp_vec b, mp_vec x, const mp_solve_opts* opts,
                    mp_solve_info* info, cudaStream_t st, const mp_ilu_s* pre, int pre_left) {
  if (method < 0 || method > 3) return set_error(MP_ERR_ARG, "method %d", method);
  if (pre && method != 3) return set_error(MP_ERR_ARG, "ILU(0) is BiCGSTAB's preconditioner");
  switch (A->prec) {
    case 2048: return solve_big_w<64>(method, A, b, x, opts, info, st, pre, pre_left);
    case 4096: return solve_big_w<128>(method, A, b, x, opts, info, st, pre, pre_left);
    case 8192: return solve_big_w<256>(method, A, b, x, opts, info, st, pre, pre_left);
    default: return set_error(MP_ERR_PREC, "precision %d", A->prec);
  }
}

}  // namespace mpk
