// spmv.cu -- p-bit sparse matrix-vector products on the sliced layout.
//
// One thread owns one row (a warp owns a 32-row chunk), so the ORDERED
// row loop of Section 3 -- y <- RN(y + RN(a*x)) in column order, skipping
// zero factors -- runs unchanged in each thread's registers, and a warp's
// loads of entry j of its 32 rows are 32 consecutive words of every plane.
//
// EXACT rows sum their products exactly: a pre-pass over the row's heads finds
// the exponent range [Emin, Emax] of its nonzero terms; each exact 2p-bit
// product P*2^(E-2p) is added as P*2^(E-Emin) into 64-bit signed counters
// over 32-bit digits (no carries while accumulating); the carries are
// resolved and the sum rounded once.  Counters live in shared memory,
// digit-major so that a warp's 32 threads always hit 32 distinct banks.  A
// row whose span does not fit the per-thread window goes to an overflow list
// handled by a warp-per-row kernel with a window of the full span cap.
#include <algorithm>
#include <climits>

#include "internal.h"
#include "mpdev.cuh"

namespace mpk {
namespace {

constexpr int kThreads = 128;   // 4 chunks per block
constexpr int kFastSpan = 384;  // bits of exponent span handled per thread

// Bits of a row sum kept below the top p bits of its largest term by the
// windowed EXACT form (the rest is checked, not computed; see below).  A row
// whose sum falls more than about kTopGuard - 48 bits below its largest term
// (the skipped columns' error bound is 42 + log2(len) bits, and 8 decisive
// bits are asked for) goes to the exact kernel; fewer guard bits skip more
// columns of every product.
constexpr int kTopGuard = 80;

template <int W>
struct Win {
  static constexpr int fast = (kFastSpan + 64 * W + 96) / 32 + 1;  // digits per thread
  static constexpr int cap = (SPAN_CAP + 64 * W + 96) / 32 + 1;    // digits for the cap
  static constexpr int fast_cols = (kFastSpan + 64 * W + 64) / kR + 4;  // radix-2^29 digits
  static constexpr int top_cols = (32 * W + 64 + kTopGuard) / kR + 6;   // windowed form
};

// Radix-2^29 digits of a row whose terms span `span` bits: the terms' digits
// (offset / 29 + NA + NX) and the carries of up to 2^31 terms plus a sign.
__host__ __device__ inline int digits_cols(int64_t span, int W) {
  return (int)((span + 64 * W + 64) / kR) + 4;
}

// Launch variants (a bit field): bit 0 = the row loop stages the next
// entry's operands (ORDERED: p <= 512 only; EXACT: column form only, word
// form stages at p <= 512), bit 1 = products from radix-2^29 column sums,
// bit 2 = EXACT: column sums computed 16 columns at a time instead of 8
// (windowed form: the register-capped kernel, four 128-thread blocks per SM);
// ORDERED: the register-capped kernel (three blocks of <= 128 threads per SM);
// bit 3 = x gathered from a record copy made before the product;
// bit 4 = EXACT (p >= 512, column form): the windowed kernel.
constexpr int kVarStage = 1, kVarCols = 2, kVarWide = 4, kVarRec = 8, kVarTop = 16;
// A matrix's launch configuration for one mode with the library's defaults
// filled in (chosen from measurements of the n = 10^6 sweep on GB300: the
// word form with a half-and-half L1/shared split for EXACT at p <= 256, the
// register-capped windowed column form from p = 512; column products for
// ORDERED from p = 256 on, register-capped blocks at p = 128 and 1024).
struct LaunchCfg {
  int tpb;
  bool stage, cols, wide, rec, top;
  int carve;  // -1: the driver's choice
};

LaunchCfg launch_cfg(const mp_csr_s* M, int mode, int W) {
  const int v = M->cfg_var[mode];
  LaunchCfg c;
  // record copy of x: worth its extra pass over x from p = 256 on when the
  // gathers are scattered (a stencil's consecutive columns are not) and n is
  // large enough for the pass to pay
  c.rec = v < 0 ? (W >= 8 && M->n >= (int64_t(1) << 16) && M->gather_sectors > 16.0)
                : (v & kVarRec) != 0;
  c.top = false;
  if (mode == MP_ORDERED) {
    c.cols = v < 0 ? W >= 8 : (v & kVarCols) != 0;
    c.stage = W <= 16 && (v < 0 || (v & kVarStage));
    c.tpb = M->cfg_tpb[0] < 0 ? 128 : M->cfg_tpb[0];
    // register-capped kernel (the default at p = 128 and p = 1024)
    c.wide = (v < 0 ? (W == 4 || W == 32) : (v & kVarWide) != 0) && c.tpb <= 128;
    c.carve = M->cfg_carve[0];
  } else {
    c.cols = v < 0 ? W >= 16 : (v & kVarCols) != 0;
    c.top = c.cols && W >= 16 && (v < 0 || (v & kVarTop) != 0);
    c.stage = c.cols ? (v < 0 ? W == 16 : (v & kVarStage) != 0) : W <= 16;
    c.wide = c.cols && (v < 0 ? c.top : (v & kVarWide) != 0);
    c.tpb = M->cfg_tpb[1] < 0 ? 128 : M->cfg_tpb[1];
    c.carve = M->cfg_carve[1] < 0 ? (W <= 8 ? 50 : -1) : M->cfg_carve[1];
  }
  return c;
}

__host__ __device__ inline int digits_for(int64_t span, int W) {
  return (int)((span + 64 * W + 96) / 32) + 1;
}

struct SellView {
  int64_t nchunks, nslots;
  const int64_t* __restrict__ chunk_off;
  const int32_t* __restrict__ row_of;
  const int32_t* __restrict__ row_len;
  const int32_t* __restrict__ col;
  const uint64_t* __restrict__ val;
  // optional: rows whose instance is marked done are skipped (batched solves)
  const int32_t* __restrict__ rinst;
  const int* __restrict__ idone;
  // optional: x as records (element i's L+1 words at xrec + i * xrs, xrs even,
  // 16-byte aligned) for gathers of whole elements instead of one word per plane
  const uint64_t* __restrict__ xrec;
  int xrs;
};

SellView view(const Sell& S, const int32_t* rinst = nullptr, const int* idone = nullptr) {
  return SellView{S.nchunks, S.nslots, S.chunk_off, S.row_of, S.row_len, S.col, S.val,
                  rinst, idone, nullptr, 0};
}

// Record stride (64-bit words) of a p-bit element: L+1 rounded up to even.
inline int record_words(int W) { return ((W / 2 + 1) + 1) & ~1; }

// x[c] gathered from the record copy when there is one, else from the planes.
template <int W>
__device__ __forceinline__ void gather_x(Num<W>& v, const SellView& S, const uint64_t* __restrict__ x,
                                         int64_t ldx, int32_t c) {
  if (S.xrec) {
    constexpr int L = W / 2;
    const uint4* r = reinterpret_cast<const uint4*>(S.xrec + (int64_t)c * S.xrs);
    uint32_t w[2 * ((L + 2) / 2) * 2];
#pragma unroll
    for (int k = 0; k < (L + 2) / 2; ++k) {
      const uint4 q = __ldg(r + k);
      w[4 * k] = q.x;
      w[4 * k + 1] = q.y;
      w[4 * k + 2] = q.z;
      w[4 * k + 3] = q.w;
    }
    unpack_head(((uint64_t)w[1] << 32) | w[0], v.e, v.s);
#pragma unroll
    for (int k = 0; k < W; ++k) v.m[k] = w[2 + k];
  } else {
    load<W>(v, x, ldx, c);
  }
}

__device__ __forceinline__ uint64_t gather_head(const SellView& S, const uint64_t* __restrict__ x,
                                                int32_t c) {
  return S.xrec ? __ldg(S.xrec + (int64_t)c * S.xrs) : __ldg(x + c);
}

// Record copy of x for the gathers.  A warp takes 32 consecutive elements:
// it loads their planes (consecutive lanes, consecutive addresses), lays the
// 32 records out in shared memory and writes them as one contiguous run of
// 32 records, so that its stores are coalesced too (a thread writing its own
// record would leave a warp's stores a record apart).  256 threads a block.
template <int W>
__global__ void __launch_bounds__(256) to_records_kernel(const uint64_t* __restrict__ x,
                                                         int64_t ldx, int64_t n,
                                                         uint64_t* __restrict__ xr) {
  constexpr int L = W / 2;
  constexpr int RS = (L + 2) & ~1;  // words per record: L + 1 rounded up to even
  constexpr int SP = RS + 1;        // odd stride in shared memory: no bank conflicts
  __shared__ uint64_t tile[8][32 * SP];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t* t = tile[warp];
  const int64_t ntiles = (n + 31) / 32;
  for (int64_t tl = blockIdx.x * 8LL + warp; tl < ntiles; tl += (int64_t)gridDim.x * 8) {
    const int64_t i0 = tl * 32;
    const int cnt = (int)(n - i0 < 32 ? n - i0 : 32);
    if (lane < cnt) {
#pragma unroll
      for (int k = 0; k <= L; ++k) t[lane * SP + k] = __ldg(x + (int64_t)k * ldx + i0 + lane);
      if (RS > L + 1) t[lane * SP + L + 1] = 0u;
    }
    __syncwarp();
    uint64_t* dst = xr + i0 * RS;
    for (int w = lane; w < cnt * RS; w += 32) dst[w] = t[(w / RS) * SP + (w % RS)];
    __syncwarp();
  }
}

__device__ __forceinline__ bool row_skipped(const SellView& S, int32_t row) {
  return row < 0 || (S.idone != nullptr && S.idone[S.rinst[row]] != 0);
}

__device__ __forceinline__ void record_status(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

// Whether a row loop keeps the next entry's operands in registers while the
// current one is computed (at p = 1024 the extra registers would spill).
template <int W>
struct Pipelined {
  static constexpr bool value = W <= 16;
};

// ---------------------------------------------------------------------------
// ORDERED
// ---------------------------------------------------------------------------

// The column form of the ORDERED product: the short product from p = 512 on.
template <int W>
__device__ __forceinline__ void ordered_product_cols(const Num<W>& a, const Num<W>& b, Num<W>& r) {
  if constexpr (W >= 16)
    mul_rn_short<W>(a, b, r);
  else
    mul_rn_cols<W>(a, b, r);
}

template <int W, bool PIPE, bool COLS>
__device__ __forceinline__ void ordered_rows(const SellView& S, const uint64_t* __restrict__ x,
                                             int64_t ldx, uint64_t* __restrict__ y, int64_t ldy,
                                             const int* __restrict__ gate) {
  if (gate && *gate) return;
  const int lane = threadIdx.x & 31;
  const int64_t chunk = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (chunk >= S.nchunks) return;
  const int64_t slot = chunk * 32 + lane;
  const int32_t row = S.row_of[slot];
  if (row_skipped(S, row)) return;
  const int32_t len = S.row_len[slot];
  const int64_t base = S.chunk_off[chunk] + lane;
  Num<W> acc;
  set_zero(acc, 0u);
  if (PIPE) {
    // Software pipeline: the column index two entries ahead and the operands
    // one entry ahead are in flight while the current entry is computed.
    Num<W> an, xn;
    int32_t c1 = 0;
    if (len > 0) {
      const int32_t c0 = S.col[base];
      if (len > 1) c1 = S.col[base + 32];
      load_stream<W>(an, S.val, S.nslots, base);
      gather_x<W>(xn, S, x, ldx, c0);
    }
    for (int32_t j = 0; j < len; ++j) {
      const Num<W> a = an, xv = xn;
      if (j + 1 < len) {
        const int64_t k1 = base + (int64_t)(j + 1) * 32;
        const int32_t c = c1;
        if (j + 2 < len) c1 = S.col[k1 + 32];
        load_stream<W>(an, S.val, S.nslots, k1);
        gather_x<W>(xn, S, x, ldx, c);
      }
      if (zero_e(a.e) || zero_e(xv.e)) continue;  // zero fast path
      Num<W> t, s;
      if (COLS)
        ordered_product_cols<W>(a, xv, t);
      else
        mul_rn<W>(a, xv, t);
      add_rn<W>(acc, t, s);
      acc = s;
    }
  } else {
    for (int32_t j = 0; j < len; ++j) {
      const int64_t k = base + (int64_t)j * 32;
      const int32_t c = S.col[k];
      Num<W> a, xv;
      load_stream<W>(a, S.val, S.nslots, k);
      gather_x<W>(xv, S, x, ldx, c);
      if (zero_e(a.e) || zero_e(xv.e)) continue;  // zero fast path
      Num<W> t, s;
      if (COLS)
        ordered_product_cols<W>(a, xv, t);
      else
        mul_rn<W>(a, xv, t);
      add_rn<W>(acc, t, s);
      acc = s;
    }
  }
  if (row >= 0) store<W>(acc, y, ldy, row);
}

template <int W, bool PIPE, bool COLS>
__global__ void __launch_bounds__(256) spmv_ordered_kernel(
    const SellView S, const uint64_t* __restrict__ x, int64_t ldx, uint64_t* __restrict__ y,
    int64_t ldy, const int* __restrict__ gate) {
  ordered_rows<W, PIPE, COLS>(S, x, ldx, y, ldy, gate);
}

// The same with at most 128 threads per block and registers capped so that
// three such blocks fit on an SM: more warps to hide the multiply latency
// where the uncapped kernel is held to two blocks by its registers.
template <int W, bool PIPE, bool COLS>
__global__ void __launch_bounds__(128, 3) spmv_ordered_kernel_capped(
    const SellView S, const uint64_t* __restrict__ x, int64_t ldx, uint64_t* __restrict__ y,
    int64_t ldy, const int* __restrict__ gate) {
  ordered_rows<W, PIPE, COLS>(S, x, ldx, y, ldy, gate);
}

// ---------------------------------------------------------------------------
// EXACT (and the residual r = RN(b - A x))
// ---------------------------------------------------------------------------

template <int W>
__device__ __forceinline__ void value_as_product(const Num<W>& b, uint32_t (&P)[2 * W]) {
#pragma unroll
  for (int k = 0; k < W; ++k) {
    P[k] = 0u;
    P[W + k] = b.m[k];
  }
}

// y_i of an EXACT product (no b term) in one pass over the row: the thread's
// window of counters (the per-thread span kFastSpan, as in the two-pass
// form) is anchored kFastSpan/2 bits below the row's first nonzero term, so
// no pre-pass over the row's exponents is needed.  Every term that lands in
// the window is added as it is read; a term outside it (the row's terms span
// more than kFastSpan/2 bits around the first one) sends the row to the
// overflow list, whose warp-per-row kernel computes it from scratch.  The
// range [emin, emax] of the terms seen bounds the digits that are resolved
// and rounded, exactly as the two-pass form's window anchored at emin.
template <int W, bool COLS, bool PIPE, int G>
__device__ __forceinline__ void exact_row_one_pass(const SellView& S,
                                                   const uint64_t* __restrict__ x, int64_t ldx,
                                                   uint64_t* __restrict__ y, int64_t ldy,
                                                   int32_t* __restrict__ ovf, int64_t slot,
                                                   int32_t row, int32_t len, int64_t base) {
  extern __shared__ int64_t sacc[];
  constexpr int NDW = COLS ? Win<W>::fast_cols : Win<W>::fast;
  constexpr int64_t H = kFastSpan / 2;
  constexpr int R = COLS ? kR : 32;  // bits per counter digit
  const int stride = blockDim.x;
  int64_t* c = sacc + threadIdx.x;
#pragma unroll 4
  for (int d = 0; d < NDW; ++d) c[d * stride] = 0;
  int64_t eb = 0, emin = LLONG_MAX, emax = LLONG_MIN;
  bool over = false;
  uint32_t P[2 * W];
  // adds a * x (sign folded into ng) at bit offset off in [0, 2H]
  auto term = [&](const Num<W>& a, const Num<W>& xv, uint32_t ng) {
    const int64_t E = a.e + xv.e;
    if (emin > emax) eb = E - H;  // the first term sets the anchor
    const int64_t off = E - eb;
    if (off < 0 || off > 2 * H) {
      over = true;
      return;
    }
    emin = min(emin, E);
    emax = max(emax, E);
    if (COLS) {
      add_product_cols<W, G>(c, stride, a.m, xv.m, (uint32_t)off, ng);
    } else {
      if (W >= 16)
        mul_full_ilp<W>(a.m, xv.m, P);
      else
        mul_full<W>(a.m, xv.m, P);
      add_term<W>(c, stride, P, off, ng);
    }
  };
  if (PIPE) {
    Num<W> an, xn;
    int32_t c1 = 0;
    if (len > 0) {
      const int32_t c0 = S.col[base];
      if (len > 1) c1 = S.col[base + 32];
      load_stream<W>(an, S.val, S.nslots, base);
      gather_x<W>(xn, S, x, ldx, c0);
    }
    for (int32_t j = 0; j < len && !over; ++j) {
      const Num<W> a = an, xv = xn;
      if (j + 1 < len) {
        const int64_t k1 = base + (int64_t)(j + 1) * 32;
        const int32_t cn = c1;
        if (j + 2 < len) c1 = S.col[k1 + 32];
        load_stream<W>(an, S.val, S.nslots, k1);
        gather_x<W>(xn, S, x, ldx, cn);
      }
      if (zero_e(a.e) || zero_e(xv.e)) continue;
      term(a, xv, a.s ^ xv.s);
    }
  } else {
    for (int32_t j = 0; j < len && !over; ++j) {
      const int64_t k = base + (int64_t)j * 32;
      const int32_t col = S.col[k];
      Num<W> a, xv;
      load_stream<W>(a, S.val, S.nslots, k);
      gather_x<W>(xv, S, x, ldx, col);
      if (zero_e(a.e) || zero_e(xv.e)) continue;
      term(a, xv, a.s ^ xv.s);
    }
  }
  if (over) {
    const int pos = atomicAdd(ovf, 1);
    ovf[1 + pos] = (int32_t)slot;
    return;
  }
  Num<W> r;
  if (emin > emax) {  // no terms
    set_zero(r, 0u);
    store<W>(r, y, ldy, row);
    return;
  }
  // digits below d0 hold nothing: resolve from d0, whose weight is 2^(lo - 2p)
  const int d0 = (int)((emin - eb) / R);
  const int64_t lo = eb + (int64_t)R * d0;
  int64_t* c0 = c + d0 * stride;
  if (COLS) {
    int nw = 0;
    const uint32_t negative = resolve_cols(c0, stride, digits_cols(emax - lo, W), &nw);
    round_words<W>(c0, stride, nw, lo - 64 * W, negative, r);
  } else {
    const int nd = digits_for(emax - lo, W);
    const uint32_t negative = resolve_digits(c0, stride, nd);
    if (negative) negate_words(c0, stride, nd);
    round_words<W>(c0, stride, nd, lo - 64 * W, negative, r);
  }
  store<W>(r, y, ldy, row);
}

template <int W, bool RESID, bool COLS, bool PIPE = Pipelined<W>::value || COLS, int G = 8>
__global__ void __launch_bounds__(256) spmv_exact_kernel(
    const SellView S, const uint64_t* __restrict__ x, int64_t ldx, uint64_t* __restrict__ y,
    int64_t ldy, const uint64_t* __restrict__ bv, int64_t ldb, int32_t* __restrict__ ovf,
    int* __restrict__ status, const int* __restrict__ gate) {
  extern __shared__ int64_t sacc[];
  if (gate && *gate) return;
  const int lane = threadIdx.x & 31;
  const int64_t chunk = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (chunk >= S.nchunks) return;
  const int64_t slot = chunk * 32 + lane;
  const int32_t row = S.row_of[slot];
  if (row_skipped(S, row)) return;
  const int32_t len = S.row_len[slot];
  const int64_t base = S.chunk_off[chunk] + lane;

  if constexpr (!RESID) {
    exact_row_one_pass<W, COLS, PIPE, G>(S, x, ldx, y, ldy, ovf, slot, row, len, base);
    return;
  }
  // the residual: pass 1, the exponent range of the nonzero terms
  int64_t emin = LLONG_MAX, emax = LLONG_MIN;
  Num<W> b;
  if (RESID) {
    load<W>(b, bv, ldb, row);
    if (!zero_e(b.e)) emin = emax = b.e;
  }
  // four entries' loads in flight at a time (the heads only)
  for (int32_t j0 = 0; j0 < len; j0 += 4) {
    int32_t cc[4];
    uint64_t ha[4], hx[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t k = base + (int64_t)(j0 + u) * 32;
      cc[u] = (j0 + u < len) ? S.col[k] : 0;
      ha[u] = (j0 + u < len) ? __ldg(S.val + k) : pack_head(EXP_ZERO, 0u);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) hx[u] = gather_head(S, x, cc[u]);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      int64_t ea, ex;
      uint32_t sa, sx;
      unpack_head(ha[u], ea, sa);
      unpack_head(hx[u], ex, sx);
      if (zero_e(ea) || zero_e(ex)) continue;
      const int64_t E = ea + ex;
      emin = min(emin, E);
      emax = max(emax, E);
    }
  }
  Num<W> r;
  if (emin > emax) {  // no terms
    set_zero(r, 0u);
    store<W>(r, y, ldy, row);
    return;
  }
  const int64_t span = emax - emin;
  if (span > SPAN_CAP) {
    set_zero(r, 0u);
    store<W>(r, y, ldy, row);
    record_status(status, MP_ERR_SPAN);
    return;
  }
  const int nd = COLS ? digits_cols(span, W) : digits_for(span, W);
  if (nd > (COLS ? Win<W>::fast_cols : Win<W>::fast)) {
    const int pos = atomicAdd(ovf, 1);
    ovf[1 + pos] = (int32_t)slot;
    return;
  }
  const int stride = blockDim.x;
  int64_t* c = sacc + threadIdx.x;
  for (int d = 0; d < nd; ++d) c[d * stride] = 0;

  // pass 2: exact products into the counters
  uint32_t P[2 * W];
  if (RESID && !zero_e(b.e)) {
    if (COLS) {
      add_value_cols<W>(c, stride, b.m, (uint32_t)(b.e - emin + 32 * W), b.s);
    } else {
      value_as_product<W>(b, P);
      add_term<W>(c, stride, P, b.e - emin, b.s);
    }
  }
  // adds the term a * x (sign already folded into ng)
  auto term = [&](const Num<W>& a, const Num<W>& xv, uint32_t ng) {
    if (COLS) {
      add_product_cols<W, G>(c, stride, a.m, xv.m, (uint32_t)(a.e + xv.e - emin), ng);
    } else {
      if (W >= 16)
        mul_full_ilp<W>(a.m, xv.m, P);
      else
        mul_full<W>(a.m, xv.m, P);
      add_term<W>(c, stride, P, a.e + xv.e - emin, ng);
    }
  };
  // staging: at p = 1024 only the column form has registers to spare (its
  // occupancy is bounded by the shared-memory window anyway)
  if (PIPE) {
    Num<W> an, xn;
    int32_t c1 = 0;
    if (len > 0) {
      const int32_t c0 = S.col[base];
      if (len > 1) c1 = S.col[base + 32];
      load_stream<W>(an, S.val, S.nslots, base);
      gather_x<W>(xn, S, x, ldx, c0);
    }
    for (int32_t j = 0; j < len; ++j) {
      const Num<W> a = an, xv = xn;
      if (j + 1 < len) {
        const int64_t k1 = base + (int64_t)(j + 1) * 32;
        const int32_t cn = c1;
        if (j + 2 < len) c1 = S.col[k1 + 32];
        load_stream<W>(an, S.val, S.nslots, k1);
        gather_x<W>(xn, S, x, ldx, cn);
      }
      if (zero_e(a.e) || zero_e(xv.e)) continue;
      term(a, xv, a.s ^ xv.s ^ (RESID ? 1u : 0u));
    }
  } else {
    for (int32_t j = 0; j < len; ++j) {
      const int64_t k = base + (int64_t)j * 32;
      const int32_t col = S.col[k];
      Num<W> a, xv;
      load_stream<W>(a, S.val, S.nslots, k);
      gather_x<W>(xv, S, x, ldx, col);
      if (zero_e(a.e) || zero_e(xv.e)) continue;
      term(a, xv, a.s ^ xv.s ^ (RESID ? 1u : 0u));
    }
  }
  if (COLS) {
    int nw = 0;
    const uint32_t negative = resolve_cols(c, stride, nd, &nw);
    round_words<W>(c, stride, nw, emin - 64 * W, negative, r);
  } else {
    const uint32_t negative = resolve_digits(c, stride, nd);
    if (negative) negate_words(c, stride, nd);
    round_words<W>(c, stride, nd, emin - 64 * W, negative, r);
  }
  store<W>(r, y, ldy, row);
}

// EXACT in a window under the largest term (p >= 512, column products): the
// counters cover only the top p + kTopGuard bits (plus carries) of the row
// sum, columns of a product below the window are not computed, and the
// result is rounded when the bits between the possible error of the skipped
// columns (< 2^eb) and the round bit decide the rounding (guard_bits_decide),
// or when every skipped column is provably zero.  Otherwise (heavy
// cancellation, exact ties) the row goes to the exact warp-per-row kernel
// through the overflow list, so the result is always the exact sum rounded
// once.  The window is a third of the full one and about a third of the
// multiply-adds are skipped.
// G = 4 marks the register-capped form: at most 128 threads per block and
// four blocks per SM (the window's 48 KB allow four).
template <int W, bool PIPE, int G>
__global__ void __launch_bounds__(G == 4 ? 128 : 256, G == 4 ? 4 : 1) spmv_exact_top_kernel(
    const SellView S, const uint64_t* __restrict__ x, int64_t ldx, uint64_t* __restrict__ y,
    int64_t ldy, int32_t* __restrict__ ovf, int* __restrict__ status,
    const int* __restrict__ gate) {
  extern __shared__ int64_t sacc[];
  if (gate && *gate) return;
  const int lane = threadIdx.x & 31;
  const int64_t chunk = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (chunk >= S.nchunks) return;
  const int64_t slot = chunk * 32 + lane;
  const int32_t row = S.row_of[slot];
  if (row_skipped(S, row)) return;
  const int32_t len = S.row_len[slot];
  const int64_t base = S.chunk_off[chunk] + lane;
  int64_t emin = LLONG_MAX, emax = LLONG_MIN;
  for (int32_t j0 = 0; j0 < len; j0 += 4) {
    int32_t cc[4];
    uint64_t ha[4], hx[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t k = base + (int64_t)(j0 + u) * 32;
      cc[u] = (j0 + u < len) ? S.col[k] : 0;
      ha[u] = (j0 + u < len) ? __ldg(S.val + k) : pack_head(EXP_ZERO, 0u);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) hx[u] = gather_head(S, x, cc[u]);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      int64_t ea, ex;
      uint32_t sa, sx;
      unpack_head(ha[u], ea, sa);
      unpack_head(hx[u], ex, sx);
      if (zero_e(ea) || zero_e(ex)) continue;
      emin = min(emin, ea + ex);
      emax = max(emax, ea + ex);
    }
  }
  Num<W> r;
  if (emin > emax) {
    set_zero(r, 0u);
    store<W>(r, y, ldy, row);
    return;
  }
  const int64_t span = emax - emin;
  if (span > SPAN_CAP) {
    set_zero(r, 0u);
    store<W>(r, y, ldy, row);
    record_status(status, MP_ERR_SPAN);
    return;
  }
  const int wb = (int)((span + 32 * W - kTopGuard) / kR);  // window base digit
  const int nd = digits_cols(span, W) - wb;
  auto to_exact_path = [&]() {
    const int pos = atomicAdd(ovf, 1);
    ovf[1 + pos] = (int32_t)slot;
  };
  if (nd > Win<W>::top_cols) {
    to_exact_path();
    return;
  }
  const int stride = blockDim.x;
  int64_t* c = sacc + threadIdx.x;
  for (int d = 0; d < nd; ++d) c[d * stride] = 0;
  bool errp = false;
  auto term = [&](const Num<W>& a, const Num<W>& xv) {
    const uint32_t off = (uint32_t)(a.e + xv.e - emin), q = off / kR;
    add_product_cols_top<W, G>(c, stride, a.m, xv.m, (int)q - wb, off - kR * q, a.s ^ xv.s, errp);
  };
  if (PIPE) {
    Num<W> an, xn;
    int32_t c1 = 0;
    if (len > 0) {
      const int32_t c0 = S.col[base];
      if (len > 1) c1 = S.col[base + 32];
      load_stream<W>(an, S.val, S.nslots, base);
      gather_x<W>(xn, S, x, ldx, c0);
    }
    for (int32_t j = 0; j < len; ++j) {
      const Num<W> a = an, xv = xn;
      if (j + 1 < len) {
        const int64_t k1 = base + (int64_t)(j + 1) * 32;
        const int32_t cn = c1;
        if (j + 2 < len) c1 = S.col[k1 + 32];
        load_stream<W>(an, S.val, S.nslots, k1);
        gather_x<W>(xn, S, x, ldx, cn);
      }
      if (zero_e(a.e) || zero_e(xv.e)) continue;
      term(a, xv);
    }
  } else {
    for (int32_t j = 0; j < len; ++j) {
      const int64_t k = base + (int64_t)j * 32;
      Num<W> a, xv;
      load_stream<W>(a, S.val, S.nslots, k);
      gather_x<W>(xv, S, x, ldx, S.col[k]);
      if (zero_e(a.e) || zero_e(xv.e)) continue;
      term(a, xv);
    }
  }
  int nw = 0;
  const uint32_t negative = resolve_cols(c, stride, nd, &nw);
  int t = nw - 1;
  while (t >= 0 && (uint32_t)c[t * stride] == 0u) --t;
  if (t < 0) {  // the window sums to zero: exact only if nothing was skipped
    if (errp) {
      to_exact_path();
    } else {
      set_zero(r, 0u);
      store<W>(r, y, ldy, row);
    }
    return;
  }
  if (errp) {
    // skipped columns: each < 2^35 at the window's scale, at most 73 per term
    const int64_t eb = 42 + (32 - __clz((uint32_t)len));
    const int64_t nb = 32 * (int64_t)t + (32 - __clz((uint32_t)c[t * stride]));
    if (!guard_bits_decide(c, stride, nw, eb, nb - 32 * W - 1)) {
      to_exact_path();
      return;
    }
  }
  round_words<W>(c, stride, nw, emin - 64 * W + (int64_t)kR * wb, negative, r);
  store<W>(r, y, ldy, row);
}

// Rows from the overflow list: one warp per row, lanes over the row's
// entries, a shared window of the full span cap filled with atomics.  A row
// whose terms span more than the cap gives +0 and MP_ERR_SPAN (the one-pass
// form sends rows here without measuring their span).
template <int W, bool RESID>
__global__ void __launch_bounds__(32) spmv_exact_wide_kernel(
    const SellView S, const uint64_t* __restrict__ x, int64_t ldx, uint64_t* __restrict__ y,
    int64_t ldy, const uint64_t* __restrict__ bv, int64_t ldb, const int32_t* __restrict__ ovf,
    int* __restrict__ status, const int* __restrict__ gate) {
  __shared__ int64_t acc[Win<W>::cap];
  if (gate && *gate) return;
  const int count = ovf[0];
  const int lane = threadIdx.x;
  for (int item = blockIdx.x; item < count; item += gridDim.x) {
    const int64_t slot = ovf[1 + item];
    const int64_t chunk = slot >> 5;
    const int t = (int)(slot & 31);
    const int32_t row = S.row_of[slot];
    const int32_t len = S.row_len[slot];
    const int64_t base = S.chunk_off[chunk] + t;
    int64_t emin = LLONG_MAX, emax = LLONG_MIN;
    Num<W> b;
    if (RESID) {
      load<W>(b, bv, ldb, row);
      if (!zero_e(b.e)) emin = emax = b.e;
    }
    for (int32_t j = lane; j < len; j += 32) {
      const int64_t k = base + (int64_t)j * 32;
      int64_t ea, ex;
      uint32_t sa, sx;
      unpack_head(__ldg(S.val + k), ea, sa);
      unpack_head(__ldg(x + S.col[k]), ex, sx);
      if (!zero_e(ea) && !zero_e(ex)) {
        emin = min(emin, ea + ex);
        emax = max(emax, ea + ex);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      emin = min(emin, __shfl_xor_sync(0xffffffffu, emin, o));
      emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
    }
    if (emin > emax || emax - emin > SPAN_CAP) {  // no terms (y = +0), or beyond the cap
      if (lane == 0) {
        Num<W> z;
        set_zero(z, 0u);
        store<W>(z, y, ldy, row);
        if (emin <= emax) record_status(status, MP_ERR_SPAN);
      }
      __syncwarp();
      continue;
    }
    for (int d = lane; d < Win<W>::cap; d += 32) acc[d] = 0;
    __syncwarp();
    uint32_t P[2 * W];
    if (RESID && lane == 0 && !zero_e(b.e)) {
      value_as_product<W>(b, P);
      uint32_t D[2 * W + 1];
      const int64_t off = b.e - emin;
      shifted_digits<W>(P, (uint32_t)(off & 31), D);
      for (int k = 0; k <= 2 * W; ++k) {
        const int64_t v = (int64_t)D[k];
        atomicAdd((unsigned long long*)&acc[(off >> 5) + k], (unsigned long long)(b.s ? -v : v));
      }
    }
    for (int32_t j = lane; j < len; j += 32) {
      const int64_t k = base + (int64_t)j * 32;
      Num<W> a, xv;
      load<W>(a, S.val, S.nslots, k);
      load<W>(xv, x, ldx, S.col[k]);
      if (zero_e(a.e) || zero_e(xv.e)) continue;
      mul_full<W>(a.m, xv.m, P);
      uint32_t D[2 * W + 1];
      const int64_t off = a.e + xv.e - emin;
      shifted_digits<W>(P, (uint32_t)(off & 31), D);
      const uint32_t ng = a.s ^ xv.s ^ (RESID ? 1u : 0u);
      for (int kk = 0; kk <= 2 * W; ++kk) {
        const int64_t v = (int64_t)D[kk];
        atomicAdd((unsigned long long*)&acc[(off >> 5) + kk], (unsigned long long)(ng ? -v : v));
      }
    }
    __syncwarp();
    if (lane == 0) {
      const int nd = Win<W>::cap;
      const uint32_t negative = resolve_digits(acc, 1, nd);
      if (negative) negate_words(acc, 1, nd);
      Num<W> r;
      round_words<W>(acc, 1, nd, emin - 64 * W, negative, r);
      store<W>(r, y, ldy, row);
    }
    __syncwarp();
  }
}

// Operand of the tuner: nonzero x_i with every mantissa word drawn from an
// integer hash of (i, word) (top bit set), a random sign and an exponent in
// [-8, 8], so that the timed products carry full-width operands.
__device__ __forceinline__ uint32_t tune_hash(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return (uint32_t)(z ^ (z >> 31));
}

template <int W>
__global__ void tune_fill_kernel(uint64_t* x, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    Num<W> v;
#pragma unroll
    for (int k = 0; k < W; ++k) v.m[k] = tune_hash((uint64_t)i * 64 + k);
    v.m[W - 1] |= 0x80000000u;
    const uint32_t h = tune_hash((uint64_t)i * 64 + 63);
    v.e = (int64_t)(h % 17u) - 8;
    v.s = (h >> 16) & 1u;
    store<W>(v, x, n, i);
  }
}

// Gradient of a loss on the sparsity pattern: for every stored a_ij,
// g[pos(i,j)] = RN((-lam_i) * x_j), pos being the entry's position in the
// caller's CSR.  Same traversal as the products (thread per row).
template <int W>
__global__ void __launch_bounds__(kThreads) pattern_grad_kernel(
    const SellView S, const int64_t* __restrict__ src, const uint64_t* __restrict__ lam,
    int64_t ldl, const uint64_t* __restrict__ x, int64_t ldx, uint64_t* __restrict__ g,
    int64_t ldg) {
  const int lane = threadIdx.x & 31;
  const int64_t chunk = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (chunk >= S.nchunks) return;
  const int64_t slot = chunk * 32 + lane;
  const int32_t row = S.row_of[slot];
  if (row < 0) return;
  const int32_t len = S.row_len[slot];
  const int64_t base = S.chunk_off[chunk] + lane;
  Num<W> l;
  load<W>(l, lam, ldl, row);
  l.s ^= 1u;
  for (int32_t j = 0; j < len; ++j) {
    const int64_t k = base + (int64_t)j * 32;
    Num<W> xv, t;
    load<W>(xv, x, ldx, S.col[k]);
    mul_rn<W>(l, xv, t);
    store<W>(t, g, ldg, src[k]);
  }
}

template <int W>
mp_status spmv_w(const mp_csr_s* M, const Sell& S, int mode, const uint64_t* x, int64_t ldx,
                 uint64_t* y, int64_t ldy, const uint64_t* b, int64_t ldb, const int* gate,
                 cudaStream_t st, const int32_t* rinst = nullptr, const int* idone = nullptr) {
  if (S.nchunks == 0) return MP_OK;
  SellView V = view(S, rinst, idone);
  const LaunchCfg cf = launch_cfg(M, mode == MP_ORDERED && !b ? MP_ORDERED : MP_EXACT, W);
  const int tpb = cf.tpb;
  if (cf.rec) {  // gathers from a record copy of x (one pass over x first)
    mp_csr_s* Mw = const_cast<mp_csr_s*>(M);
    const int rs = record_words(W);
    uint64_t*& xrec = is_transposed(M, S) ? Mw->xrec_t : Mw->xrec;
    if (!xrec)
      MPK_CUDA(cudaMalloc((void**)&xrec, sizeof(uint64_t) * rs * (size_t)(M->n > 0 ? M->n : 1)));
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t nb = std::min<int64_t>((M->n + 255) / 256, (int64_t)sms * 8);
    to_records_kernel<W><<<(int)std::max<int64_t>(nb, 1), 256, 0, st>>>(x, ldx, M->n, xrec);
    count_launch();
    V.xrec = xrec;
    V.xrs = rs;
  }
  const int blocks = (int)((S.nchunks * 32 + tpb - 1) / tpb);
  if (mode == MP_ORDERED && !b) {
    constexpr bool P = Pipelined<W>::value;
    auto ordered = [&](auto kern) -> mp_status {
      if (cf.carve >= 0)
        MPK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cf.carve));
      kern<<<blocks, tpb, 0, st>>>(V, x, ldx, y, ldy, gate);
      return MP_OK;
    };
    mp_status r;
    if (cf.wide && tpb <= 128) {
      if (cf.stage && cf.cols)
        r = ordered(spmv_ordered_kernel_capped<W, P, true>);
      else if (cf.stage)
        r = ordered(spmv_ordered_kernel_capped<W, P, false>);
      else if (cf.cols)
        r = ordered(spmv_ordered_kernel_capped<W, false, true>);
      else
        r = ordered(spmv_ordered_kernel_capped<W, false, false>);
    } else if (cf.stage && cf.cols) {
      r = ordered(spmv_ordered_kernel<W, P, true>);
    } else if (cf.stage) {
      r = ordered(spmv_ordered_kernel<W, P, false>);
    } else if (cf.cols) {
      r = ordered(spmv_ordered_kernel<W, false, true>);
    } else {
      r = ordered(spmv_ordered_kernel<W, false, false>);
    }
    if (r != MP_OK) return r;
    count_launch();
    return launch_check("spmv_ordered_kernel");
  }
  int* status = status_word();
  if (!status) return set_error(MP_ERR_CUDA, "status word unavailable");
  int32_t* const ovf = ovf_of(M, S);
  MPK_CUDA(cudaMemsetAsync(ovf, 0, sizeof(int32_t), st));
  const bool cols = cf.cols;
  // the windowed form serves y = A x only; the residual keeps the full window
  const bool top = cf.top && !b;
  const size_t smem = (size_t)(top ? Win<W>::top_cols : cols ? Win<W>::fast_cols : Win<W>::fast) *
                     tpb * sizeof(int64_t);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  auto exact = [&](auto kern, const uint64_t* bb) -> mp_status {
    MPK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // shared memory vs L1 split: more digit windows per SM, or more cache for
    // the gathers of x
    MPK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  cf.carve < 0 ? (int)cudaSharedmemCarveoutDefault : cf.carve));
    kern<<<blocks, tpb, smem, st>>>(V, x, ldx, y, ldy, bb, ldb, ovf, status, gate);
    return MP_OK;
  };
  mp_status r;
  if (b) {
    r = cols ? exact(spmv_exact_kernel<W, true, true>, b) : exact(spmv_exact_kernel<W, true, false>, b);
    if (r != MP_OK) return r;
    spmv_exact_wide_kernel<W, true><<<sms * 4, 32, 0, st>>>(V, x, ldx, y, ldy, b, ldb, ovf,
                                                            status, gate);
  } else {
    const bool stage = cf.stage, wide = cf.wide;
    auto launch_top = [&](auto kern) -> mp_status {
      MPK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      MPK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                    cf.carve < 0 ? (int)cudaSharedmemCarveoutDefault : cf.carve));
      kern<<<blocks, tpb, smem, st>>>(V, x, ldx, y, ldy, ovf, status, gate);
      return MP_OK;
    };
    bool launched = false;
    if constexpr (W >= 16) {
      if (top) {
        // bit 2 on the windowed form: the register-capped kernel (<= 128 threads)
        const bool capped = wide && tpb <= 128;
        r = capped ? (stage ? launch_top(spmv_exact_top_kernel<W, true, 4>)
                            : launch_top(spmv_exact_top_kernel<W, false, 4>))
            : stage ? launch_top(spmv_exact_top_kernel<W, true, 8>)
                    : launch_top(spmv_exact_top_kernel<W, false, 8>);
        launched = true;
      }
    }
    if (launched)
      ;
    else if (!cols)
      r = exact(spmv_exact_kernel<W, false, false>, nullptr);
    else if (stage && wide)
      r = exact(spmv_exact_kernel<W, false, true, true, 16>, nullptr);
    else if (stage)
      r = exact(spmv_exact_kernel<W, false, true, true, 8>, nullptr);
    else if (wide)
      r = exact(spmv_exact_kernel<W, false, true, false, 16>, nullptr);
    else
      r = exact(spmv_exact_kernel<W, false, true, false, 8>, nullptr);
    if (r != MP_OK) return r;
    spmv_exact_wide_kernel<W, false><<<sms * 4, 32, 0, st>>>(V, x, ldx, y, ldy, nullptr, 0,
                                                             ovf, status, gate);
  }
  count_launch(2);
  return launch_check("spmv_exact_kernel");
}

mp_status check_spmv_args(mp_csr A, const mp_vec& x, const mp_vec& y, int mode) {
  if (!A) return set_error(MP_ERR_ARG, "matrix is null");
  if (mode != MP_ORDERED && mode != MP_EXACT) return set_error(MP_ERR_ARG, "mode %d", mode);
  mp_status r;
  if ((r = check_vec(x, A->n, A->prec, "x")) != MP_OK) return r;
  if ((r = check_vec(y, A->n, A->prec, "y")) != MP_OK) return r;
  if (A->n > 0 && x.data == y.data) return set_error(MP_ERR_ARG, "x and y must not alias");
  return MP_OK;
}

}  // namespace

mp_status launch_spmv(const mp_csr_s* M, const Sell& S, int mode, const uint64_t* x, int64_t ldx,
                      uint64_t* y, int64_t ldy, const uint64_t* b, int64_t ldb, const int* gate,
                      cudaStream_t st) {
  if (prec_big(M->prec)) return launch_spmv_big(M, S, mode, x, ldx, y, ldy, b, ldb, gate, st);
  return dispatch_w(M->prec, [&](auto w) {
    constexpr int W = decltype(w)::value;
    return spmv_w<W>(M, S, mode, x, ldx, y, ldy, b, ldb, gate, st);
  });
}

mp_status launch_spmv_batched(const mp_csr_s* M, int mode, const uint64_t* x, int64_t ldx,
                              uint64_t* y, int64_t ldy, const int32_t* rinst, const int* idone,
                              cudaStream_t st) {
  return dispatch_w(M->prec, [&](auto w) {
    constexpr int W = decltype(w)::value;
    return spmv_w<W>(M, M->A, mode, x, ldx, y, ldy, nullptr, 0, nullptr, st, rinst, idone);
  });
}

}  // namespace mpk

using namespace mpk;

extern "C" {

mp_status mp_spmv(mp_csr A, mp_vec x, mp_vec y, mp_mode mode, void* stream) {
  mp_status r = check_spmv_args(A, x, y, mode);
  if (r != MP_OK) return r;
  return launch_spmv(A, A->A, mode, x.data, x.ld, y.data, y.ld, nullptr, 0, nullptr,
                     static_cast<cudaStream_t>(stream));
}

mp_status mp_spmv_t(mp_csr A, mp_vec x, mp_vec y, mp_mode mode, void* stream) {
  mp_status r = check_spmv_args(A, x, y, mode);
  if (r != MP_OK) return r;
  if (!A->has_t) return set_error(MP_ERR_ARG, "matrix was created without MP_CSR_TRANSPOSE");
  return launch_spmv(A, A->AT, mode, x.data, x.ld, y.data, y.ld, nullptr, 0, nullptr,
                     static_cast<cudaStream_t>(stream));
}

mp_status mp_csr_set_config(mp_csr A, int32_t mode, int32_t tpb, int32_t variant,
                            int32_t carveout) {
  if (!A) return set_error(MP_ERR_ARG, "matrix is null");
  if (mode != MP_ORDERED && mode != MP_EXACT) return set_error(MP_ERR_ARG, "mode %d", mode);
  if (tpb != -1 && tpb != 32 && tpb != 64 && tpb != 128 && tpb != 256)
    return set_error(MP_ERR_ARG, "threads per block %d not in {-1,32,64,128,256}", tpb);
  if (variant < -1 || variant > 31) return set_error(MP_ERR_ARG, "variant %d not in -1..31", variant);
  if (carveout < -1 || carveout > 100) return set_error(MP_ERR_ARG, "carve-out %d", carveout);
  A->cfg_tpb[mode] = tpb;
  A->cfg_var[mode] = variant;
  A->cfg_carve[mode] = carveout;
  return MP_OK;
}

mp_status mp_csr_get_config(mp_csr A, int32_t mode, int32_t* tpb, int32_t* variant,
                            int32_t* carveout) {
  if (!A) return set_error(MP_ERR_ARG, "matrix is null");
  if (mode != MP_ORDERED && mode != MP_EXACT) return set_error(MP_ERR_ARG, "mode %d", mode);
  const LaunchCfg c = launch_cfg(A, mode, A->prec / 32);
  if (tpb) *tpb = c.tpb;
  if (variant)
    *variant = (c.cols ? kVarCols : 0) | (c.stage ? kVarStage : 0) | (c.wide ? kVarWide : 0) |
               (c.rec ? kVarRec : 0) | (c.top ? kVarTop : 0);
  if (carveout) *carveout = c.carve;
  return MP_OK;
}

mp_status mp_csr_tune(mp_csr A, int32_t mode, int32_t reps, int32_t* tpb_out, int32_t* var_out,
                      int32_t* carve_out, double* ms_out, void* stream) {
  if (!A) return set_error(MP_ERR_ARG, "matrix is null");
  if (mode != MP_ORDERED && mode != MP_EXACT) return set_error(MP_ERR_ARG, "mode %d", mode);
  if (reps < 1) return set_error(MP_ERR_ARG, "reps %d", reps);
  if (prec_big(A->prec))
    return set_error(MP_ERR_PREC, "p = %d runs one fixed warp-per-row form; the tuner covers p <= 1024",
                     A->prec);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int L = A->prec / 64;
  const int64_t n = A->n > 0 ? A->n : 1;
  uint64_t *x = nullptr, *y = nullptr;
  MPK_CUDA(cudaMalloc((void**)&x, sizeof(uint64_t) * (L + 1) * (size_t)n));
  if (cudaMalloc((void**)&y, sizeof(uint64_t) * (L + 1) * (size_t)n) != cudaSuccess) {
    cudaFree(x);
    return set_error(MP_ERR_ALLOC, "tuner vectors");
  }
  mp_status r = dispatch_w(A->prec, [&](auto w) {
    constexpr int W = decltype(w)::value;
    tune_fill_kernel<W><<<(int)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, st>>>(x, n);
    count_launch();
    return launch_check("tune_fill_kernel");
  });
  const int32_t old_t = A->cfg_tpb[mode], old_v = A->cfg_var[mode], old_c = A->cfg_carve[mode];
  float best = 1e30f;
  int32_t bt = old_t, bv = old_v, bc = old_c;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // ORDERED: both product forms, staging for p <= 512; EXACT: the word
  // form, and the column form with and without staging, 8 or 16 columns at
  // a time, each under four shared-memory carve-outs
  int32_t vars[12], carves[4] = {-1, 25, 50, 75};
  int nvar = 0, ncarve = mode == MP_EXACT ? 4 : 1;
  if (mode == MP_ORDERED) {
    for (int32_t v = 0; v <= (kVarCols | kVarStage); v += (A->prec > 512 ? kVarCols : 1))
      vars[nvar++] = v;
    // the register-capped form of the default product form
    vars[nvar++] = kVarWide | (A->prec >= 256 ? kVarCols : 0) | (A->prec <= 512 ? kVarStage : 0);
  } else {
    vars[nvar++] = 0;
    for (int32_t v : {kVarCols, kVarCols | kVarStage, kVarCols | kVarWide,
                      kVarCols | kVarStage | kVarWide})
      vars[nvar++] = v;
    if (A->prec >= 512) {  // the windowed form, plain and register-capped
      vars[nvar++] = kVarTop | kVarCols;
      vars[nvar++] = kVarTop | kVarCols | kVarStage;
      vars[nvar++] = kVarTop | kVarCols | kVarWide;
      vars[nvar++] = kVarTop | kVarCols | kVarWide | kVarStage;
    }
  }
  // the same gathering x from its record copy, for the default form
  {
    const int32_t saved = A->cfg_var[mode];
    A->cfg_var[mode] = -1;
    const LaunchCfg d = launch_cfg(A, mode, A->prec / 32);
    A->cfg_var[mode] = saved;
    const int32_t dv = (d.cols ? kVarCols : 0) | (d.stage ? kVarStage : 0) |
                       (d.wide ? kVarWide : 0) | (d.top ? kVarTop : 0);
    bool listed = false;
    for (int i = 0; i < nvar; ++i) listed = listed || vars[i] == dv;
    if (!listed) vars[nvar++] = dv;
    vars[nvar++] = dv | kVarRec;
  }
  for (int32_t tpb : {64, 128, 256}) {
    for (int vi = 0; vi < nvar && r == MP_OK; ++vi) {
      for (int ci = 0; ci < ncarve && r == MP_OK; ++ci) {
        A->cfg_tpb[mode] = tpb;
        A->cfg_var[mode] = vars[vi];
        A->cfg_carve[mode] = carves[ci];
        r = launch_spmv(A, A->A, mode, x, n, y, n, nullptr, 0, nullptr, st);
        cudaEventRecord(e0, st);
        for (int k = 0; k < reps && r == MP_OK; ++k)
          r = launch_spmv(A, A->A, mode, x, n, y, n, nullptr, 0, nullptr, st);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= reps;
        if (r == MP_OK && ms < best) {
          best = ms;
          bt = tpb;
          bv = vars[vi];
          bc = carves[ci];
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(st);
  cudaFree(x);
  cudaFree(y);
  A->cfg_tpb[mode] = r == MP_OK ? bt : old_t;
  A->cfg_var[mode] = r == MP_OK ? bv : old_v;
  A->cfg_carve[mode] = r == MP_OK ? bc : old_c;
  if (r != MP_OK) return r;
  if (ms_out) *ms_out = best;
  return mp_csr_get_config(A, mode, tpb_out, var_out, carve_out);
}

mp_status mp_csr_grad(mp_csr A, mp_vec lam, mp_vec x, mp_vec g, void* stream) {
  if (!A) return set_error(MP_ERR_ARG, "matrix is null");
  if (!prec_ok(A->prec)) return set_error(MP_ERR_PREC, "pattern gradient at p = %d: p <= 1024", A->prec);
  mp_status r;
  if ((r = check_vec(lam, A->n, A->prec, "lam")) != MP_OK) return r;
  if ((r = check_vec(x, A->n, A->prec, "x")) != MP_OK) return r;
  if ((r = check_vec(g, A->nnz, A->prec, "g")) != MP_OK) return r;
  if (A->A.nchunks == 0) return MP_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const SellView V = view(A->A);
  const int blocks = (int)((A->A.nchunks * 32 + kThreads - 1) / kThreads);
  return dispatch_w(A->prec, [&](auto w) {
    constexpr int W = decltype(w)::value;
    pattern_grad_kernel<W><<<blocks, kThreads, 0, st>>>(V, A->A.src, lam.data, lam.ld, x.data, x.ld,
                                                        g.data, g.ld);
    count_launch();
    return launch_check("pattern_grad_kernel");
  });
}

mp_status mp_residual(mp_csr A, mp_vec b, mp_vec x, mp_vec r_, void* stream) {
  mp_status r = check_spmv_args(A, x, r_, MP_EXACT);
  if (r != MP_OK) return r;
  if ((r = check_vec(b, A->n, A->prec, "b")) != MP_OK) return r;
  return launch_spmv(A, A->A, MP_EXACT, x.data, x.ld, r_.data, r_.ld, b.data, b.ld, nullptr,
                     static_cast<cudaStream_t>(stream));
}

}  // extern "C"
