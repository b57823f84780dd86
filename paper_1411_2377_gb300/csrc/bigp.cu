// bigp.cu -- CSR SpMV (ORDERED and EXACT), exact dot products and axpy at
// p = 2048, 4096 and 8192 bits, the precisions at which the paper's solves of
// Tables 1-2 converge.
//
// Above 1024 bits a value no longer fits in one thread's registers, so each
// value is handled by a whole warp.  Mantissas sit in the warp's slice of
// shared memory; the 32 lanes split the W^2 partial products of a product
// (each lane walks pairs of adjacent schoolbook columns, each column a 96-bit
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
#include "bigp.cuh"

namespace mpk {
namespace {

using namespace bigp;

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
                                                                const uint64_t* __restrict__ rb,
                                                                int64_t ldb,
                                                                const int* __restrict__ gate) {
  // rb != nullptr: the residual y = RN(b - A x), b_i an extra exact term.
  extern __shared__ __align__(16) unsigned char smem[];
  if (gate && *gate) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const WarpMem m = carve<W>(smem, warp, true);
  const uint32_t flip = rb ? 1u : 0u;
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
    int64_t eb = EXP_ZERO;
    uint32_t sb = 0u;
    if (rb) {
      unpack_head(__ldg(rb + row), eb, sb);
      if (!zero_e(eb) && lane == 0) {
        lo = min(lo, (long long)eb);
        hi = max(hi, (long long)eb);
      }
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
      if (!zero_e(eb)) {  // b = (Mb 2^p) 2^(eb - 2p): its words sit above W zero words
        wload<W>(m.A, rb, ldb, row, lane);
        __syncwarp();
        for (int k = lane; k < 2 * W; k += 32) m.cnt[k] = k < W ? 0 : (int64_t)m.A[k - W];
        __syncwarp();
        wplace<W>(m.acc, m, eb - lo, sb != 0u, lane);
      }
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
        wplace<W>(m.acc, m, ea + ex - lo, (sa ^ sx ^ flip) != 0u, lane);
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
                                    int64_t n, long long* emin, long long* emax,
                                    const int* __restrict__ gate) {
  if (gate && *gate) return;
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
    int64_t n, const long long* __restrict__ span, int64_t* part, int nb,
    const int* __restrict__ gate) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (gate && *gate) return;
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
                                                               int64_t ldo, int* status,
                                                               const int* __restrict__ gate) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (gate && *gate) return;
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



template <int W>
int big_dot_blocks(int64_t n) {
  int64_t b = (n + 4 * kBigWarps - 1) / (4 * kBigWarps);  // about four elements per warp
  const int64_t lim = (int64_t)big_sm_count() * 2;
  if (b > lim) b = lim;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

mp_status launch_spmv_big(const mp_csr_s* M, const Sell& S, int mode, const uint64_t* x,
                          int64_t ldx, uint64_t* y, int64_t ldy, const uint64_t* rb, int64_t ldb,
                          const int* gate, cudaStream_t st) {
  if (rb && mode != MP_EXACT) return set_error(MP_ERR_ARG, "a residual is an EXACT row sum");
  if (S.nchunks == 0) return MP_OK;
  BigSell B{S.nslots, S.nchunks, S.chunk_off, S.row_of, S.row_len, S.col, S.val};
  // the matrix's overflow-list word (unused at these precisions) is the row counter
  unsigned* next = reinterpret_cast<unsigned*>(ovf_of(M, S));
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
      big_exact_kernel<W><<<grid, kBigThreads, sm, st>>>(B, x, ldx, y, ldy, status, next, rb, ldb,
                                                           gate);
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
                         int64_t n, uint64_t* out, int64_t ldo, void* scratch, const int* gate,
                         cudaStream_t st) {
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
    big_dot_span_kernel<<<sgrid, 256, 0, st>>>(x, y, n, span, span + 5, gate);
    big_dot_accum_kernel<W><<<nb, kBigThreads, sm, st>>>(x, ldx, y, ldy, n, span, part, nb, gate);
    big_dot_finalize_kernel<W><<<1, 256, sm1, st>>>(span, part, nb, out, ldo, status, gate);
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
