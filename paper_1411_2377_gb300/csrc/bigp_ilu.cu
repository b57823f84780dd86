// bigp_ilu.cu -- ILU(0) at p = 2048, 4096, 8192 (Section 4.2, Table 3: the
// BiCGSTAB+ILU(0) runs that converge are the 2048-8192-bit ones), one value
// per warp with the mantissas in the warp's shared memory.
//
// The factor storage, the levels and the arithmetic are those of ilu.cu (the
// textbook IKJ factorisation, every step rounded, nothing skipped); here each
// level is one launch of one warp per row:
//   factorisation: for stored (i, k), k < i ascending: l_ik = RN(a_ik/u_kk),
//     then for stored (i, j), j > k ascending, with (k, j) stored:
//     a_ij = RN(a_ij - RN(l_ik u_kj));
//   forward:  y_i = r_i - RN(l_ik y_k) for k < i ascending, rounded per step;
//   backward: w_i = RN((y_i - RN(u_ik w_k) for k > i ascending) / u_ii).
// A row reads only rows of earlier levels, which earlier launches finished;
// the row's own entries change within the factorisation launch, so every
// load of the factor and of w goes through L2 (ld.global.cg), never the
// read-only path.
#include "bigp.cuh"

namespace mpk {
namespace {

using namespace bigp;

// Per-warp shared memory: a WarpMem (no exact window), then the division's
// scratch S [W + 6] int64, Q [W + 4] and U [2W + 2] words, and l [W] words.
template <int W>
struct IluMem {
  static constexpr size_t kDiv = 8 * (size_t)(W + 6) + 4 * (size_t)(W + 4) + 4 * (size_t)(2 * W + 2);
  static constexpr size_t kBytes = BigMem<W>::bytes(false) + kDiv + 4 * (size_t)W;
};

struct IluWarp {
  WarpMem m;
  int64_t* S;
  uint32_t *Q, *U, *L;
};

template <int W>
__device__ __forceinline__ IluWarp ilu_carve(unsigned char* smem, int warp) {
  unsigned char* b = smem + (size_t)warp * IluMem<W>::kBytes;
  IluWarp u;
  u.m = carve<W>(b, 0, false);
  u.S = reinterpret_cast<int64_t*>(b + BigMem<W>::bytes(false));
  u.Q = reinterpret_cast<uint32_t*>(u.S + (W + 6));
  u.U = u.Q + (W + 4);
  u.L = u.U + (2 * W + 2);
  return u;
}

// Head of element i into (e, s) and, when nonzero, its mantissa into dst.
template <int W>
__device__ __forceinline__ void wget(uint32_t* dst, const uint64_t* v, int64_t ld, int64_t i,
                                     int64_t& e, uint32_t& s, int lane) {
  unpack_head(__ldcg(v + i), e, s);
  if (!zero_e(e)) {
    for (int k = lane; k < W / 2; k += 32) {
      const uint64_t limb = __ldcg(v + (int64_t)(k + 1) * ld + i);
      dst[2 * k] = (uint32_t)limb;
      dst[2 * k + 1] = (uint32_t)(limb >> 32);
    }
  }
  __syncwarp();
}

// (Y, ye, ys) <- RN(y - RN(a b)) with the signed-zero rules of round to
// nearest: a zero product leaves a nonzero y as it is and gives
// (+-0) - (+-0) its IEEE sign; a zero y takes -RN(a b).  a's and b's
// mantissas are in shared memory when their exponents are nonzero.
template <int W>
__device__ __forceinline__ void wsub_prod(uint32_t* Y, int64_t& ye, uint32_t& ys,
                                          const uint32_t* a, int64_t ea, uint32_t sa,
                                          const uint32_t* b, int64_t eb, uint32_t sb,
                                          const WarpMem& m, int lane) {
  const uint32_t ts = sa ^ sb ^ 1u;  // the sign of -(a b)
  if (zero_e(ea) || zero_e(eb)) {    // -(a b) is a zero of sign ts
    if (zero_e(ye)) ys = ys & ts;
    return;
  }
  const int64_t te = wmul_rn<W>(a, b, ea + eb, m, m.T, lane);
  if (zero_e(ye)) {
    for (int k = lane; k < W; k += 32) Y[k] = m.T[k];
    ye = te;
    ys = ts;
    __syncwarp();
    return;
  }
  wadd<W>(Y, ye, ys, m.T, te, ts, m.cnt, lane);
  __syncwarp();
}

template <int W>
__global__ void __launch_bounds__(kBigThreads) big_ilu_level_kernel(
    const int32_t* __restrict__ rows, int64_t count, const int64_t* __restrict__ rowptr,
    const int32_t* __restrict__ col, const int64_t* __restrict__ diag, uint64_t* lu, int64_t nnz,
    int* status) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t t = (int64_t)blockIdx.x * kBigWarps + warp;
  if (t >= count) return;  // the whole warp
  const IluWarp u = ilu_carve<W>(smem, warp);
  const WarpMem& m = u.m;
  const int32_t i = rows[t];
  const int64_t a = rowptr[i], b = rowptr[i + 1];
  for (int64_t ik = a; ik < b && col[ik] < i; ++ik) {
    const int32_t k = col[ik];
    int64_t ek, ea;
    uint32_t sk, sa;
    wget<W>(m.X, lu, nnz, diag[k], ek, sk, lane);  // u_kk
    if (zero_e(ek)) {
      if (lane == 0) atomicCAS(status, 0, (int)MP_ERR_DIVZERO);
      return;
    }
    wget<W>(m.A, lu, nnz, ik, ea, sa, lane);  // a_ik
    int64_t el = EXP_ZERO;
    const uint32_t sl = sa ^ sk;
    if (!zero_e(ea)) el = wdiv<W>(m.A, ea, m.X, ek, u.U, m.cnt, u.Q, u.S, u.L, lane);
    __syncwarp();
    wstore<W>(u.L, el, sl, lu, nnz, ik, lane);  // l_ik
    int64_t q = diag[k] + 1;  // row k's entries right of its diagonal
    const int64_t qe = rowptr[k + 1];
    for (int64_t ij = ik + 1; ij < b; ++ij) {
      const int32_t j = col[ij];
      while (q < qe && col[q] < j) ++q;
      if (q >= qe) break;
      if (col[q] != j) continue;
      int64_t ekj, eij;
      uint32_t skj, sij;
      wget<W>(m.X, lu, nnz, q, ekj, skj, lane);   // u_kj
      wget<W>(m.Y, lu, nnz, ij, eij, sij, lane);  // a_ij
      wsub_prod<W>(m.Y, eij, sij, u.L, el, sl, m.X, ekj, skj, m, lane);
      wstore<W>(m.Y, eij, sij, lu, nnz, ij, lane);
      __syncwarp();
    }
  }
  int64_t ed;
  uint32_t sd;
  wget<W>(m.X, lu, nnz, diag[i], ed, sd, lane);
  if (zero_e(ed) && lane == 0) atomicCAS(status, 0, (int)MP_ERR_DIVZERO);
}

// One level of the forward (UPPER = false: y_i into w from r) or backward
// (UPPER = true: w_i in place) solve.
template <int W, bool UPPER>
__global__ void __launch_bounds__(kBigThreads) big_trsv_level_kernel(
    const int32_t* __restrict__ rows, int64_t count, const int64_t* __restrict__ rowptr,
    const int32_t* __restrict__ col, const int64_t* __restrict__ diag, const uint64_t* lu,
    int64_t nnz, const uint64_t* r, int64_t ldr, uint64_t* w, int64_t ldw,
    const int* __restrict__ gate) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (gate && *gate) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t t = (int64_t)blockIdx.x * kBigWarps + warp;
  if (t >= count) return;
  const IluWarp u = ilu_carve<W>(smem, warp);
  const WarpMem& m = u.m;
  const int32_t i = rows[t];
  int64_t ey;
  uint32_t sy;
  if (UPPER)
    wget<W>(m.Y, w, ldw, i, ey, sy, lane);
  else
    wget<W>(m.Y, r, ldr, i, ey, sy, lane);
  const int64_t k0 = UPPER ? diag[i] + 1 : rowptr[i];
  const int64_t k1 = UPPER ? rowptr[i + 1] : diag[i];  // sorted columns: diag splits L and U
  for (int64_t k = k0; k < k1; ++k) {
    int64_t ea, ex;
    uint32_t sa, sx;
    wget<W>(m.A, lu, nnz, k, ea, sa, lane);
    wget<W>(m.X, w, ldw, col[k], ex, sx, lane);
    wsub_prod<W>(m.Y, ey, sy, m.A, ea, sa, m.X, ex, sx, m, lane);
  }
  if (!UPPER) {
    wstore<W>(m.Y, ey, sy, w, ldw, i, lane);
    return;
  }
  int64_t ed;
  uint32_t sd;
  wget<W>(m.X, lu, nnz, diag[i], ed, sd, lane);  // nonzero: checked when the factor was built
  int64_t eq = EXP_ZERO;
  if (!zero_e(ey)) eq = wdiv<W>(m.Y, ey, m.X, ed, u.U, m.cnt, u.Q, u.S, m.T, lane);
  __syncwarp();
  wstore<W>(m.T, eq, sy ^ sd, w, ldw, i, lane);
}

int grid_for(int64_t count) { return (int)((count + kBigWarps - 1) / kBigWarps); }

template <int W>
mp_status factor_w(const mp_ilu_s* M, int* status, cudaStream_t st) {
  const size_t sm = (size_t)kBigWarps * IluMem<W>::kBytes;
  MPK_CUDA(cudaFuncSetAttribute(big_ilu_level_kernel<W>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  for (int64_t l = 0; l < M->nl; ++l) {
    const int64_t cnt = M->lvl_l[l + 1] - M->lvl_l[l];
    big_ilu_level_kernel<W><<<grid_for(cnt), kBigThreads, sm, st>>>(
        M->rows_l + M->lvl_l[l], cnt, M->rowptr, M->col, M->diag, M->lu, M->nnz, status);
  }
  count_launch((int)M->nl);
  return launch_check("big_ilu_level_kernel");
}

template <int W>
mp_status apply_w(const mp_ilu_s* M, const uint64_t* r, int64_t ldr, uint64_t* w, int64_t ldw,
                  const int* gate, cudaStream_t st) {
  const size_t sm = (size_t)kBigWarps * IluMem<W>::kBytes;
  MPK_CUDA(cudaFuncSetAttribute(big_trsv_level_kernel<W, false>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  MPK_CUDA(cudaFuncSetAttribute(big_trsv_level_kernel<W, true>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  for (int64_t l = 0; l < M->nl; ++l) {
    const int64_t cnt = M->lvl_l[l + 1] - M->lvl_l[l];
    big_trsv_level_kernel<W, false><<<grid_for(cnt), kBigThreads, sm, st>>>(
        M->rows_l + M->lvl_l[l], cnt, M->rowptr, M->col, M->diag, M->lu, M->nnz, r, ldr, w, ldw,
        gate);
  }
  for (int64_t l = 0; l < M->nu; ++l) {
    const int64_t cnt = M->lvl_u[l + 1] - M->lvl_u[l];
    big_trsv_level_kernel<W, true><<<grid_for(cnt), kBigThreads, sm, st>>>(
        M->rows_u + M->lvl_u[l], cnt, M->rowptr, M->col, M->diag, M->lu, M->nnz, r, ldr, w, ldw,
        gate);
  }
  count_launch((int)(M->nl + M->nu));
  return launch_check("big_trsv_level_kernel");
}

}  // namespace

mp_status launch_ilu0_factor_big(const mp_ilu_s* M, int* status, cudaStream_t st) {
  switch (M->prec) {
    case 2048: return factor_w<64>(M, status, st);
    case 4096: return factor_w<128>(M, status, st);
    case 8192: return factor_w<256>(M, status, st);
    default: return set_error(MP_ERR_PREC, "precision %d", M->prec);
  }
}

mp_status launch_ilu0_apply_big(const mp_ilu_s* M, const uint64_t* r, int64_t ldr, uint64_t* w,
                                int64_t ldw, const int* gate, cudaStream_t st) {
  switch (M->prec) {
    case 2048: return apply_w<64>(M, r, ldr, w, ldw, gate, st);
    case 4096: return apply_w<128>(M, r, ldr, w, ldw, gate, st);
    case 8192: return apply_w<256>(M, r, ldr, w, ldw, gate, st);
    default: return set_error(MP_ERR_PREC, "precision %d", M->prec);
  }
}

}  // namespace mpk
