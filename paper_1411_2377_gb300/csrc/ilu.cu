// ilu.cu -- ILU(0) preconditioning (Section 4's BiCGSTAB+ILU(0) rows; the
// paper prints no algorithm, the textbook IKJ form is taken).
//
// The factors share A's pattern and live in CSR order (sorted columns):
// L (unit lower) left of the diagonal, U from it.  Rows are grouped into
// levels of the dependency graph (row i needs every row k < i that it
// stores for the factorisation and the forward solve; every row k > i for
// the backward solve), and each level is one launch of one thread per row,
// so every row reads only rows that earlier launches finished.  Within a row
// the arithmetic is the oracle's, step for step:
//   factorisation: for stored (i, k), k < i ascending: l_ik = RN(a_ik/u_kk),
//     then for stored (i, j), j > k ascending, with (k, j) stored:
//     a_ij = RN(a_ij - RN(l_ik u_kj));
//   forward:  y_i = r_i - RN(l_ik y_k) for k < i ascending, rounded per step;
//   backward: w_i = RN((y_i - RN(u_ik w_k) for k > i ascending) / u_ii).
// Nothing is skipped (zero products included), so signed zeros follow the
// same steps as in the oracle.  At p = 2048-8192 the factorisation and the
// solves are bigp_ilu.cu's warp-per-row kernels on the same storage.
#include <algorithm>
#include <vector>

#include "internal.h"
#include "mpdev.cuh"

namespace mpk {
namespace {

// Plain (weak) loads, for data the same kernel writes: a row's own factor
// entries in the factorisation (written by the same thread) and w in the
// one-block solves (written by threads of the same block before a barrier,
// which orders them for every load of the block).  Only the read-only path
// (ld.global.nc, what load() uses) may not see such writes.
template <int W>
__device__ __forceinline__ void load_w(Num<W>& a, const uint64_t* w, int64_t ld, int64_t i) {
  unpack_head(w[i], a.e, a.s);
#pragma unroll
  for (int k = 0; k < W / 2; ++k) {
    const uint64_t l = w[(int64_t)(k + 1) * ld + i];
    a.m[2 * k] = (uint32_t)l;
    a.m[2 * k + 1] = (uint32_t)(l >> 32);
  }
}

// acc <- RN(acc - RN(f_k z_k)) for k = k0, ..., k1 - 1 in turn (f the factor
// entries, z = w at their columns): the products do not depend on acc, so
// their loads and multiplications run in batches of B (4, 2 or 1 by the
// registers a value takes), then the batch's subtractions in order.  WL:
// load w with plain loads (the one-block solves, where this kernel wrote it).
template <int W, bool WL>
__device__ __forceinline__ void sub_products(Num<W>& acc, const uint64_t* __restrict__ lu,
                                             int64_t nnz, const int32_t* __restrict__ col,
                                             const uint64_t* w, int64_t ldw, int64_t k0,
                                             int64_t k1) {
  constexpr int B = W <= 8 ? 4 : (W <= 16 ? 2 : 1);
  for (int64_t k = k0; k < k1; k += B) {
    Num<W> pr[B];
#pragma unroll
    for (int u = 0; u < B; ++u) {
      if (k + u < k1) {
        Num<W> f, z;
        load<W>(f, lu, nnz, k + u);
        if (WL)
          load_w<W>(z, w, ldw, col[k + u]);
        else
          load<W>(z, w, ldw, col[k + u]);
        mul_rn_fast<W>(f, z, pr[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < B; ++u) {
      if (k + u < k1) {
        Num<W> t;
        sub_rn<W>(acc, pr[u], t);
        acc = t;
      }
    }
  }
}

// Sliced layout -> CSR order: thread per (chunk, lane) row; `planes` words
// per value (head and limbs).
__global__ void to_csr_kernel(int64_t nchunks, const int64_t* __restrict__ chunk_off,
                              const int32_t* __restrict__ row_of,
                              const int32_t* __restrict__ row_len,
                              const int32_t* __restrict__ scol, const uint64_t* __restrict__ sval,
                              int64_t nslots, const int64_t* __restrict__ rowptr,
                              int32_t* __restrict__ col, uint64_t* __restrict__ lu, int64_t nnz,
                              int planes) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nchunks * 32) return;
  const int64_t c = t >> 5;
  const int lane = (int)(t & 31);
  const int32_t row = row_of[t];
  if (row < 0) return;
  const int32_t len = row_len[t];
  for (int32_t j = 0; j < len; ++j) {
    const int64_t s = chunk_off[c] + (int64_t)j * 32 + lane;
    const int64_t k = rowptr[row] + j;
    col[k] = scol[s];
    for (int q = 0; q < planes; ++q) lu[(int64_t)q * nnz + k] = sval[(int64_t)q * nslots + s];
  }
}

template <int W>
__global__ void ilu_level_kernel(const int32_t* __restrict__ rows, int64_t count,
                                 const int64_t* __restrict__ rowptr,
                                 const int32_t* __restrict__ col, const int64_t* __restrict__ diag,
                                 uint64_t* __restrict__ lu, int64_t nnz, int* status) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= count) return;
  const int32_t i = rows[t];
  const int64_t a = rowptr[i], b = rowptr[i + 1];
  for (int64_t ik = a; ik < b && col[ik] < i; ++ik) {
    const int32_t k = col[ik];
    Num<W> ukk, aik, l;
    load_w<W>(ukk, lu, nnz, diag[k]);
    if (zero_e(ukk.e)) {
      atomicCAS(status, 0, (int)MP_ERR_DIVZERO);
      return;
    }
    load_w<W>(aik, lu, nnz, ik);
    div_rn<W>(aik, ukk, l);
    store<W>(l, lu, nnz, ik);
    int64_t q = diag[k] + 1;  // row k's entries right of its diagonal
    const int64_t qe = rowptr[k + 1];
    for (int64_t ij = ik + 1; ij < b; ++ij) {
      const int32_t j = col[ij];
      while (q < qe && col[q] < j) ++q;
      if (q >= qe) break;
      if (col[q] != j) continue;
      Num<W> ukj, aij, t1, t2;
      load_w<W>(ukj, lu, nnz, q);
      load_w<W>(aij, lu, nnz, ij);
      mul_rn_fast<W>(l, ukj, t1);
      sub_rn<W>(aij, t1, t2);
      store<W>(t2, lu, nnz, ij);
    }
  }
  Num<W> d;
  load_w<W>(d, lu, nnz, diag[i]);
  if (zero_e(d.e)) atomicCAS(status, 0, (int)MP_ERR_DIVZERO);
}

template <int W>
__global__ void lsolve_level_kernel(const int32_t* __restrict__ rows, int64_t count,
                                    const int64_t* __restrict__ rowptr,
                                    const int32_t* __restrict__ col,
                                    const int64_t* __restrict__ diag,
                                    const uint64_t* __restrict__ lu, int64_t nnz,
                                    const uint64_t* __restrict__ r, int64_t ldr, uint64_t* w,
                                    int64_t ldw, const int* __restrict__ gate) {
  if (gate && *gate) return;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= count) return;
  const int32_t i = rows[t];
  Num<W> acc;
  load<W>(acc, r, ldr, i);
  sub_products<W, false>(acc, lu, nnz, col, w, ldw, rowptr[i], diag[i]);  // k < i: left of (i, i)
  store<W>(acc, w, ldw, i);
}

template <int W>
__global__ void usolve_level_kernel(const int32_t* __restrict__ rows, int64_t count,
                                    const int64_t* __restrict__ rowptr,
                                    const int32_t* __restrict__ col,
                                    const int64_t* __restrict__ diag,
                                    const uint64_t* __restrict__ lu, int64_t nnz, uint64_t* w,
                                    int64_t ldw, const int* __restrict__ gate) {
  if (gate && *gate) return;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= count) return;
  const int32_t i = rows[t];
  Num<W> acc, d, q;
  load<W>(acc, w, ldw, i);
  sub_products<W, false>(acc, lu, nnz, col, w, ldw, diag[i] + 1, rowptr[i + 1]);
  load<W>(d, lu, nnz, diag[i]);  // nonzero: checked when the factor was built
  div_rn<W>(acc, d, q);
  store<W>(q, w, ldw, i);
}

// The whole forward (L) or backward (U) solve in one block: the levels in
// order, the rows of a level spread over the threads, a block barrier
// between levels (a row's inputs are rows of earlier levels, written by
// threads of this block before the barrier).  One launch instead of one per
// level, for matrices small enough that one block keeps up.
template <int W, bool UPPER>
__global__ void __launch_bounds__(256) trsv_block_kernel(
    const int32_t* __restrict__ rows, const int64_t* __restrict__ lvl, int64_t nlev,
    const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
    const int64_t* __restrict__ diag, const uint64_t* __restrict__ lu, int64_t nnz,
    const uint64_t* __restrict__ r, int64_t ldr, uint64_t* w, int64_t ldw,
    const int* __restrict__ gate) {
  if (gate && *gate) return;
  for (int64_t l = 0; l < nlev; ++l) {
    const int64_t a = lvl[l], b = lvl[l + 1];
    for (int64_t t = a + threadIdx.x; t < b; t += blockDim.x) {
      const int32_t i = rows[t];
      Num<W> acc;
      if (UPPER) {
        load_w<W>(acc, w, ldw, i);
        sub_products<W, true>(acc, lu, nnz, col, w, ldw, diag[i] + 1, rowptr[i + 1]);
        Num<W> d, q;
        load<W>(d, lu, nnz, diag[i]);
        div_rn<W>(acc, d, q);
        store<W>(q, w, ldw, i);
      } else {
        load<W>(acc, r, ldr, i);
        sub_products<W, true>(acc, lu, nnz, col, w, ldw, rowptr[i], diag[i]);
        store<W>(acc, w, ldw, i);
      }
    }
    __syncthreads();
  }
}

int blocks_for(int64_t count, int tpb) { return (int)std::max<int64_t>(1, (count + tpb - 1) / tpb); }

// Up to this many rows the solves run as one block (one launch per solve).
constexpr int64_t kOneBlockRows = 1 << 18;

}  // namespace

mp_status launch_ilu0_apply(const mp_ilu_s* M, const uint64_t* r, int64_t ldr, uint64_t* w,
                            int64_t ldw, const int* gate, cudaStream_t st) {
  if (prec_big(M->prec)) return launch_ilu0_apply_big(M, r, ldr, w, ldw, gate, st);
  return dispatch_w(M->prec, [&](auto wc) {
    constexpr int W = decltype(wc)::value;
    constexpr int tpb = 64;
    if (M->n <= kOneBlockRows) {
      trsv_block_kernel<W, false><<<1, 256, 0, st>>>(M->rows_l, M->d_lvl_l, M->nl, M->rowptr,
                                                     M->col, M->diag, M->lu, M->nnz, r, ldr, w,
                                                     ldw, gate);
      trsv_block_kernel<W, true><<<1, 256, 0, st>>>(M->rows_u, M->d_lvl_u, M->nu, M->rowptr,
                                                    M->col, M->diag, M->lu, M->nnz, r, ldr, w,
                                                    ldw, gate);
      count_launch(2);
      return launch_check("ILU(0) triangular solves");
    }
    for (int64_t l = 0; l < M->nl; ++l) {
      const int64_t cnt = M->lvl_l[l + 1] - M->lvl_l[l];
      lsolve_level_kernel<W><<<blocks_for(cnt, tpb), tpb, 0, st>>>(
          M->rows_l + M->lvl_l[l], cnt, M->rowptr, M->col, M->diag, M->lu, M->nnz, r, ldr, w,
          ldw, gate);
    }
    for (int64_t l = 0; l < M->nu; ++l) {
      const int64_t cnt = M->lvl_u[l + 1] - M->lvl_u[l];
      usolve_level_kernel<W><<<blocks_for(cnt, tpb), tpb, 0, st>>>(
          M->rows_u + M->lvl_u[l], cnt, M->rowptr, M->col, M->diag, M->lu, M->nnz, w, ldw, gate);
    }
    count_launch((int)(M->nl + M->nu));
    return launch_check("ILU(0) triangular solves");
  });
}

}  // namespace mpk

using namespace mpk;

namespace {

void free_ilu(mp_ilu_s* M) {
  if (!M) return;
  cudaFree(M->rowptr);
  cudaFree(M->col);
  cudaFree(M->diag);
  cudaFree(M->lu);
  cudaFree(M->rows_l);
  cudaFree(M->rows_u);
  cudaFree(M->d_lvl_l);
  cudaFree(M->d_lvl_u);
  delete[] M->lvl_l;
  delete[] M->lvl_u;
  delete M;
}

// Rows grouped by level; lvl receives the level boundaries.
void levels(int64_t n, const std::vector<int64_t>& lev, std::vector<int32_t>& rows,
            std::vector<int64_t>& lvl) {
  const int64_t nlev = n > 0 ? *std::max_element(lev.begin(), lev.end()) + 1 : 0;
  lvl.assign(nlev + 1, 0);
  for (int64_t i = 0; i < n; ++i) lvl[lev[i] + 1]++;
  for (int64_t l = 0; l < nlev; ++l) lvl[l + 1] += lvl[l];
  std::vector<int64_t> next(lvl.begin(), lvl.end() - 1);
  rows.assign(n, 0);
  for (int64_t i = 0; i < n; ++i) rows[next[lev[i]]++] = (int32_t)i;
}

}  // namespace

extern "C" {

mp_status mp_ilu0_create(mp_csr A, void* stream, mp_ilu* out) {
  if (!A || !out) return set_error(MP_ERR_ARG, "matrix or out is null");
  *out = nullptr;
  if (!prec_ok(A->prec) && !prec_big(A->prec))
    return set_error(MP_ERR_PREC, "ILU(0) at p = %d", A->prec);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t n = A->n, nnz = A->nnz, nch = A->A.nchunks;
  const int L = A->prec / 64;
  // the pattern back in CSR order, on the host
  std::vector<int64_t> coff(nch + 1);
  std::vector<int32_t> rof(nch * 32), rlen(nch * 32);
  if (nch > 0) {
    MPK_CUDA(cudaMemcpyAsync(coff.data(), A->A.chunk_off, sizeof(int64_t) * (nch + 1),
                             cudaMemcpyDeviceToHost, st));
    MPK_CUDA(cudaMemcpyAsync(rof.data(), A->A.row_of, sizeof(int32_t) * nch * 32,
                             cudaMemcpyDeviceToHost, st));
    MPK_CUDA(cudaMemcpyAsync(rlen.data(), A->A.row_len, sizeof(int32_t) * nch * 32,
                             cudaMemcpyDeviceToHost, st));
    MPK_CUDA(cudaStreamSynchronize(st));
  }
  std::vector<int64_t> rowptr(n + 1, 0);
  for (int64_t t = 0; t < nch * 32; ++t)
    if (rof[t] >= 0) rowptr[rof[t] + 1] = rlen[t];
  for (int64_t i = 0; i < n; ++i) rowptr[i + 1] += rowptr[i];
  mp_ilu_s* M = new (std::nothrow) mp_ilu_s;
  if (!M) return set_error(MP_ERR_ALLOC, "host allocation failed");
  M->n = n;
  M->nnz = nnz;
  M->prec = A->prec;
  auto fail = [&](mp_status s) {
    cudaStreamSynchronize(st);
    free_ilu(M);
    return s;
  };
  if (cudaError_t ce = cudaGetDevice(&M->device)) return fail(cuda_error(ce, "cudaGetDevice"));
  auto dmalloc = [&](auto** p, size_t count) -> bool {
    return cudaMalloc((void**)p, sizeof(**p) * std::max<size_t>(count, 1)) == cudaSuccess;
  };
  if (!dmalloc(&M->rowptr, n + 1) || !dmalloc(&M->col, nnz) || !dmalloc(&M->diag, n) ||
      !dmalloc(&M->lu, (size_t)(L + 1) * nnz))
    return fail(set_error(MP_ERR_ALLOC, "ILU(0) factor"));
  if (cudaMemcpyAsync(M->rowptr, rowptr.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice,
                      st) != cudaSuccess)
    return fail(set_error(MP_ERR_CUDA, "ILU(0) upload"));
  if (nch > 0) {
    to_csr_kernel<<<blocks_for(nch * 32, 128), 128, 0, st>>>(
        nch, A->A.chunk_off, A->A.row_of, A->A.row_len, A->A.col, A->A.val, A->A.nslots,
        M->rowptr, M->col, M->lu, nnz, L + 1);
    count_launch();
  }
  mp_status r = launch_check("to_csr_kernel");
  if (r != MP_OK) return fail(r);
  std::vector<int32_t> col(nnz);
  if (nnz > 0 && (cudaMemcpyAsync(col.data(), M->col, sizeof(int32_t) * nnz,
                                  cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                  cudaStreamSynchronize(st) != cudaSuccess))
    return fail(set_error(MP_ERR_CUDA, "ILU(0) pattern"));
  // diagonal positions and level schedules
  std::vector<int64_t> diag(n, -1), levl(n, 0), levu(n, 0);
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      if (col[k] == i) diag[i] = k;
      if (col[k] < i) levl[i] = std::max(levl[i], levl[col[k]] + 1);
    }
    if (diag[i] < 0) return fail(set_error(MP_ERR_DIVZERO, "ILU(0): row %lld has no diagonal entry", (long long)i));
  }
  for (int64_t i = n - 1; i >= 0; --i)
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
      if (col[k] > i) levu[i] = std::max(levu[i], levu[col[k]] + 1);
  std::vector<int32_t> rl, ru;
  std::vector<int64_t> ll, lu_;
  levels(n, levl, rl, ll);
  levels(n, levu, ru, lu_);
  M->nl = (int64_t)ll.size() - 1;
  M->nu = (int64_t)lu_.size() - 1;
  M->lvl_l = new (std::nothrow) int64_t[ll.size()];
  M->lvl_u = new (std::nothrow) int64_t[lu_.size()];
  if (!M->lvl_l || !M->lvl_u) return fail(set_error(MP_ERR_ALLOC, "ILU(0) levels"));
  std::copy(ll.begin(), ll.end(), M->lvl_l);
  std::copy(lu_.begin(), lu_.end(), M->lvl_u);
  if (!dmalloc(&M->rows_l, n) || !dmalloc(&M->rows_u, n) || !dmalloc(&M->d_lvl_l, ll.size()) ||
      !dmalloc(&M->d_lvl_u, lu_.size()))
    return fail(set_error(MP_ERR_ALLOC, "ILU(0) levels"));
  if (cudaMemcpyAsync(M->d_lvl_l, ll.data(), sizeof(int64_t) * ll.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(M->d_lvl_u, lu_.data(), sizeof(int64_t) * lu_.size(), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return fail(set_error(MP_ERR_CUDA, "ILU(0) upload"));
  if (n > 0 && (cudaMemcpyAsync(M->diag, diag.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, st) != cudaSuccess ||
                cudaMemcpyAsync(M->rows_l, rl.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st) != cudaSuccess ||
                cudaMemcpyAsync(M->rows_u, ru.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st) != cudaSuccess))
    return fail(set_error(MP_ERR_CUDA, "ILU(0) upload"));
  int* status = status_word();
  if (!status) return fail(set_error(MP_ERR_CUDA, "status word unavailable"));
  int* dz = nullptr;
  if (!dmalloc(&dz, 1) || cudaMemsetAsync(dz, 0, sizeof(int), st) != cudaSuccess) {
    cudaFree(dz);
    return fail(set_error(MP_ERR_ALLOC, "ILU(0) status"));
  }
  if (prec_big(A->prec)) r = launch_ilu0_factor_big(M, dz, st);
  else r = dispatch_w(A->prec, [&](auto w) {
    constexpr int W = decltype(w)::value;
    for (int64_t l = 0; l < M->nl; ++l) {
      const int64_t cnt = M->lvl_l[l + 1] - M->lvl_l[l];
      ilu_level_kernel<W><<<blocks_for(cnt, 64), 64, 0, st>>>(
          M->rows_l + M->lvl_l[l], cnt, M->rowptr, M->col, M->diag, M->lu, nnz, dz);
    }
    count_launch((int)M->nl);
    return launch_check("ilu_level_kernel");
  });
  int hz = 0;
  if (r == MP_OK && (cudaMemcpyAsync(&hz, dz, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                     cudaStreamSynchronize(st) != cudaSuccess))
    r = set_error(MP_ERR_CUDA, "ILU(0) factorisation");
  cudaFree(dz);
  if (r != MP_OK) return fail(r);
  if (hz != 0) return fail(set_error(MP_ERR_DIVZERO, "ILU(0): zero pivot"));
  *out = M;
  return MP_OK;
}

mp_status mp_ilu0_destroy(mp_ilu M) {
  if (!M) return MP_OK;
  cudaDeviceSynchronize();
  free_ilu(M);
  return MP_OK;
}

mp_status mp_ilu0_info(mp_ilu M, int64_t* levels_l, int64_t* levels_u) {
  if (!M) return set_error(MP_ERR_ARG, "factor is null");
  if (levels_l) *levels_l = M->nl;
  if (levels_u) *levels_u = M->nu;
  return MP_OK;
}

mp_status mp_ilu0_factor(mp_ilu M, mp_vec lu, void* stream) {
  if (!M) return set_error(MP_ERR_ARG, "factor is null");
  mp_status r;
  if ((r = check_vec(lu, M->nnz, M->prec, "lu")) != MP_OK) return r;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (int q = 0; q <= M->prec / 64; ++q)
    if (M->nnz > 0)
      MPK_CUDA(cudaMemcpyAsync(lu.data + (int64_t)q * lu.ld, M->lu + (int64_t)q * M->nnz,
                               sizeof(uint64_t) * M->nnz, cudaMemcpyDeviceToDevice, st));
  return MP_OK;
}

mp_status mp_ilu0_apply(mp_ilu M, mp_vec r, mp_vec w, void* stream) {
  if (!M) return set_error(MP_ERR_ARG, "factor is null");
  mp_status s;
  if ((s = check_vec(r, M->n, M->prec, "r")) != MP_OK) return s;
  if ((s = check_vec(w, M->n, M->prec, "w")) != MP_OK) return s;
  if (M->n > 0 && r.data == w.data) return set_error(MP_ERR_ARG, "r and w must not alias");
  return launch_ilu0_apply(M, r.data, r.ld, w.data, w.ld, nullptr, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
