// csr.cu -- building the device matrix (Section 2's CSR storage at p bits).
//
// The host orders rows and chunks (O(n): row lengths only) and, for the rare
// rows whose columns are not strictly increasing, sorts them.  Everything per
// entry runs on the device: the column checks, the placement of each entry
// in the sliced row-length-sorted layout (SELL-32-sigma), the gather of the
// p-bit values into it, the estimate of how scattered the x gathers are, and
// A^T by a counting sort (atomics for the counts and positions, then each
// row of A^T sorted by original row, so the result does not depend on the
// order the atomics ran in).  The caller's arrays are uploaded once.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "internal.h"
#include "mpdev.cuh"

namespace mpk {
namespace {

// First index of a malformed raw value (or INT64_MAX): a head whose exponent
// is the zero sentinel needs zero limbs; any other needs a top limb with its
// top bit set and |e| < 2^60.
__global__ void validate_values(const uint64_t* __restrict__ v, int64_t nnz, int L,
                                unsigned long long* bad) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz;
       k += (int64_t)gridDim.x * blockDim.x) {
    int64_t e;
    uint32_t s;
    unpack_head(v[k], e, s);
    bool ok;
    if (e == EXP_ZERO) {
      uint64_t any = 0;
      for (int j = 1; j <= L; ++j) any |= v[(int64_t)j * nnz + k];
      ok = any == 0;
    } else {
      const int64_t lim = int64_t(1) << 60;
      ok = (v[(int64_t)L * nnz + k] >> 63) != 0 && e < lim && e > -lim;
    }
    if (!ok) atomicMin(bad, (unsigned long long)k);
  }
}

template <int W>
__global__ void f64_to_planes(const double* __restrict__ d, int64_t n, uint64_t* __restrict__ out,
                              unsigned long long* bad) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double v = d[k];
    if (!isfinite(v)) atomicMin(bad, (unsigned long long)k);
    Num<W> r;
    from_f64<W>(isfinite(v) ? v : 0.0, r);
    store<W>(r, out, n, k);
  }
}

// The same for p > 1024 (L limbs): a double's 53-bit mantissa m lands in
// the top limb (M = m 2^(p-53)), the other limbs are zero.
__global__ void f64_to_planes_wide(const double* __restrict__ d, int64_t n, int L,
                                   uint64_t* __restrict__ out, unsigned long long* bad) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double v = d[k];
    uint64_t top = 0;
    int64_t e = EXP_ZERO;
    if (!isfinite(v)) {
      atomicMin(bad, (unsigned long long)k);
    } else if (v != 0.0) {
      int ex = 0;
      const double f = frexp(fabs(v), &ex);  // [1/2, 1)
      top = (uint64_t)ldexp(f, 53) << 11;
      e = ex;
    }
    out[k] = pack_head(e, signbit(v) ? 1u : 0u);
    for (int j = 1; j < L; ++j) out[(int64_t)j * n + k] = 0;
    out[(int64_t)L * n + k] = top;
  }
}

// out slot s <- raw value src[s] (padding slots, src = -1, become +0).
__global__ void gather_planes(const uint64_t* __restrict__ raw, int64_t nnz,
                              const int64_t* __restrict__ src, int64_t nslots, int L,
                              uint64_t* __restrict__ out) {
  const uint64_t zero_head = pack_head(EXP_ZERO, 0u);
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nslots;
       s += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = src[s];
    for (int j = 0; j <= L; ++j) {
      uint64_t w = (j == 0) ? zero_head : 0u;
      if (k >= 0) w = raw[(int64_t)j * nnz + k];
      out[(int64_t)j * nslots + s] = w;
    }
  }
}

// ---- index work on the device -------------------------------------------

// Columns of the caller's CSR: the first entry whose column is out of range
// (the smallest such index, by atomicMin) and the number of rows whose
// columns are not strictly increasing (such rows -- unsorted, or with a
// repeated column -- take the host path, which sorts or reports them).
__global__ void check_cols(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                           int64_t n, unsigned long long* first_bad, unsigned int* unsorted) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = rowptr[i], b = rowptr[i + 1];
    bool inc = true;
    for (int64_t k = a; k < b; ++k) {
      const int32_t c = colidx[k];
      if (c < 0 || (int64_t)c >= n) {
        atomicMin(first_bad, (unsigned long long)k);
        break;
      }
      if (k > a && c <= colidx[k - 1]) inc = false;
    }
    if (!inc) atomicAdd(unsorted, 1u);
  }
}

// The sliced layout's index arrays: slot chunk_off[c] + 32 j + t holds entry
// j of row row_of[32 c + t] -- its column and its raw value index (srcs[k],
// or the CSR index k itself when srcs is null); padding slots hold column 0
// and index -1.  One warp per chunk, so each store of 32 slots is coalesced.
__global__ void fill_slots(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ cols,
                           const int64_t* __restrict__ srcs, const int64_t* __restrict__ chunk_off,
                           const int32_t* __restrict__ row_of, const int32_t* __restrict__ row_len,
                           int64_t nchunks, int32_t* __restrict__ col, int64_t* __restrict__ src) {
  const int t = threadIdx.x & 31;
  for (int64_t c = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; c < nchunks;
       c += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int32_t r = row_of[c * 32 + t];
    const int32_t len = r >= 0 ? row_len[c * 32 + t] : 0;
    const int64_t k0 = r >= 0 ? rowptr[r] : 0;
    const int64_t clen = (chunk_off[c + 1] - chunk_off[c]) / 32;
    for (int64_t j = 0; j < clen; ++j) {
      const int64_t s = chunk_off[c] + 32 * j + t;
      if (j < len) {
        const int64_t k = k0 + j;
        col[s] = cols[k];
        src[s] = srcs ? srcs[k] : k;
      } else {
        col[s] = 0;
        src[s] = -1;
      }
    }
  }
}

// How scattered the x gathers are, on every fourth chunk: for each entry
// column j of the chunk, the number of distinct 4-element groups (col >> 2)
// among the lanes that hold an entry (summed into touched) and one count per
// such column (groups).  Integer sums: the same totals in any order.
__global__ void gather_groups(const int64_t* __restrict__ chunk_off,
                              const int32_t* __restrict__ row_len, const int32_t* __restrict__ col,
                              int64_t nchunks, unsigned long long* touched,
                              unsigned long long* groups) {
  const int t = threadIdx.x & 31;
  unsigned long long tc = 0, gc = 0;
  for (int64_t c4 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; 4 * c4 < nchunks;
       c4 += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int64_t c = 4 * c4;
    const int64_t clen = (chunk_off[c + 1] - chunk_off[c]) / 32;
    const int32_t len = row_len[c * 32 + t];
    for (int64_t j = 0; j < clen; ++j) {
      const bool active = j < len;
      const unsigned int any = __ballot_sync(0xffffffffu, active);
      if (any == 0u) continue;
      const int key = active ? (col[chunk_off[c] + 32 * j + t] >> 2) : -1 - t;
      const unsigned int same = __match_any_sync(0xffffffffu, key);
      const bool leader = (same & ((1u << t) - 1u)) == 0u;
      tc += __popc(__ballot_sync(0xffffffffu, active && leader));
      gc += 1;
    }
  }
  if (t == 0 && gc) {
    atomicAdd(touched, tc);
    atomicAdd(groups, gc);
  }
}

// A^T by a counting sort on the device: column counts (atomics: the counts
// do not depend on the order), a scatter of each entry to its column's row
// of A^T (positions by atomics: any order), then each row of A^T sorted by
// the original row index (unique within the row), so the result does not
// depend on the order of the scatter.
__global__ void col_counts(const int32_t* __restrict__ cols, int64_t nnz,
                           unsigned long long* __restrict__ cnt) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz;
       k += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&cnt[cols[k]], 1ull);
}

__global__ void scatter_t(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ cols,
                          const int64_t* __restrict__ srcs, int64_t n,
                          const int64_t* __restrict__ tptr, unsigned long long* __restrict__ next,
                          int32_t* __restrict__ tcols, int64_t* __restrict__ tsrc) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      const int32_t c = cols[k];
      const int64_t pos = tptr[c] + (int64_t)atomicAdd(&next[c], 1ull);
      tcols[pos] = (int32_t)i;
      tsrc[pos] = srcs ? srcs[k] : k;
    }
  }
}

constexpr int64_t kRowSortMax = 256;  // longer rows of A^T are sorted on the host

__global__ void sort_rows_t(const int64_t* __restrict__ tptr, int64_t n, int32_t* __restrict__ tcols,
                            int64_t* __restrict__ tsrc, unsigned int* long_rows) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = tptr[j], b = tptr[j + 1];
    if (b - a > kRowSortMax) {
      atomicAdd(long_rows, 1u);
      continue;
    }
    for (int64_t k = a + 1; k < b; ++k) {  // insertion sort by original row
      const int32_t key = tcols[k];
      const int64_t v = tsrc[k];
      int64_t m = k - 1;
      while (m >= a && tcols[m] > key) {
        tcols[m + 1] = tcols[m];
        tsrc[m + 1] = tsrc[m];
        --m;
      }
      tcols[m + 1] = key;
      tsrc[m + 1] = v;
    }
  }
}

int grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 65535LL * 8) b = 65535LL * 8;
  return (int)b;
}

struct HostSell {
  int64_t nslots = 0, nchunks = 0;
  std::vector<int64_t> chunk_off;
  std::vector<int32_t> row_of, row_len;
};

// The sliced layout's row and chunk order, from the row lengths alone:
// rows sorted longest first inside each sigma window (stable), 32 rows per
// chunk, chunks laid out longest first across the whole matrix so that the
// long sequential row chains start at the beginning of a launch instead of
// forming its tail (each chunk keeps its 32 rows from one sigma window: x
// locality within the chunk).  The entries themselves are placed on the
// device (fill_slots).
void build_sell_meta(int64_t n, const int64_t* rowptr, HostSell& h) {
  std::vector<int32_t> perm(n);
  std::iota(perm.begin(), perm.end(), 0);
  for (int64_t w0 = 0; w0 < n; w0 += kSigma) {
    const int64_t w1 = std::min<int64_t>(n, w0 + kSigma);
    std::stable_sort(perm.begin() + w0, perm.begin() + w1, [&](int32_t a, int32_t b) {
      return (rowptr[a + 1] - rowptr[a]) > (rowptr[b + 1] - rowptr[b]);
    });
  }
  h.nchunks = (n + 31) / 32;
  std::vector<int64_t> clen(h.nchunks, 0);
  for (int64_t c = 0; c < h.nchunks; ++c)
    for (int t = 0; t < 32 && c * 32 + t < n; ++t) {
      const int32_t r = perm[c * 32 + t];
      clen[c] = std::max<int64_t>(clen[c], rowptr[r + 1] - rowptr[r]);
    }
  std::vector<int64_t> corder(h.nchunks);
  std::iota(corder.begin(), corder.end(), 0);
  std::stable_sort(corder.begin(), corder.end(),
                   [&](int64_t a, int64_t b) { return clen[a] > clen[b]; });
  h.chunk_off.assign(h.nchunks + 1, 0);
  h.row_of.assign(h.nchunks * 32, -1);
  h.row_len.assign(h.nchunks * 32, 0);
  for (int64_t c = 0; c < h.nchunks; ++c) {
    const int64_t src_chunk = corder[c];
    for (int t = 0; t < 32; ++t) {
      const int64_t i = src_chunk * 32 + t;
      if (i >= n) break;
      const int32_t r = perm[i];
      h.row_of[c * 32 + t] = r;
      h.row_len[c * 32 + t] = (int32_t)(rowptr[r + 1] - rowptr[r]);
    }
    h.chunk_off[c + 1] = h.chunk_off[c] + 32 * clen[src_chunk];
  }
  h.nslots = h.chunk_off[h.nchunks];
}

template <class T>
mp_status dalloc(T** p, size_t count, int64_t& bytes) {
  *p = nullptr;
  const size_t b = std::max<size_t>(count, 1) * sizeof(T);
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), b);
  if (e != cudaSuccess) return cuda_error(e, "cudaMalloc");
  bytes += (int64_t)b;
  return MP_OK;
}

void free_sell(Sell& s) {
  cudaFree(s.chunk_off);
  cudaFree(s.row_of);
  cudaFree(s.row_len);
  cudaFree(s.col);
  cudaFree(s.val);
  cudaFree(s.src);
  s = Sell{};
}

// Device storage of one sliced matrix: the row and chunk order from the
// host, the entries placed by fill_slots from the device CSR (d_rowptr,
// d_cols, d_srcs: null = entry k is raw value k), the p-bit values gathered
// from the caller's raw planes.
mp_status make_sell(const HostSell& h, int64_t n, int64_t nnz, int L, const int64_t* d_rowptr,
                    const int32_t* d_cols, const int64_t* d_srcs, const uint64_t* d_raw,
                    cudaStream_t st, Sell& S, int64_t& bytes) {
  S.n = n;
  S.nnz = nnz;
  S.nslots = h.nslots;
  S.nchunks = h.nchunks;
  mp_status r;
  if ((r = dalloc(&S.chunk_off, h.chunk_off.size(), bytes)) != MP_OK) return r;
  if ((r = dalloc(&S.row_of, h.row_of.size(), bytes)) != MP_OK) return r;
  if ((r = dalloc(&S.row_len, h.row_len.size(), bytes)) != MP_OK) return r;
  if ((r = dalloc(&S.col, (size_t)h.nslots, bytes)) != MP_OK) return r;
  if ((r = dalloc(&S.val, (size_t)(L + 1) * h.nslots, bytes)) != MP_OK) return r;
  // the slot -> caller position map stays (gradients on the pattern use it)
  if ((r = dalloc(&S.src, (size_t)h.nslots, bytes)) != MP_OK) return r;
  MPK_CUDA(cudaMemcpyAsync(S.chunk_off, h.chunk_off.data(), h.chunk_off.size() * 8,
                           cudaMemcpyHostToDevice, st));
  if (!h.row_of.empty()) {
    MPK_CUDA(cudaMemcpyAsync(S.row_of, h.row_of.data(), h.row_of.size() * 4,
                             cudaMemcpyHostToDevice, st));
    MPK_CUDA(cudaMemcpyAsync(S.row_len, h.row_len.data(), h.row_len.size() * 4,
                             cudaMemcpyHostToDevice, st));
  }
  if (h.nslots > 0) {
    fill_slots<<<grid_for(h.nchunks * 32, 256), 256, 0, st>>>(d_rowptr, d_cols, d_srcs, S.chunk_off,
                                                             S.row_of, S.row_len, h.nchunks, S.col,
                                                             S.src);
    gather_planes<<<grid_for(h.nslots, 256), 256, 0, st>>>(d_raw, nnz, S.src, h.nslots, L, S.val);
    count_launch(2);
    if ((r = launch_check("fill_slots / gather_planes")) != MP_OK) return r;
  }
  MPK_CUDA(cudaStreamSynchronize(st));
  return MP_OK;
}

// Mean number of distinct 4-element groups a warp's gather of one plane of x
// touches (8 when the 32 lanes read consecutive columns, up to 32), sampled
// on every fourth chunk: picks the default gather layout.
mp_status gather_sectors(const Sell& S, cudaStream_t st, double* out) {
  *out = 0.0;
  if (S.nslots == 0) return MP_OK;
  unsigned long long* d = nullptr;
  MPK_CUDA(cudaMalloc(&d, 2 * sizeof(unsigned long long)));
  unsigned long long h[2] = {0, 0};
  cudaError_t e = cudaMemsetAsync(d, 0, sizeof h, st);
  if (e == cudaSuccess) {
    gather_groups<<<grid_for((S.nchunks + 3) / 4 * 32, 256), 256, 0, st>>>(
        S.chunk_off, S.row_len, S.col, S.nchunks, d, d + 1);
    count_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof h, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_error(e, "gather_groups");
  *out = h[1] ? (double)h[0] / (double)h[1] : 0.0;
  return MP_OK;
}

// Shared body of mp_csr_create / mp_csr_create_f64.  Exactly one of
// `values` (planes) and `values64` is non-null.
mp_status create_impl(int64_t n, const int64_t* rowptr, const int32_t* colidx,
                      const uint64_t* values, const double* values64, int32_t prec,
                      int32_t flags, void* stream, mp_csr* out) {
  if (!out) return set_error(MP_ERR_ARG, "out is null");
  *out = nullptr;
  if (!prec_ok(prec) && !prec_big(prec))
    return set_error(MP_ERR_PREC, "precision %d not in {128,256,512,1024,2048,4096,8192}", prec);
  if (n < 0 || n >= (int64_t(1) << 31)) return set_error(MP_ERR_ARG, "n = %lld out of range", (long long)n);
  if (!rowptr) return set_error(MP_ERR_ARG, "rowptr is null");
  if (rowptr[0] != 0) return set_error(MP_ERR_ARG, "rowptr[0] = %lld, expected 0", (long long)rowptr[0]);
  for (int64_t i = 0; i < n; ++i)
    if (rowptr[i + 1] < rowptr[i]) return set_error(MP_ERR_ARG, "row %lld: rowptr decreases", (long long)i);
  const int64_t nnz = rowptr[n];
  if (nnz > 0 && (!colidx || (!values && !values64)))
    return set_error(MP_ERR_ARG, "colidx or values is null");
  if (flags & ~MP_CSR_TRANSPOSE) return set_error(MP_ERR_ARG, "unknown flags %d", flags);
  const int L = prec / 64;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0;
  MPK_CUDA(cudaGetDevice(&dev));

  mp_csr_s* M = new (std::nothrow) mp_csr_s;
  if (!M) return set_error(MP_ERR_ALLOC, "host allocation failed");
  M->n = n;
  M->nnz = nnz;
  M->prec = prec;
  M->device = dev;
  mp_status r = MP_OK;
  uint64_t* d_raw = nullptr;
  unsigned long long* d_bad = nullptr;
  int64_t* d_rowptr = nullptr;
  int32_t* d_colidx = nullptr;
  int32_t* d_cols = nullptr;   // columns in summation order when the host re-sorted rows
  int64_t* d_srcs = nullptr;   // their raw value indices (null: entry k is value k)
  int64_t* d_tptr = nullptr;
  unsigned long long* d_tcnt = nullptr;
  int32_t* d_tcols = nullptr;
  int64_t* d_tsrc = nullptr;
  int64_t tmp = 0;
  auto release = [&]() {
    cudaStreamSynchronize(st);
    cudaFree(d_raw);
    cudaFree(d_bad);
    cudaFree(d_rowptr);
    cudaFree(d_colidx);
    cudaFree(d_cols);
    cudaFree(d_srcs);
    cudaFree(d_tptr);
    cudaFree(d_tcnt);
    cudaFree(d_tcols);
    cudaFree(d_tsrc);
  };
  auto fail = [&](mp_status s) {
    release();
    free_sell(M->A);
    free_sell(M->AT);
    cudaFree(M->ovf);
    cudaFree(M->ovf_t);
    delete M;
    return s;
  };
  auto cuda_fail = [&](cudaError_t e, const char* what) { return fail(cuda_error(e, what)); };

  // Columns, on the device: in range (the first offending entry reported by
  // its row), and strictly increasing per row; rows that are not (unsorted,
  // or with a repeated column) are put in ascending column order on the host
  // (a stable sort per row; a repeated column is an error).
  if ((r = dalloc(&d_rowptr, (size_t)n + 1, tmp)) != MP_OK) return fail(r);
  if ((r = dalloc(&d_colidx, (size_t)nnz, tmp)) != MP_OK) return fail(r);
  {
    cudaError_t e = cudaMemcpyAsync(d_rowptr, rowptr, (size_t)(n + 1) * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && nnz > 0)
      e = cudaMemcpyAsync(d_colidx, colidx, (size_t)nnz * 4, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "index upload");
  }
  if (nnz > 0) {
    unsigned long long* d_chk = nullptr;
    if ((r = dalloc(&d_chk, 2, tmp)) != MP_OK) return fail(r);
    unsigned long long h[2] = {~0ull, 0ull};
    cudaError_t e = cudaMemcpyAsync(d_chk, h, sizeof h, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
      check_cols<<<grid_for(n, 256), 256, 0, st>>>(d_rowptr, d_colidx, n, d_chk,
                                                   reinterpret_cast<unsigned int*>(d_chk + 1));
      count_launch();
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d_chk, sizeof h, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d_chk);
    if (e != cudaSuccess) return cuda_fail(e, "column check");
    if (h[0] != ~0ull) {
      const int64_t k = (int64_t)h[0];
      const int64_t row = std::upper_bound(rowptr, rowptr + n + 1, k) - rowptr - 1;
      return fail(set_error(MP_ERR_ARG, "row %lld: column %d out of range", (long long)row,
                            colidx[k]));
    }
    if ((uint32_t)h[1] != 0u) {  // some rows need the host's sort
      std::vector<int32_t> cols(colidx, colidx + nnz);
      std::vector<int64_t> srcs(nnz);
      std::iota(srcs.begin(), srcs.end(), 0);
      std::vector<int64_t> idx;
      for (int64_t i = 0; i < n; ++i) {
        const int64_t a = rowptr[i], b = rowptr[i + 1];
        bool sorted = true;
        for (int64_t k = a + 1; k < b && sorted; ++k) sorted = colidx[k] > colidx[k - 1];
        if (sorted) continue;
        idx.resize(b - a);
        std::iota(idx.begin(), idx.end(), a);
        std::stable_sort(idx.begin(), idx.end(),
                         [&](int64_t u, int64_t v) { return colidx[u] < colidx[v]; });
        for (int64_t k = a; k < b; ++k) {
          cols[k] = colidx[idx[k - a]];
          srcs[k] = idx[k - a];
          if (k > a && cols[k] == cols[k - 1])
            return fail(set_error(MP_ERR_ARG, "row %lld: column %d repeated", (long long)i,
                                  cols[k]));
        }
      }
      if ((r = dalloc(&d_cols, (size_t)nnz, tmp)) != MP_OK) return fail(r);
      if ((r = dalloc(&d_srcs, (size_t)nnz, tmp)) != MP_OK) return fail(r);
      e = cudaMemcpyAsync(d_cols, cols.data(), (size_t)nnz * 4, cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_srcs, srcs.data(), (size_t)nnz * 8, cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return cuda_fail(e, "sorted column upload");
    }
  }
  const int32_t* cols_dev = d_cols ? d_cols : d_colidx;

  // Values: uploaded once (planes, or doubles converted exactly) and checked.
  if ((r = dalloc(&d_raw, (size_t)(L + 1) * nnz, tmp)) != MP_OK) return fail(r);
  if ((r = dalloc(&d_bad, 1, tmp)) != MP_OK) return fail(r);
  {
    const unsigned long long none = ~0ull;
    cudaError_t e = cudaMemcpyAsync(d_bad, &none, 8, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
  }
  if (nnz > 0) {
    if (values) {
      cudaError_t e = cudaMemcpyAsync(d_raw, values, (size_t)(L + 1) * nnz * 8,
                                      cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(values)");
      validate_values<<<grid_for(nnz, 256), 256, 0, st>>>(d_raw, nnz, L, d_bad);
      count_launch();
    } else {
      double* d64 = nullptr;
      if ((r = dalloc(&d64, nnz, tmp)) != MP_OK) return fail(r);
      const cudaError_t e = cudaMemcpyAsync(d64, values64, (size_t)nnz * 8, cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) {
        cudaFree(d64);
        return cuda_fail(e, "cudaMemcpyAsync(values)");
      }
      if (prec_big(prec)) {
        f64_to_planes_wide<<<grid_for(nnz, 256), 256, 0, st>>>(d64, nnz, L, d_raw, d_bad);
        count_launch();
        r = launch_check("f64_to_planes_wide");
      } else {
        r = dispatch_w(prec, [&](auto w) {
          constexpr int W = decltype(w)::value;
          f64_to_planes<W><<<grid_for(nnz, 256), 256, 0, st>>>(d64, nnz, d_raw, d_bad);
          count_launch();
          return launch_check("f64_to_planes");
        });
      }
      cudaStreamSynchronize(st);
      cudaFree(d64);
      if (r != MP_OK) return fail(r);
    }
    if ((r = launch_check("validate_values")) != MP_OK) return fail(r);
    unsigned long long bad = 0;
    cudaError_t e = cudaMemcpyAsync(&bad, d_bad, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "validation");
    if (bad != ~0ull) {
      const int64_t k = (int64_t)bad;
      const int64_t row = std::upper_bound(rowptr, rowptr + n + 1, k) - rowptr - 1;
      return fail(set_error(MP_ERR_ARG, "row %lld: value %lld is %s", (long long)row,
                            (long long)k, values ? "not a normalised p-bit record" : "not finite"));
    }
  }

  // The sliced layout of A: row and chunk order on the host (row lengths
  // only), the entries and values placed on the device.
  {
    HostSell hs;
    build_sell_meta(n, rowptr, hs);
    if ((r = make_sell(hs, n, nnz, L, d_rowptr, cols_dev, d_srcs, d_raw, st, M->A, M->bytes)) !=
        MP_OK)
      return fail(r);
    if ((r = gather_sectors(M->A, st, &M->gather_sectors)) != MP_OK) return fail(r);
  }

  if (flags & MP_CSR_TRANSPOSE) {
    // A^T on the device: row j of A^T lists the rows i of A with a_ij stored,
    // ascending (column counts, an exclusive scan on the host, a scatter,
    // then each row sorted by i; rows longer than kRowSortMax are sorted on
    // the host).
    std::vector<int64_t> tptr(n + 1, 0);
    if ((r = dalloc(&d_tcnt, (size_t)n + 1, tmp)) != MP_OK) return fail(r);
    if ((r = dalloc(&d_tptr, (size_t)n + 1, tmp)) != MP_OK) return fail(r);
    if ((r = dalloc(&d_tcols, (size_t)nnz, tmp)) != MP_OK) return fail(r);
    if ((r = dalloc(&d_tsrc, (size_t)nnz, tmp)) != MP_OK) return fail(r);
    cudaError_t e = cudaMemsetAsync(d_tcnt, 0, ((size_t)n + 1) * 8, st);
    if (e == cudaSuccess && nnz > 0) {
      col_counts<<<grid_for(nnz, 256), 256, 0, st>>>(cols_dev, nnz, d_tcnt);
      count_launch();
      e = cudaGetLastError();
    }
    std::vector<unsigned long long> cnt(n + 1, 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(cnt.data(), d_tcnt, (size_t)n * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "transpose counts");
    for (int64_t j = 0; j < n; ++j) tptr[j + 1] = tptr[j] + (int64_t)cnt[j];
    unsigned int long_rows = 0;
    e = cudaMemcpyAsync(d_tptr, tptr.data(), ((size_t)n + 1) * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_tcnt, 0, ((size_t)n + 1) * 8, st);
    if (e == cudaSuccess && nnz > 0) {
      scatter_t<<<grid_for(n, 256), 256, 0, st>>>(d_rowptr, cols_dev, d_srcs, n, d_tptr, d_tcnt,
                                                  d_tcols, d_tsrc);
      e = cudaMemsetAsync(d_tcnt, 0, sizeof(unsigned int), st);
      if (e == cudaSuccess) {
        sort_rows_t<<<grid_for(n, 256), 256, 0, st>>>(d_tptr, n, d_tcols, d_tsrc,
                                                       reinterpret_cast<unsigned int*>(d_tcnt));
        count_launch(2);
        e = cudaGetLastError();
      }
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(&long_rows, d_tcnt, sizeof long_rows, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "transpose scatter");
    if (long_rows > 0) {  // rows too long for one thread's sort
      std::vector<int32_t> tc(nnz);
      std::vector<int64_t> ts(nnz);
      e = cudaMemcpyAsync(tc.data(), d_tcols, (size_t)nnz * 4, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(ts.data(), d_tsrc, (size_t)nnz * 8, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return cuda_fail(e, "transpose download");
      std::vector<std::pair<int32_t, int64_t>> row;
      for (int64_t j = 0; j < n; ++j) {
        const int64_t a = tptr[j], b = tptr[j + 1];
        if (b - a <= kRowSortMax) continue;
        row.clear();
        for (int64_t k = a; k < b; ++k) row.emplace_back(tc[k], ts[k]);
        std::sort(row.begin(), row.end());
        for (int64_t k = a; k < b; ++k) {
          tc[k] = row[k - a].first;
          ts[k] = row[k - a].second;
        }
      }
      e = cudaMemcpyAsync(d_tcols, tc.data(), (size_t)nnz * 4, cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_tsrc, ts.data(), (size_t)nnz * 8, cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return cuda_fail(e, "transpose upload");
    }
    HostSell ht;
    build_sell_meta(n, tptr.data(), ht);
    if ((r = make_sell(ht, n, nnz, L, d_tptr, d_tcols, d_tsrc, d_raw, st, M->AT, M->bytes)) !=
        MP_OK)
      return fail(r);
    M->has_t = true;
  }
  if ((r = dalloc(&M->ovf, (size_t)n + 1, M->bytes)) != MP_OK) return fail(r);
  if (M->has_t && (r = dalloc(&M->ovf_t, (size_t)n + 1, M->bytes)) != MP_OK) return fail(r);
  {
    cudaError_t e = cudaMemsetAsync(M->ovf, 0, sizeof(int32_t), st);
    if (e == cudaSuccess && M->ovf_t) e = cudaMemsetAsync(M->ovf_t, 0, sizeof(int32_t), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(cuda_error(e, "finishing create"));
  }
  release();
  if (!status_word()) {
    mp_csr_destroy(M);
    return set_error(MP_ERR_CUDA, "status word unavailable");
  }
  *out = M;
  return MP_OK;
}

}  // namespace
}  // namespace mpk

using namespace mpk;

extern "C" {

mp_status mp_csr_create(int64_t n, const int64_t* rowptr, const int32_t* colidx,
                        const uint64_t* values, int32_t prec_bits, int32_t flags, void* stream,
                        mp_csr* out) {
  return create_impl(n, rowptr, colidx, values, nullptr, prec_bits, flags, stream, out);
}

mp_status mp_csr_create_f64(int64_t n, const int64_t* rowptr, const int32_t* colidx,
                            const double* values, int32_t prec_bits, int32_t flags, void* stream,
                            mp_csr* out) {
  return create_impl(n, rowptr, colidx, nullptr, values, prec_bits, flags, stream, out);
}

mp_status mp_csr_destroy(mp_csr A) {
  if (!A) return MP_OK;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(A->device);
  cudaDeviceSynchronize();
  free_sell(A->A);
  free_sell(A->AT);
  cudaFree(A->ovf);
  cudaFree(A->ovf_t);
  cudaFree(A->a64);
  cudaFree(A->xrec);
  cudaFree(A->xrec_t);
  cudaFree(A->rowscale);
  delete A;
  cudaSetDevice(cur);
  return MP_OK;
}

mp_status mp_csr_info(mp_csr A, int64_t* n, int64_t* nnz, int32_t* prec_bits, int64_t* slots,
                      int64_t* device_bytes) {
  if (!A) return set_error(MP_ERR_ARG, "matrix is null");
  if (n) *n = A->n;
  if (nnz) *nnz = A->nnz;
  if (prec_bits) *prec_bits = A->prec;
  if (slots) *slots = A->A.nslots;
  if (device_bytes) *device_bytes = A->bytes;
  return MP_OK;
}

}  // extern "C"
