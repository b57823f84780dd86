// csr.cu -- building the device matrix (Section 2's CSR storage at p bits).
//
// Index work runs on the host once per matrix: validation, a stable sort of
// each row's columns, the sliced row-length-sorted layout (SELL-32-sigma) and
// the stable counting sort that orders A^T's rows by ascending original row.
// The p-bit values move on the device: the caller's planes are uploaded once
// and gathered into the sliced layout of A (and of A^T) by a kernel, with no
// atomics, so the layout is deterministic.
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

int grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 65535LL * 8) b = 65535LL * 8;
  return (int)b;
}

struct HostSell {
  int64_t nslots = 0, nchunks = 0;
  double gather_sectors = 0.0;  // mean distinct 4-element groups per warp gather
  std::vector<int64_t> chunk_off;
  std::vector<int32_t> row_of, row_len, col;
  std::vector<int64_t> src;  // raw value index per slot, -1 = padding
};

// rowptr/cols/srcs describe a CSR matrix whose row entries are already in
// the summation order; srcs[k] is the raw value index of entry k.
void build_sell(int64_t n, const int64_t* rowptr, const int32_t* cols, const int64_t* srcs,
                HostSell& h) {
  std::vector<int32_t> perm(n);
  std::iota(perm.begin(), perm.end(), 0);
  for (int64_t w0 = 0; w0 < n; w0 += kSigma) {
    const int64_t w1 = std::min<int64_t>(n, w0 + kSigma);
    std::stable_sort(perm.begin() + w0, perm.begin() + w1, [&](int32_t a, int32_t b) {
      return (rowptr[a + 1] - rowptr[a]) > (rowptr[b + 1] - rowptr[b]);
    });
  }
  h.nchunks = (n + 31) / 32;
  // Chunks are laid out (and so scheduled) longest first across the whole
  // matrix, so the long sequential row chains start at the beginning of a
  // launch instead of forming its tail; each chunk keeps its 32 rows from one
  // sigma window (x locality within the chunk).
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
  h.col.assign(h.nslots, 0);
  h.src.assign(h.nslots, -1);
  for (int64_t c = 0; c < h.nchunks; ++c) {
    for (int t = 0; t < 32; ++t) {
      const int32_t r = h.row_of[c * 32 + t];
      if (r < 0) continue;
      for (int64_t j = 0; j < h.row_len[c * 32 + t]; ++j) {
        const int64_t s = h.chunk_off[c] + j * 32 + t;
        h.col[s] = cols[rowptr[r] + j];
        h.src[s] = srcs[rowptr[r] + j];
      }
    }
  }
  // How scattered the x gathers are: distinct 32-byte groups of four
  // consecutive elements that a warp's gather of one plane touches (8 when
  // the 32 lanes read consecutive columns, up to 32), sampled on every
  // fourth chunk.  Picks the default gather layout.
  int64_t groups = 0, touched = 0;
  for (int64_t c = 0; c < h.nchunks; c += 4) {
    const int64_t len = (h.chunk_off[c + 1] - h.chunk_off[c]) / 32;
    for (int64_t j = 0; j < len; ++j) {
      int32_t g[32];
      int m = 0;
      for (int t = 0; t < 32; ++t) {
        if (j < h.row_len[c * 32 + t]) g[m++] = h.col[h.chunk_off[c] + j * 32 + t] >> 2;
      }
      if (m == 0) continue;
      std::sort(g, g + m);
      touched += std::unique(g, g + m) - g;
      ++groups;
    }
  }
  h.gather_sectors = groups ? (double)touched / (double)groups : 0.0;
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

mp_status upload_sell(const HostSell& h, int64_t n, int64_t nnz, int L, const uint64_t* d_raw,
                      cudaStream_t st, Sell& S, int64_t& bytes) {
  S.n = n;
  S.nnz = nnz;
  S.nslots = h.nslots;
  S.nchunks = h.nchunks;
  mp_status r;
  if ((r = dalloc(&S.chunk_off, h.chunk_off.size(), bytes)) != MP_OK) return r;
  if ((r = dalloc(&S.row_of, h.row_of.size(), bytes)) != MP_OK) return r;
  if ((r = dalloc(&S.row_len, h.row_len.size(), bytes)) != MP_OK) return r;
  if ((r = dalloc(&S.col, h.col.size(), bytes)) != MP_OK) return r;
  if ((r = dalloc(&S.val, (size_t)(L + 1) * h.nslots, bytes)) != MP_OK) return r;
  MPK_CUDA(cudaMemcpyAsync(S.chunk_off, h.chunk_off.data(), h.chunk_off.size() * 8,
                           cudaMemcpyHostToDevice, st));
  if (!h.row_of.empty()) {
    MPK_CUDA(cudaMemcpyAsync(S.row_of, h.row_of.data(), h.row_of.size() * 4,
                             cudaMemcpyHostToDevice, st));
    MPK_CUDA(cudaMemcpyAsync(S.row_len, h.row_len.data(), h.row_len.size() * 4,
                             cudaMemcpyHostToDevice, st));
  }
  if (h.nslots > 0) {
    MPK_CUDA(cudaMemcpyAsync(S.col, h.col.data(), h.col.size() * 4, cudaMemcpyHostToDevice, st));
    // the slot -> caller position map stays (gradients on the pattern use it)
    if ((r = dalloc(&S.src, h.src.size(), bytes)) != MP_OK) return r;
    MPK_CUDA(cudaMemcpyAsync(S.src, h.src.data(), h.src.size() * 8, cudaMemcpyHostToDevice, st));
    gather_planes<<<grid_for(h.nslots, 256), 256, 0, st>>>(d_raw, nnz, S.src, h.nslots, L, S.val);
    count_launch();
    r = launch_check("gather_planes");
    cudaStreamSynchronize(st);
    if (r != MP_OK) return r;
  }
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

  // Columns: in range, unique per row; entries taken in ascending column
  // order (a stable sort per row when the caller's order differs).
  std::vector<int32_t> cols(nnz);
  std::vector<int64_t> srcs(nnz);
  std::vector<int64_t> idx;
  for (int64_t i = 0; i < n; ++i) {
    const int64_t a = rowptr[i], b = rowptr[i + 1];
    bool sorted = true;
    for (int64_t k = a; k < b; ++k) {
      if (colidx[k] < 0 || colidx[k] >= n)
        return set_error(MP_ERR_ARG, "row %lld: column %d out of range", (long long)i, colidx[k]);
      if (k > a && colidx[k] <= colidx[k - 1]) sorted = false;
    }
    if (sorted) {
      for (int64_t k = a; k < b; ++k) {
        cols[k] = colidx[k];
        srcs[k] = k;
      }
    } else {
      idx.resize(b - a);
      std::iota(idx.begin(), idx.end(), a);
      std::stable_sort(idx.begin(), idx.end(),
                       [&](int64_t u, int64_t v) { return colidx[u] < colidx[v]; });
      for (int64_t k = a; k < b; ++k) {
        cols[k] = colidx[idx[k - a]];
        srcs[k] = idx[k - a];
        if (k > a && cols[k] == cols[k - 1])
          return set_error(MP_ERR_ARG, "row %lld: column %d repeated", (long long)i, cols[k]);
      }
    }
  }

  mp_csr_s* M = new (std::nothrow) mp_csr_s;
  if (!M) return set_error(MP_ERR_ALLOC, "host allocation failed");
  M->n = n;
  M->nnz = nnz;
  M->prec = prec;
  M->device = dev;
  mp_status r = MP_OK;
  uint64_t* d_raw = nullptr;
  unsigned long long* d_bad = nullptr;
  int64_t tmp = 0;
  auto fail = [&](mp_status s) {
    cudaStreamSynchronize(st);
    cudaFree(d_raw);
    cudaFree(d_bad);
    free_sell(M->A);
    free_sell(M->AT);
    cudaFree(M->ovf);
    delete M;
    return s;
  };
  if ((r = dalloc(&d_raw, (size_t)(L + 1) * nnz, tmp)) != MP_OK) return fail(r);
  if ((r = dalloc(&d_bad, 1, tmp)) != MP_OK) return fail(r);
  {
    const unsigned long long none = ~0ull;
    cudaError_t e = cudaMemcpyAsync(d_bad, &none, 8, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return fail(cuda_error(e, "cudaMemcpyAsync"));
  }
  if (nnz > 0) {
    if (values) {
      cudaError_t e = cudaMemcpyAsync(d_raw, values, (size_t)(L + 1) * nnz * 8,
                                      cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) return fail(cuda_error(e, "cudaMemcpyAsync(values)"));
      validate_values<<<grid_for(nnz, 256), 256, 0, st>>>(d_raw, nnz, L, d_bad);
      count_launch();
    } else {
      double* d64 = nullptr;
      if ((r = dalloc(&d64, nnz, tmp)) != MP_OK) return fail(r);
      cudaMemcpyAsync(d64, values64, (size_t)nnz * 8, cudaMemcpyHostToDevice, st);
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
    if (e != cudaSuccess) return fail(cuda_error(e, "validation"));
    if (bad != ~0ull) {
      const int64_t k = (int64_t)bad;
      const int64_t row = std::upper_bound(rowptr, rowptr + n + 1, k) - rowptr - 1;
      return fail(set_error(MP_ERR_ARG, "row %lld: value %lld is %s", (long long)row,
                            (long long)k, values ? "not a normalised p-bit record" : "not finite"));
    }
  }

  HostSell hs;
  build_sell(n, rowptr, cols.data(), srcs.data(), hs);
  M->gather_sectors = hs.gather_sectors;
  if ((r = upload_sell(hs, n, nnz, L, d_raw, st, M->A, M->bytes)) != MP_OK) return fail(r);

  if (flags & MP_CSR_TRANSPOSE) {
    // Stable counting sort by column: row j of A^T lists rows i ascending.
    std::vector<int64_t> tptr(n + 1, 0);
    for (int64_t k = 0; k < nnz; ++k) tptr[cols[k] + 1]++;
    for (int64_t j = 0; j < n; ++j) tptr[j + 1] += tptr[j];
    std::vector<int64_t> next(tptr.begin(), tptr.end() - 1);
    std::vector<int32_t> tcols(nnz);
    std::vector<int64_t> tsrc(nnz);
    for (int64_t i = 0; i < n; ++i) {
      for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
        const int64_t pos = next[cols[k]]++;
        tcols[pos] = (int32_t)i;
        tsrc[pos] = srcs[k];
      }
    }
    HostSell ht;
    build_sell(n, tptr.data(), tcols.data(), tsrc.data(), ht);
    if ((r = upload_sell(ht, n, nnz, L, d_raw, st, M->AT, M->bytes)) != MP_OK) return fail(r);
    M->has_t = true;
  }
  if ((r = dalloc(&M->ovf, (size_t)n + 1, M->bytes)) != MP_OK) return fail(r);
  {
    cudaError_t e = cudaMemsetAsync(M->ovf, 0, sizeof(int32_t), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(cuda_error(e, "finishing create"));
  }
  cudaFree(d_raw);
  cudaFree(d_bad);
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
  cudaFree(A->a64);
  cudaFree(A->xrec);
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
