// blas.cu -- exact dot products (dot.cuh: two kernels per group of up to
// five dots), axpy, elementwise operations, conversions.
#include <climits>
#include <mutex>

#include "dot.cuh"
#include "internal.h"
#include "mpdev.cuh"

namespace mpk {
namespace {

int sm_count() { return dot_sm_count(); }

template <int W>
mp_status dot_w(const DotArgs& args, void* scratch, const int* gate, cudaStream_t st) {
  DotDev a{};
  a.k = args.k;
  a.n = args.n;
  for (int j = 0; j < 5; ++j) {
    a.x[j] = args.x[j];
    a.y[j] = args.y[j];
    a.ldx[j] = args.ldx[j];
    a.ldy[j] = args.ldy[j];
    a.out[j] = args.out[j];
    a.out_ld[j] = args.out_ld[j];
  }
  int* status = status_word();
  if (!status) return set_error(MP_ERR_CUDA, "status word unavailable");
  return dot_launch<W>(a, scratch, dot_blocks<W>(args.n), status, gate, st);
}

// ---------------------------------------------------------------------------
// Elementwise kernels
// ---------------------------------------------------------------------------

int ew_blocks(int64_t n) {
  int64_t b = (n + 255) / 256;
  const int64_t lim = (int64_t)sm_count() * 16;
  if (b > lim) b = lim;
  return (int)(b < 1 ? 1 : b);
}

template <int W>
__global__ void axpy_kernel(const uint64_t* __restrict__ al, int64_t n,
                            const uint64_t* __restrict__ x, int64_t ldx, uint64_t* __restrict__ y,
                            int64_t ldy) {
  Num<W> alpha;
  load<W>(alpha, al, 1, 0);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    Num<W> xv, yv, t, r;
    load<W>(xv, x, ldx, i);
    load<W>(yv, y, ldy, i);
    mul_rn_fast<W>(alpha, xv, t);
    add_rn<W>(yv, t, r);
    store<W>(r, y, ldy, i);
  }
}

template <int W>
__global__ void ewise_kernel(int op, int64_t n, const uint64_t* __restrict__ a, int64_t lda,
                             const uint64_t* __restrict__ b, int64_t ldb, uint64_t* out,
                             int64_t ldo, int* status) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    Num<W> x, y, r;
    load<W>(x, a, lda, i);
    load<W>(y, b, ldb, i);
    switch (op) {
      case MP_OP_MUL: mul_rn<W>(x, y, r); break;
      case MP_OP_ADD: add_rn<W>(x, y, r); break;
      case MP_OP_SUB: sub_rn<W>(x, y, r); break;
      default:
        if (zero_e(y.e)) {
          set_zero(r, 0u);
          atomicCAS(status, 0, (int)MP_ERR_DIVZERO);
        } else {
          div_rn<W>(x, y, r);
        }
    }
    store<W>(r, out, ldo, i);
  }
}

template <int W>
__global__ void from_f64_kernel(const double* __restrict__ d, int64_t n, uint64_t* out,
                                int64_t ld, int* status) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = d[i];
    Num<W> r;
    if (!isfinite(v)) atomicCAS(status, 0, (int)MP_ERR_ARG);
    from_f64<W>(isfinite(v) ? v : 0.0, r);
    store<W>(r, out, ld, i);
  }
}

// The same two conversions for p > 1024 (L limbs, a thread per element): a
// double's 53-bit mantissa lands in the top limb; the nearest double takes
// the top 53 bits, the next bit and a sticky bit over all lower limbs.
__global__ void from_f64_wide_kernel(const double* __restrict__ d, int64_t n, uint64_t* out,
                                     int64_t ld, int L, int* status) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double v = d[i];
    if (!isfinite(v)) {
      atomicCAS(status, 0, (int)MP_ERR_ARG);
      v = 0.0;
    }
    uint64_t top = 0;
    int64_t e = EXP_ZERO;
    if (v != 0.0) {
      int ex = 0;
      top = (uint64_t)ldexp(frexp(fabs(v), &ex), 53) << 11;
      e = ex;
    }
    out[i] = pack_head(e, signbit(v) ? 1u : 0u);
    for (int k = 1; k < L; ++k) out[(int64_t)k * ld + i] = 0;
    out[(int64_t)L * ld + i] = top;
  }
}

__global__ void to_f64_wide_kernel(const uint64_t* __restrict__ a, int64_t n, int64_t ld, int L,
                                   double* d) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t e;
    uint32_t s;
    unpack_head(a[i], e, s);
    if (zero_e(e)) {
      d[i] = s ? -0.0 : 0.0;
      continue;
    }
    const uint64_t t = a[(int64_t)L * ld + i];
    uint64_t rest = 0;
    for (int k = 1; k < L; ++k) rest |= a[(int64_t)k * ld + i];
    uint64_t q = t >> 11;
    const uint64_t rb = (t >> 10) & 1u;
    const bool sticky = (t & 0x3ffu) != 0u || rest != 0u;
    if (rb && (sticky || (q & 1u))) q += 1u;
    const int64_t ec = e < -4000 ? -4000 : (e > 4000 ? 4000 : e);
    const double v = ldexp((double)q, (int)ec - 53);
    d[i] = s ? -v : v;
  }
}

template <int W>
__global__ void to_f64_kernel(const uint64_t* __restrict__ a, int64_t n, int64_t ld, double* d) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    Num<W> x;
    load<W>(x, a, ld, i);
    d[i] = to_f64<W>(x);
  }
}

}  // namespace

size_t dot_scratch_bytes(int prec, int k) {
  const int64_t big = int64_t(1) << 40;  // the largest grid
  const int kk = k < 1 ? 1 : k;
  switch (prec) {
    case 128: return dot_scratch_size<4>(kk, dot_blocks<4>(big));
    case 256: return dot_scratch_size<8>(kk, dot_blocks<8>(big));
    case 512: return dot_scratch_size<16>(kk, dot_blocks<16>(big));
    default: return dot_scratch_size<32>(kk, dot_blocks<32>(big));
  }
}

mp_status launch_dot(int prec, const DotArgs& a, void* scratch, const int* gate,
                     cudaStream_t st) {
  if (a.k < 1 || a.k > 5) return set_error(MP_ERR_ARG, "dot count %d", a.k);
  return dispatch_w(prec, [&](auto w) {
    constexpr int W = decltype(w)::value;
    return dot_w<W>(a, scratch, gate, st);
  });
}

// Zeroes the head of a dot scratch buffer (the finalize's arrival counter).
mp_status init_dot_scratch(void* scratch, cudaStream_t st) {
  reset_dot_head<<<1, 32, 0, st>>>(static_cast<long long*>(scratch));
  count_launch();
  return launch_check("reset_dot_head");
}

}  // namespace mpk

using namespace mpk;

namespace {
std::mutex g_init_mu;
bool g_dot_ready[64] = {};
size_t g_dot_bytes[64] = {};
}  // namespace

extern "C" {

mp_status mp_dot(mp_vec x, mp_vec y, mp_vec out, void* stream) {
  mp_status r;
  const bool big = prec_big(x.prec_bits);
  if (!prec_ok(x.prec_bits) && !big) return set_error(MP_ERR_PREC, "precision %d", x.prec_bits);
  if ((r = check_vec(x, x.n, x.prec_bits, "x")) != MP_OK) return r;
  if ((r = check_vec(y, x.n, x.prec_bits, "y")) != MP_OK) return r;
  if ((r = check_vec(out, 1, x.prec_bits, "out")) != MP_OK) return r;
  if (x.n > MP_DOT_MAX_N)
    return set_error(MP_ERR_ARG, "mp_dot: length %lld exceeds the maximum %lld", (long long)x.n,
                     (long long)MP_DOT_MAX_N);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t bytes = big ? dot_big_scratch_bytes(x.prec_bits) : dot_scratch_bytes(x.prec_bits, 1);
  int dev = 0;
  MPK_CUDA(cudaGetDevice(&dev));
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_init_mu);
    scratch = dot_scratch(bytes);
    if (!scratch) return set_error(MP_ERR_ALLOC, "dot scratch of %zu bytes", bytes);
    if (!g_dot_ready[dev] || g_dot_bytes[dev] < bytes) {
      if ((r = init_dot_scratch(scratch, st)) != MP_OK) return r;
      g_dot_ready[dev] = true;
      g_dot_bytes[dev] = bytes;
    }
  }
  if (big)
    return launch_dot_big(x.prec_bits, x.data, x.ld, y.data, y.ld, x.n, out.data, out.ld, scratch,
                          nullptr, st);
  DotArgs a;
  a.k = 1;
  a.n = x.n;
  a.x[0] = x.data;
  a.y[0] = y.data;
  a.ldx[0] = x.ld;
  a.ldy[0] = y.ld;
  a.out[0] = out.data;
  a.out_ld[0] = out.ld;
  return launch_dot(x.prec_bits, a, scratch, nullptr, st);
}

mp_status mp_axpy(mp_vec alpha, mp_vec x, mp_vec y, void* stream) {
  mp_status r;
  const bool big = prec_big(x.prec_bits);
  if (!prec_ok(x.prec_bits) && !big) return set_error(MP_ERR_PREC, "precision %d", x.prec_bits);
  if ((r = check_vec(alpha, 1, x.prec_bits, "alpha")) != MP_OK) return r;
  if ((r = check_vec(x, x.n, x.prec_bits, "x")) != MP_OK) return r;
  if ((r = check_vec(y, x.n, x.prec_bits, "y")) != MP_OK) return r;
  if (x.n == 0) return MP_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (big) return launch_axpy_big(x.prec_bits, alpha.data, x.n, x.data, x.ld, y.data, y.ld, st);
  return dispatch_w(x.prec_bits, [&](auto w) {
    constexpr int W = decltype(w)::value;
    axpy_kernel<W><<<ew_blocks(x.n), 256, 0, st>>>(alpha.data, x.n, x.data, x.ld, y.data, y.ld);
    count_launch();
    return launch_check("axpy_kernel");
  });
}

mp_status mp_ewise(int32_t op, mp_vec a, mp_vec b, mp_vec out, void* stream) {
  mp_status r;
  if (op < MP_OP_MUL || op > MP_OP_DIV) return set_error(MP_ERR_ARG, "op %d", op);
  if (!prec_ok(a.prec_bits)) return set_error(MP_ERR_PREC, "precision %d", a.prec_bits);
  if ((r = check_vec(b, a.n, a.prec_bits, "b")) != MP_OK) return r;
  if ((r = check_vec(out, a.n, a.prec_bits, "out")) != MP_OK) return r;
  if ((r = check_vec(a, a.n, a.prec_bits, "a")) != MP_OK) return r;
  if (a.n == 0) return MP_OK;
  int* status = status_word();
  if (!status) return set_error(MP_ERR_CUDA, "status word unavailable");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return dispatch_w(a.prec_bits, [&](auto w) {
    constexpr int W = decltype(w)::value;
    ewise_kernel<W><<<ew_blocks(a.n), 256, 0, st>>>(op, a.n, a.data, a.ld, b.data, b.ld,
                                                    out.data, out.ld, status);
    count_launch();
    return launch_check("ewise_kernel");
  });
}

mp_status mp_vec_from_f64(const double* d, mp_vec out, void* stream) {
  mp_status r;
  const bool big = prec_big(out.prec_bits);
  if (!prec_ok(out.prec_bits) && !big) return set_error(MP_ERR_PREC, "precision %d", out.prec_bits);
  if ((r = check_vec(out, out.n, out.prec_bits, "out")) != MP_OK) return r;
  if (out.n == 0) return MP_OK;
  if (!d) return set_error(MP_ERR_ARG, "d is null");
  int* status = status_word();
  if (!status) return set_error(MP_ERR_CUDA, "status word unavailable");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (big) {
    from_f64_wide_kernel<<<ew_blocks(out.n), 256, 0, st>>>(d, out.n, out.data, out.ld,
                                                           out.prec_bits / 64, status);
    count_launch();
    return launch_check("from_f64_wide_kernel");
  }
  return dispatch_w(out.prec_bits, [&](auto w) {
    constexpr int W = decltype(w)::value;
    from_f64_kernel<W><<<ew_blocks(out.n), 256, 0, st>>>(d, out.n, out.data, out.ld, status);
    count_launch();
    return launch_check("from_f64_kernel");
  });
}

mp_status mp_vec_to_f64(mp_vec a, double* d, void* stream) {
  mp_status r;
  const bool big = prec_big(a.prec_bits);
  if (!prec_ok(a.prec_bits) && !big) return set_error(MP_ERR_PREC, "precision %d", a.prec_bits);
  if ((r = check_vec(a, a.n, a.prec_bits, "a")) != MP_OK) return r;
  if (a.n == 0) return MP_OK;
  if (!d) return set_error(MP_ERR_ARG, "d is null");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (big) {
    to_f64_wide_kernel<<<ew_blocks(a.n), 256, 0, st>>>(a.data, a.n, a.ld, a.prec_bits / 64, d);
    count_launch();
    return launch_check("to_f64_wide_kernel");
  }
  return dispatch_w(a.prec_bits, [&](auto w) {
    constexpr int W = decltype(w)::value;
    to_f64_kernel<W><<<ew_blocks(a.n), 256, 0, st>>>(a.data, a.n, a.ld, d);
    count_launch();
    return launch_check("to_f64_kernel");
  });
}

}  // extern "C"

// ---------------------------------------------------------------------------
// mp_dot_noalloc: the exact dot product with its scratch in a fixed device
// array instead of memory from cudaMalloc.
//
// Some callers cannot let a library allocate device memory: a process whose
// GPU memory is owned by another allocator (a framework's caching allocator
// that has reserved the memory, a server held to a fixed memory budget) would
// see cudaMalloc fail or break its budget, and cudaMalloc/cudaFree can
// synchronise the device, which latency-bound callers must avoid.  mp_dot
// allocates its scratch on first use; this variant never does.  Its scratch
// is the file-scope array below, present on every GPU that loads the
// library until the process exits.
// ---------------------------------------------------------------------------

namespace mpk {
namespace {

constexpr int kNoAllocBlocks = 64;  // grid of the variant (grid-stride loops cover any n)
constexpr size_t kNoAllocBytes = dot_scratch_size<32>(1, kNoAllocBlocks);

static_assert(kNoAllocBytes == MP_DOT_NOALLOC_SCRATCH_BYTES, "scratch size stated in mpkrylov.h");

static __device__ __align__(256) unsigned char g_dot_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[64] = {};

// Device address of the array for the current device, looked up once per
// device (host code may not use the array's name as a device address).
mp_status noalloc_scratch(void** out) {
  int dev = 0;
  MPK_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return set_error(MP_ERR_CUDA, "device %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_dot_noalloc_scratch);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(g_dot_noalloc_scratch)");
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return MP_OK;
}

template <int W>
mp_status dot_noalloc_w(const DotDev& a, void* scratch, int* status, cudaStream_t st) {
  const int64_t b = (a.n + kDotThreads - 1) / kDotThreads;
  const int nb = (int)(b < 1 ? 1 : (b > kNoAllocBlocks ? kNoAllocBlocks : b));
  const size_t need = dot_scratch_size<W>(1, nb);
  if (need > kNoAllocBytes)
    return set_error(MP_ERR_ARG, "mp_dot_noalloc needs %zu scratch bytes, the array holds %zu",
                     need, kNoAllocBytes);
  // The array keeps the previous call's contents.  Nothing needs clearing:
  // every block writes its exponent range before the finalize reads it, the
  // finalize reads only the partial digits the blocks wrote in this call,
  // and this form runs no step after the dot (its arrival counter is unused).
  return dot_launch<W>(a, scratch, nb, status, nullptr, st);
}

}  // namespace
}  // namespace mpk

extern "C" {

mp_status mp_dot_noalloc(mp_vec x, mp_vec y, mp_vec out, void* stream) {
  mp_status r;
  if (!prec_ok(x.prec_bits)) return set_error(MP_ERR_PREC, "precision %d", x.prec_bits);
  if ((r = check_vec(x, x.n, x.prec_bits, "x")) != MP_OK) return r;
  if ((r = check_vec(y, x.n, x.prec_bits, "y")) != MP_OK) return r;
  if ((r = check_vec(out, 1, x.prec_bits, "out")) != MP_OK) return r;
  if (x.n > MP_DOT_NOALLOC_MAX_N)
    return set_error(MP_ERR_ARG, "mp_dot_noalloc: length %lld exceeds the maximum %lld",
                     (long long)x.n, (long long)MP_DOT_NOALLOC_MAX_N);
  void* scratch = nullptr;
  if ((r = noalloc_scratch(&scratch)) != MP_OK) return r;
  int* status = status_word();
  if (!status) return set_error(MP_ERR_CUDA, "status word unavailable");
  DotDev a{};
  a.k = 1;
  a.n = x.n;
  a.x[0] = x.data;
  a.y[0] = y.data;
  a.ldx[0] = x.ld;
  a.ldy[0] = y.ld;
  a.out[0] = out.data;
  a.out_ld[0] = out.ld;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return dispatch_w(x.prec_bits, [&](auto w) {
    constexpr int W = decltype(w)::value;
    return dot_noalloc_w<W>(a, scratch, status, st);
  });
}

}  // extern "C"
