// runtime.cu -- status codes, error strings, the per-device status word, the
// launch counter, the standalone scratch buffer and the IMAD throughput probe.
#include <atomic>
#include <cstdarg>
#include <cstring>
#include <mutex>

#include "internal.h"

namespace mpk {

// Device-side status word: kernels record the first data-dependent error
// (span overflow, zero divisor) with atomicCAS(0 -> code).
__device__ int g_mpk_status_word;

namespace {
thread_local char g_err[512] = "";
thread_local int64_t g_launches = 0;

std::mutex g_mu;
int* g_status_addr[64] = {};
void* g_scratch[64] = {};
size_t g_scratch_bytes[64] = {};
}  // namespace

namespace {
std::atomic<int> g_fail_armed{0};
char g_fail_site[64] = "";
int64_t g_fail_after = 0;
}  // namespace

cudaError_t injected_fault(const char* site) {
  if (!g_fail_armed.load(std::memory_order_relaxed)) return cudaSuccess;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_fail_armed.load(std::memory_order_relaxed) || strcmp(site, g_fail_site) != 0)
    return cudaSuccess;
  if (g_fail_after > 0) {
    --g_fail_after;
    return cudaSuccess;
  }
  g_fail_armed.store(0);
  return cudaErrorUnknown;
}

mp_status set_error(mp_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return s;
}

mp_status cuda_error(cudaError_t e, const char* where) {
  set_error(MP_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? MP_ERR_ALLOC : MP_ERR_CUDA;
}

int* status_word() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_status_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_mpk_status_word) != cudaSuccess) return nullptr;
    g_status_addr[dev] = static_cast<int*>(p);
  }
  return g_status_addr[dev];
}

void count_launch(int k) { g_launches += k; }

mp_status launch_check(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, what);
  return MP_OK;
}

mp_status private_stream_open(cudaStream_t caller, cudaStream_t* ps, cudaEvent_t* fence) {
  *ps = nullptr;
  *fence = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(ps, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(fence, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(*fence, caller);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(*ps, *fence, 0);
  if (e == cudaSuccess) return MP_OK;
  if (*fence) cudaEventDestroy(*fence);
  if (*ps) cudaStreamDestroy(*ps);
  *ps = nullptr;
  *fence = nullptr;
  return cuda_error(e, "private stream set-up");
}

void private_stream_close(cudaStream_t caller, cudaStream_t ps, cudaEvent_t fence) {
  cudaEventRecord(fence, ps);
  cudaStreamWaitEvent(caller, fence, 0);
  cudaStreamSynchronize(ps);
  cudaEventDestroy(fence);
  cudaStreamDestroy(ps);
}

cudaError_t work_malloc(void** p, size_t bytes, cudaStream_t st) {
  const cudaError_t e = injected_fault("work memory");
  return e != cudaSuccess ? e : cudaMallocAsync(p, bytes, st);
}

mp_status check_vec(const mp_vec& v, int64_t n, int prec, const char* name) {
  if (v.prec_bits != prec)
    return set_error(MP_ERR_ARG, "%s: precision %d, expected %d", name, v.prec_bits, prec);
  if (v.n != n) return set_error(MP_ERR_ARG, "%s: length %lld, expected %lld", name,
                                 (long long)v.n, (long long)n);
  if (v.ld < v.n) return set_error(MP_ERR_ARG, "%s: ld %lld < n", name, (long long)v.ld);
  if (n > 0 && v.data == nullptr) return set_error(MP_ERR_ARG, "%s: null data", name);
  return MP_OK;
}

void* dot_scratch(size_t bytes) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_scratch_bytes[dev] < bytes) {
    if (g_scratch[dev]) cudaFree(g_scratch[dev]);
    g_scratch[dev] = nullptr;
    g_scratch_bytes[dev] = 0;
    if (cudaMalloc(&g_scratch[dev], bytes) != cudaSuccess) return nullptr;
    g_scratch_bytes[dev] = bytes;
  }
  return g_scratch[dev];
}

// Independent chains of 32x32->64 multiply-adds (IMAD.WIDE.U32): each step
// multiplies the chain's high word by a per-thread constant and adds the
// chain, so nothing can be hoisted and the 8 chains per thread overlap.  The
// result is folded into `sink` so the work is kept.
__global__ void imad_probe_kernel(uint64_t* sink, uint32_t iters, uint32_t seed) {
  uint64_t acc[8];
  uint32_t b[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    b[k] = (seed ^ (threadIdx.x * 2654435761u)) + 0x9e3779b9u * (uint32_t)(k + 1) + blockIdx.x;
    acc[k] = ((uint64_t)b[k] << 32) | (b[k] * 7u + 1u);
  }
  for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = (uint64_t)(uint32_t)(acc[k] >> 32) * b[k] + acc[k];
  }
  uint64_t s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s ^= acc[k];
  if (s == 0x1234567u) sink[0] = s;
}

}  // namespace mpk

using namespace mpk;

extern "C" {

const char* mp_status_string(mp_status s) {
  switch (s) {
    case MP_OK: return "ok";
    case MP_ERR_ARG: return "invalid argument";
    case MP_ERR_PREC: return "unsupported precision";
    case MP_ERR_ALLOC: return "allocation failed";
    case MP_ERR_CUDA: return "CUDA error";
    case MP_ERR_SPAN: return "exponent span of an exact sum exceeds the cap";
    case MP_ERR_BREAKDOWN: return "Krylov breakdown";
    case MP_ERR_NOCONV: return "not converged within maxit";
    case MP_ERR_TIMEOUT: return "device wait timed out";
    case MP_ERR_DIVZERO: return "division by zero";
  }
  return "unknown status";
}

const char* mp_last_error(void) { return g_err; }

mp_status mp_debug_fail(const char* site, int64_t after) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!site || !site[0]) {
    g_fail_armed.store(0);
    g_fail_site[0] = 0;
    return MP_OK;
  }
  if (strlen(site) >= sizeof g_fail_site || after < 0)
    return set_error(MP_ERR_ARG, "fault site name too long or negative countdown");
  strcpy(g_fail_site, site);
  g_fail_after = after;
  g_fail_armed.store(1);
  return MP_OK;
}

mp_status mp_debug_pool_used(int64_t* bytes) {
  if (!bytes) return set_error(MP_ERR_ARG, "bytes is null");
  int dev = 0;
  MPK_CUDA(cudaGetDevice(&dev));
  cudaMemPool_t pool;
  MPK_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
  uint64_t used = 0;
  MPK_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used));
  *bytes = (int64_t)used;
  return MP_OK;
}

int64_t mp_launch_count(int32_t reset) {
  const int64_t v = g_launches;
  if (reset) g_launches = 0;
  return v;
}

mp_status mp_check(void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  MPK_CUDA(cudaStreamSynchronize(st));
  int* w = status_word();
  if (!w) return set_error(MP_ERR_CUDA, "no status word on this device");
  int v = 0;
  MPK_CUDA(cudaMemcpy(&v, w, sizeof v, cudaMemcpyDeviceToHost));
  if (v != 0) {
    const int z = 0;
    MPK_CUDA(cudaMemcpy(w, &z, sizeof z, cudaMemcpyHostToDevice));
    return set_error(static_cast<mp_status>(v), "device reported: %s",
                     mp_status_string(static_cast<mp_status>(v)));
  }
  return MP_OK;
}

mp_status mp_imad_probe(double* rate, void* stream) {
  if (!rate) return set_error(MP_ERR_ARG, "rate is null");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  MPK_CUDA(cudaGetDevice(&dev));
  MPK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  uint64_t* sink = nullptr;
  MPK_CUDA(cudaMalloc(&sink, sizeof(uint64_t)));
  const int threads = 512, blocks = sms * 4;
  const uint32_t iters = 4096;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 5; ++rep) {
    cudaEventRecord(e0, st);
    imad_probe_kernel<<<blocks, threads, 0, st>>>(sink, iters, 12345u + rep);
    cudaEventRecord(e1, st);
    count_launch();
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  mp_status s = launch_check("imad_probe_kernel");
  if (s != MP_OK) return s;
  const double products = (double)blocks * threads * iters * 8.0;
  *rate = products / (best * 1e-3);
  return MP_OK;
}

}  // extern "C"
