// internal.h -- host-side internals shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <type_traits>

#include "mpkrylov.h"

namespace mpk {

// Sliced, row-length-sorted layout of a CSR matrix (SELL-32-sigma).  Rows are
// sorted by length (descending, ties by row index) inside windows of
// kSigma rows and packed 32 per chunk; chunks are then ordered longest first.
// Chunk c holds its rows' entries column-major, slot chunk_off[c] + j*32 +
// lane for the j-th entry of the lane's row, so that a warp reading entry j
// of 32 rows touches 32 consecutive slots.  Each row keeps its CSR column
// order.
constexpr int kSigma = 4096;

struct Sell {
  int64_t n = 0, nnz = 0, nslots = 0, nchunks = 0;
  int64_t* chunk_off = nullptr;  // [nchunks + 1]
  int32_t* row_of = nullptr;     // [nchunks * 32], original row or -1
  int32_t* row_len = nullptr;    // [nchunks * 32]
  int32_t* col = nullptr;        // [nslots]
  uint64_t* val = nullptr;       // [(L+1) * nslots], plane-major
  int64_t* src = nullptr;        // [nslots], the entry's position in the caller's CSR (-1: padding)
};

}  // namespace mpk

struct mp_csr_s {
  int64_t n = 0, nnz = 0;
  int32_t prec = 0;
  int device = 0;
  bool has_t = false;
  mpk::Sell A, AT;
  // [n + 1]: overflow-row count then rows (EXACT wide path); ovf_t for
  // products with A^T, so that a product with A and one with A^T can run at
  // the same time (BiCG's two products)
  int32_t* ovf = nullptr;
  int32_t* ovf_t = nullptr;
  int64_t bytes = 0;
  // SpMV launch configuration per mode (ORDERED [0], EXACT [1]), set by
  // mp_csr_tune / mp_csr_set_config: threads per block, variant bits and
  // shared-memory carve-out (percent); -1 everywhere: the library's default
  // for the precision.
  int32_t cfg_tpb[2] = {-1, -1};
  int32_t cfg_var[2] = {-1, -1};
  int32_t cfg_carve[2] = {-1, -1};
  // record copy of x for the gathers (variant bit 3), allocated on first use;
  // xrec_t for products with A^T
  uint64_t* xrec = nullptr;
  uint64_t* xrec_t = nullptr;
  // mean distinct 32-byte groups a warp's gather of one x plane touches (8..32)
  double gather_sectors = 0.0;
  // FP64 copy for mixed-precision refinement (built on first use): the
  // row-equilibrated entries 2^-E_i a_ij per slot of A's layout, and 2^-E_i.
  double* a64 = nullptr;
  double* rowscale = nullptr;
};

// ILU(0) factors of a matrix in CSR order (sorted columns) with the level
// schedules of the triangular solves (rows of a level depend only on rows of
// earlier levels).
struct mp_ilu_s {
  int64_t n = 0, nnz = 0;
  int32_t prec = 0;
  int device = 0;
  int64_t* rowptr = nullptr;  // [n + 1]
  int32_t* col = nullptr;     // [nnz]
  int64_t* diag = nullptr;    // [n] position of (i, i)
  uint64_t* lu = nullptr;     // [(L+1) * nnz] plane-major, ld = nnz
  int32_t* rows_l = nullptr;  // rows by forward (and factorisation) level
  int32_t* rows_u = nullptr;  // rows by backward level
  int64_t* lvl_l = nullptr;   // host [nl + 1]
  int64_t* lvl_u = nullptr;   // host [nu + 1]
  int64_t* d_lvl_l = nullptr; // device copies of the level boundaries
  int64_t* d_lvl_u = nullptr;
  int64_t nl = 0, nu = 0;
};

namespace mpk {

// The scratch of a product with layout S of M (A or A^T): its overflow list
// and its record copy of x.
inline bool is_transposed(const mp_csr_s* M, const Sell& S) { return &S == &M->AT; }
inline int32_t* ovf_of(const mp_csr_s* M, const Sell& S) {
  return is_transposed(M, S) && M->ovf_t ? M->ovf_t : M->ovf;
}

// w = (LU)^{-1} r with an ILU(0) factor, one launch per level; gate as for
// the SpMV (a nonzero flag makes every launch return at once).
mp_status launch_ilu0_apply(const mp_ilu_s* M, const uint64_t* r, int64_t ldr, uint64_t* w,
                            int64_t ldw, const int* gate, cudaStream_t st);
// The same at p = 2048, 4096, 8192 (bigp_ilu.cu), and the factorisation
// there (zero pivots set *status to MP_ERR_DIVZERO).
mp_status launch_ilu0_apply_big(const mp_ilu_s* M, const uint64_t* r, int64_t ldr, uint64_t* w,
                                int64_t ldw, const int* gate, cudaStream_t st);
mp_status launch_ilu0_factor_big(const mp_ilu_s* M, int* status, cudaStream_t st);

// ---- errors -------------------------------------------------------------
mp_status set_error(mp_status s, const char* fmt, ...);
mp_status cuda_error(cudaError_t e, const char* where);
#define MPK_CUDA(call)                                              \
  do {                                                              \
    cudaError_t e_ = (call);                                        \
    if (e_ != cudaSuccess) return ::mpk::cuda_error(e_, #call);     \
  } while (0)

// Host-side fault injection for the error paths: returns cudaErrorUnknown
// once when mp_debug_fail armed `site` and its countdown has run out, else
// cudaSuccess.  Costs one relaxed atomic load when nothing is armed.
cudaError_t injected_fault(const char* site);

// ---- device status word and launch accounting ---------------------------
int* status_word();  // device address of the current device's status word
void count_launch(int k = 1);
mp_status launch_check(const char* what);  // cudaGetLastError after a launch

// A private non-blocking stream whose work starts after what the caller's
// stream holds now (the solvers capture graphs, which the legacy default
// stream does not allow).  On failure nothing is left created.
mp_status private_stream_open(cudaStream_t caller, cudaStream_t* ps, cudaEvent_t* fence);
// Makes the caller's stream wait for the private stream's work, waits for it
// on the host and destroys the stream and the event.
void private_stream_close(cudaStream_t caller, cudaStream_t ps, cudaEvent_t fence);
// cudaMallocAsync of a solver's work space, behind the "work memory"
// fault-injection site.
cudaError_t work_malloc(void** p, size_t bytes, cudaStream_t st);

// ---- precision ------------------------------------------------------------
inline bool prec_ok(int p) { return p == 128 || p == 256 || p == 512 || p == 1024; }
// 2048, 4096, 8192: one value per warp (bigp.cu); SpMV, dot and axpy only.
inline bool prec_big(int p) { return p == 2048 || p == 4096 || p == 8192; }
inline int planes_of(int p) { return p / 64 + 1; }

mp_status check_vec(const mp_vec& v, int64_t n, int prec, const char* name);

// Calls f(std::integral_constant<int, W>{}) with W = p/32 words.
template <class F>
mp_status dispatch_w(int p, F&& f) {
  switch (p) {
    case 128: return f(std::integral_constant<int, 4>{});
    case 256: return f(std::integral_constant<int, 8>{});
    case 512: return f(std::integral_constant<int, 16>{});
    case 1024: return f(std::integral_constant<int, 32>{});
    default: return set_error(MP_ERR_PREC, "precision %d not in {128,256,512,1024}", p);
  }
}

// ---- p > 1024 (bigp.cu) ------------------------------------------------------
// rb != nullptr: r = RN(b - A x) (EXACT).  gate as for launch_spmv.
mp_status launch_spmv_big(const mp_csr_s* M, const Sell& S, int mode, const uint64_t* x,
                          int64_t ldx, uint64_t* y, int64_t ldy, const uint64_t* rb, int64_t ldb,
                          const int* gate, cudaStream_t st);
size_t dot_big_scratch_bytes(int prec);
// scratch: a dot scratch whose header span slots are (+inf, -inf)
mp_status launch_dot_big(int prec, const uint64_t* x, int64_t ldx, const uint64_t* y, int64_t ldy,
                         int64_t n, uint64_t* out, int64_t ldo, void* scratch, const int* gate,
                         cudaStream_t st);
// BiCG (method 0), GPBiCG (1), CGS (2), BiCGSTAB (3) at p > 1024 (bigp_solve.cu)
// pre: ILU(0) preconditioner of BiCGSTAB (left when pre_left, else right)
mp_status solve_big(int method, mp_csr A, mp_vec b, mp_vec x, const mp_solve_opts* opts,
                    mp_solve_info* info, cudaStream_t st, const mp_ilu_s* pre = nullptr,
                    int pre_left = 1);
mp_status launch_axpy_big(int prec, const uint64_t* al, int64_t n, const uint64_t* x, int64_t ldx,
                          uint64_t* y, int64_t ldy, cudaStream_t st);

// ---- scratch ---------------------------------------------------------------
// Per-device scratch of the standalone dot product (grown on demand).
void* dot_scratch(size_t bytes);

// ---- kernels exported across translation units ----------------------------
// Exact dot products: k pairs (x[j], y[j]) of length n -> out[j] (device
// scalars, plane-major with ld 1 each, may point into a larger buffer).
struct DotArgs {
  int k = 0;
  int64_t n = 0;
  const uint64_t* x[5] = {};
  const uint64_t* y[5] = {};
  int64_t ldx[5] = {}, ldy[5] = {};
  uint64_t* out[5] = {};  // plane-major scalars with ld = out_ld[j]
  int64_t out_ld[5] = {};
};
size_t dot_scratch_bytes(int prec, int k);
mp_status init_dot_scratch(void* scratch, cudaStream_t st);
mp_status launch_dot(int prec, const DotArgs& a, void* scratch, const int* gate,
                     cudaStream_t st);

// SpMV / residual on a sliced matrix.  resid_b != nullptr computes
// r = RN(b - A x) (EXACT only).  gate: device flag; when nonzero at run time
// the kernels return without work (used by the solvers after convergence).
mp_status launch_spmv(const mp_csr_s* M, const Sell& S, int mode, const uint64_t* x, int64_t ldx,
                      uint64_t* y, int64_t ldy, const uint64_t* resid_b, int64_t ldb,
                      const int* gate, cudaStream_t st);
// y = A x skipping rows whose instance k = rinst[row] has idone[k] != 0.
mp_status launch_spmv_batched(const mp_csr_s* M, int mode, const uint64_t* x, int64_t ldx,
                              uint64_t* y, int64_t ldy, const int32_t* rinst, const int* idone,
                              cudaStream_t st);

}  // namespace mpk
