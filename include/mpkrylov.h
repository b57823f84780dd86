/* mpkrylov.h -- C ABI of the GB300 (sm_103a) multiple-precision sparse Krylov
 * library: p-bit CSR sparse matrix-vector products y = A x and y = A^T x,
 * exact dot products, axpy, and the BiCG and GPBiCG solvers built on them.
 *
 * The operations are those of Kouya, "A Highly Efficient Implementation of
 * Multiple Precision Sparse Matrix-Vector Multiplication and Its Application
 * to Product-type Krylov Subspace Methods": a CSR matrix whose entries carry
 * `prec` bits (Section 2, the mpfrsmatrix structure), its SpMV (Section 3),
 * and BiCG / GPBiCG with the SpMV in place of the matrix products (Section 4,
 * Fig. 5), stopped by the residual rule of Section 4.
 *
 * Number format.  A value is (-1)^s * M * 2^(e-p) with 2^(p-1) <= M < 2^p
 * (MPFR's 0.1xxx_2 * 2^e convention, Section 2), or a signed zero
 * (e == MP_EXP_ZERO, M = 0).  p is one of 128, 256, 512, 1024 for every
 * call; p = 2048, 4096, 8192 (the precisions at which the solves of the
 * paper's Tables 1-2 converge) are accepted by mp_csr_create,
 * mp_csr_create_f64, mp_spmv, mp_spmv_t (both modes), mp_residual, mp_dot,
 * mp_axpy, mp_vec_from_f64, mp_vec_to_f64, mp_bicg, mp_gpbicg, mp_cgs and
 * mp_bicgstab, which run a warp-per-value form there (one value per warp,
 * mantissa in shared memory); every other call (ILU(0), refinement, batched
 * solves, the pattern gradient, the dense MV, the tuner) returns MP_ERR_PREC
 * for them.  Every operation rounds to nearest, ties to even
 * (MPFR's RN); NaN, infinities and the other rounding modes are not
 * represented.  Nonzero exponents must satisfy |e| < 2^60.
 *
 * Memory layout ("planes").  A vector of n values with L = p/64 is L+1
 * planes of uint64 words: plane 0 holds the head words e*2 + s (as int64
 * bit patterns), plane k (1 <= k <= L) holds mantissa limb k-1, least
 * significant first.  Plane k starts ld words after plane k-1.  A scalar
 * is a vector with n = 1.
 *
 * Conventions.  Every function returns an mp_status and never aborts.
 * Device pointers are CUDA device memory of the current device; the library
 * never frees memory it did not allocate.  `stream` is a cudaStream_t (NULL =
 * the legacy default stream).  Work is enqueued asynchronously on the stream;
 * argument errors are returned immediately, while data-dependent errors found
 * by kernels (an exact sum whose exponent span exceeds MP_SPAN_CAP, a zero
 * divisor) are recorded in a per-device status word read by mp_check().
 * Kernels record there with an atomic compare-and-swap from MP_OK, so the
 * first error recorded since the last mp_check stays, whichever stream's
 * call recorded it.  Calls that share an mp_csr handle must be ordered on
 * one stream, except a product with A beside one with A^T (mp_spmv_t).
 * There is no CPU fallback: without a usable GPU every compute call returns
 * MP_ERR_CUDA.
 */
#ifndef MPKRYLOV_H
#define MPKRYLOV_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MP_OK = 0,
  MP_ERR_ARG = 1,       /* invalid argument; mp_last_error() has the details */
  MP_ERR_PREC = 2,      /* prec_bits not supported by the call (see above)    */
  MP_ERR_ALLOC = 3,     /* device or host allocation failed                    */
  MP_ERR_CUDA = 4,      /* a CUDA call failed (no device, launch error, ...)   */
  MP_ERR_SPAN = 5,      /* exact sum with exponent span > MP_SPAN_CAP          */
  MP_ERR_BREAKDOWN = 6, /* Krylov breakdown (Fig. 5 "exits")                   */
  MP_ERR_NOCONV = 7,    /* maxit reached (the paper's "NC", Tables 1-2)        */
  MP_ERR_TIMEOUT = 8,   /* a bounded device wait gave up                       */
  MP_ERR_DIVZERO = 9    /* elementwise division by zero                        */
} mp_status;

typedef enum {
  MP_ORDERED = 0, /* each product and each sum rounded, in CSR column order   */
  MP_EXACT = 1    /* each row summed exactly, rounded once                     */
} mp_mode;

typedef enum { MP_OP_MUL = 0, MP_OP_ADD = 1, MP_OP_SUB = 2, MP_OP_DIV = 3 } mp_op;

#define MP_EXP_ZERO (-(INT64_C(1) << 61))
/* Largest exponent span (max minus min term exponent e_a + e_x) of an exact
 * sum (MP_EXACT rows, dot products, residuals). */
#define MP_SPAN_CAP 16384

/* mp_csr_create flags */
#define MP_CSR_TRANSPOSE 1 /* also build A^T (needed by mp_spmv_t and mp_bicg) */

typedef struct mp_csr_s* mp_csr; /* opaque; owns its device storage */

typedef struct {
  int64_t n;          /* number of values                          */
  int32_t prec_bits;  /* p                                          */
  int64_t ld;         /* words between consecutive planes, >= n     */
  uint64_t* data;     /* device pointer to plane 0 (caller-owned)   */
} mp_vec;

/* ---- matrices ----------------------------------------------------------- */

/* Builds a device matrix from a host CSR matrix (Section 2's sparse storage:
 * per-row column indices and the nonzero values at precision prec_bits).
 *   n        rows = columns, 0 <= n < 2^31
 *   rowptr   host, n+1 entries, rowptr[0] = 0, nondecreasing
 *   colidx   host, rowptr[n] entries in [0, n); a row may list its columns
 *            in any order but not twice (the ORDERED sum runs in ascending
 *            column order)
 *   values   host planes, (L+1) * rowptr[n] words: plane k at values + k*nnz
 *   flags    MP_CSR_TRANSPOSE to build A^T as well
 * The host arrays are copied; the caller may free them on return.  The
 * device copy is a sliced, row-length-sorted layout of the same rows (see
 * mp_csr_info).  Returns MP_ERR_ARG for a malformed matrix or value, with the
 * offending row in mp_last_error(). */
mp_status mp_csr_create(int64_t n, const int64_t* rowptr, const int32_t* colidx,
                        const uint64_t* values, int32_t prec_bits, int32_t flags,
                        void* stream, mp_csr* out);

/* As mp_csr_create with double-precision host values, each converted exactly
 * to prec_bits (53 <= p; Section 4 converts the UF matrices this way).
 * NaN or infinite values give MP_ERR_ARG. */
mp_status mp_csr_create_f64(int64_t n, const int64_t* rowptr, const int32_t* colidx,
                            const double* values, int32_t prec_bits, int32_t flags,
                            void* stream, mp_csr* out);

/* Frees the matrix (waits for work queued on it to finish). */
mp_status mp_csr_destroy(mp_csr A);

/* Sizes of a matrix: rows, stored entries, precision, slots of the sliced
 * layout (stored entries plus padding) and device bytes held. Any pointer
 * may be NULL. */
mp_status mp_csr_info(mp_csr A, int64_t* n, int64_t* nnz, int32_t* prec_bits,
                      int64_t* slots, int64_t* device_bytes);

/* Launch configuration of the products of A (a tuning knob, not part of the
 * paper; results never depend on it), per mode MP_ORDERED / MP_EXACT:
 *   threads_per_block: 32, 64, 128 or 256;
 *   variant, a bit field:
 *     bit 0: the row loop loads the next entry's operands while the current
 *            one is computed (MP_ORDERED: p <= 512 only; MP_EXACT: column
 *            form only, the word form does it at p <= 512);
 *     bit 1: products formed from radix-2^29 column sums (one multiply-add
 *            per pair of 29-bit limbs, no carries inside the product; EXACT
 *            then keeps 29-bit digit counters), else from 32-bit words with
 *            carry chains.  EXACT column-form counters add parts below 2^35
 *            per term into 64-bit integers, so a row sum is exact for rows of
 *            up to 2^27 stored entries; the word form (bit 1 clear) adds
 *            32-bit digits and is exact for any row;
 *     bit 2: MP_EXACT column form: 16 columns computed at a time, not 8
 *            (with bit 4: registers capped for four blocks of at most 128
 *            threads per SM);
 *            MP_ORDERED: registers capped for three blocks of at most 128
 *            threads per SM (ignored above 128 threads per block);
 *     bit 3: x is first copied into records (each element's L+1 words
 *            contiguous) and gathered from them: one 16-byte load per two
 *            words instead of one sector per plane.  The copy lives with the
 *            matrix (n (L+2) 8 bytes, allocated on first use), so products of
 *            one matrix with this bit must not run concurrently on several
 *            streams;
 *   carveout: the shared-memory share of the unified L1/shared storage the
 *            kernels ask for, in percent (more digit windows per SM against
 *            more L1 for the gathers of x);
 *   -1 for any of them: the library's default for the precision (and, for
 *            bit 3, the size: on from p = 256 when n >= 65536).
 * mp_csr_get_config reports the configuration that runs (defaults resolved;
 * carveout -1 = the driver's choice). */
mp_status mp_csr_set_config(mp_csr A, int32_t mode, int32_t threads_per_block, int32_t variant,
                            int32_t carveout);
mp_status mp_csr_get_config(mp_csr A, int32_t mode, int32_t* threads_per_block,
                            int32_t* variant, int32_t* carveout);

/* Autotuner: times y = A x (mode) for the configurations above (64-256
 * threads; every variant; for EXACT the carve-outs default, 25, 50 and 75 %)
 * on an internal nonzero x, `reps` launches each, keeps the fastest in A and
 * returns it (as mp_csr_get_config) with its time per product (ms).
 * Allocates two n-vectors for the duration of the call.  Rows whose exponent
 * span exceeds MP_SPAN_CAP record MP_ERR_SPAN in the status word as in
 * mp_spmv. */
mp_status mp_csr_tune(mp_csr A, int32_t mode, int32_t reps, int32_t* threads_per_block,
                      int32_t* variant, int32_t* carveout, double* ms, void* stream);

/* ---- products ------------------------------------------------------------ */

/* y = A x (Section 3's SpMV).  MP_ORDERED: y_i = +0, then for each stored
 * a_ik in ascending column order with a_ik != 0 and x_k != 0 (the zero fast
 * path of Section 2), y_i = RN(y_i + RN(a_ik * x_k)).  MP_EXACT: y_i =
 * RN(sum_k a_ik x_k) with the sum formed exactly (zero terms skipped, an
 * exact zero is +0); a row whose term exponents span more than MP_SPAN_CAP
 * bits becomes +0 and records MP_ERR_SPAN.  x, y: n values at the matrix
 * precision, distinct storage. */
mp_status mp_spmv(mp_csr A, mp_vec x, mp_vec y, mp_mode mode, void* stream);

/* y = A^T x (BiCG's shadow product, Fig. 5); row j of A^T lists the rows i
 * of A with a stored a_ij in ascending i, which is the ORDERED order.
 * Requires MP_CSR_TRANSPOSE at creation.
 * Streams: each of A's two layouts (A, A^T) keeps its own working storage
 * (the record copy of x, the EXACT overflow list), so a product with A
 * (mp_spmv, mp_residual) and one with A^T may run at the same time on
 * different streams; two products with the same layout that overlap on the
 * GPU race on it. */
mp_status mp_spmv_t(mp_csr A, mp_vec x, mp_vec y, mp_mode mode, void* stream);

/* r_i = RN(b_i - sum_k a_ik x_k), summed exactly and rounded once (the
 * initial residual r0 = b - A x0 of Fig. 5). */
mp_status mp_residual(mp_csr A, mp_vec b, mp_vec x, mp_vec r, void* stream);

/* ---- vectors ------------------------------------------------------------- */

/* Longest vectors mp_dot accepts: its 64-bit digit counters, which add the
 * products' 32-bit digits of every element, stay exact for up to 2^31 - 1
 * products.  Longer vectors give MP_ERR_ARG before any CUDA call. */
#define MP_DOT_MAX_N INT64_C(2147483647)

/* out = RN(sum_i x_i y_i) formed exactly and rounded once (the inner
 * products of Fig. 5); zero pairs are skipped, an exact zero is +0.  out is
 * a device scalar (n = 1); n <= MP_DOT_MAX_N.  Uses a per-device scratch buffer allocated on
 * first use and grown (cudaFree, then cudaMalloc) when a later call needs
 * more.  Every call on a device shares that buffer, so calls that overlap on
 * the GPU (on two streams with no ordering between them) race and produce
 * wrong results: order them on one stream.  The solvers do not use it (each
 * solve has its own scratch). */
mp_status mp_dot(mp_vec x, mp_vec y, mp_vec out, void* stream);

/* y_i = RN(y_i + RN(alpha * x_i)); alpha a device scalar. */
mp_status mp_axpy(mp_vec alpha, mp_vec x, mp_vec y, void* stream);

/* out_i = RN(a_i op b_i) for op in mp_op.  A zero divisor gives +0 and
 * records MP_ERR_DIVZERO.  out may alias a or b. */
mp_status mp_ewise(int32_t op, mp_vec a, mp_vec b, mp_vec out, void* stream);

/* Exact conversion of n device doubles into a vector (53 <= p). */
mp_status mp_vec_from_f64(const double* d, mp_vec out, void* stream);

/* Nearest double of each value (reporting only). */
mp_status mp_vec_to_f64(mp_vec a, double* d, void* stream);

/* ---- allocation-free dot product (the paper has no counterpart) ---------- */

/* Longest vectors mp_dot_noalloc accepts (the bound of mp_dot). */
#define MP_DOT_NOALLOC_MAX_N MP_DOT_MAX_N
/* Size of the device array that holds mp_dot_noalloc's scratch. */
#define MP_DOT_NOALLOC_SCRATCH_BYTES 298112

/* The exact dot product of mp_dot (bit-identical results) for callers that
 * cannot let a library allocate device memory: processes whose GPU memory is
 * owned by another allocator (a framework's caching allocator that has
 * reserved the memory, a server held to a fixed memory budget), where a
 * cudaMalloc would fail or break the budget, and latency-bound callers that
 * must avoid the device-wide synchronisation cudaMalloc/cudaFree can cause.
 * It calls no cudaMalloc, cudaFree or other allocating routine: its scratch
 * is a fixed device array of MP_DOT_NOALLOC_SCRATCH_BYTES inside the library,
 * held on every GPU that loads the library until the process exits.  The
 * first call on a device looks up that array's device address
 * (cudaGetSymbolAddress) with the device current; make this first call before
 * any stream capture.  Every call on a device uses the same array, so calls
 * that overlap on the GPU (for example on two streams without ordering
 * between them) race and produce wrong results; order them on one stream.
 * Precisions: p in {128, 256, 512, 1024} only (MP_ERR_PREC otherwise; the
 * wide precisions 2048-8192 need mp_dot).  Vectors longer than
 * MP_DOT_NOALLOC_MAX_N give MP_ERR_ARG; both refusals come before any CUDA
 * call. */
mp_status mp_dot_noalloc(mp_vec x, mp_vec y, mp_vec out, void* stream);

/* ---- solvers (Fig. 5, left preconditioner K = I) ------------------------- */

typedef struct {
  double rtol;       /* stop when (r,r) <= RN(RN(rtol^2)*(r0,r0)) + RN(atol^2) */
  double atol;
  int64_t maxit;     /* iteration limit ("NC" beyond it)                        */
  int32_t mode;      /* mp_mode used for the SpMVs                              */
  int32_t poll_every;/* p > 1024: iterations between host checks of the device
                        flags (>= 1); the solvers at p <= 1024 and the batched
                        solve iterate in a device-side loop and ignore it     */
  mp_vec history;    /* optional (data may be NULL): entry i-1 receives (r_i,r_i) */
  int32_t transpose; /* 1: solve A^T x = b (needs MP_CSR_TRANSPOSE), e.g. an
                        adjoint system; 0: A x = b                            */
  int32_t time_limit_ms; /* 0: none.  > 0 (p <= 1024 and the batched solve):
                        the solve ends with MP_ERR_TIMEOUT when an iteration
                        finishes more than this many milliseconds after the
                        set-up (device clock); x holds that iterate          */
} mp_solve_opts;

typedef struct {
  int64_t iters;  /* completed iterations                                   */
  int32_t status; /* MP_OK (converged), MP_ERR_NOCONV, MP_ERR_BREAKDOWN or
                     MP_ERR_TIMEOUT (time_limit_ms ran out)                 */
  double relres;  /* sqrt((r,r)/(r0,r0)) of the last iterate, as a double    */
  double ms;      /* wall time of the solve on the stream                    */
} mp_solve_info;

/* BiCG (Fig. 5 left).  x holds x0 on entry and the last iterate on return.
 * The iteration runs on the device: after the first iteration the host
 * launches one CUDA graph whose conditional while node replays an iteration
 * until the device state says the solve has ended, then reads a few status
 * bytes (p > 1024: the iterations are launched from the host, which reads
 * the device state every poll_every iterations).
 * Returns info->status.  Needs MP_CSR_TRANSPOSE. */
mp_status mp_bicg(mp_csr A, mp_vec b, mp_vec x, const mp_solve_opts* opts,
                  mp_solve_info* info, void* stream);

/* GPBiCG (Fig. 5 right, Zhang's method: z = zeta r + eta z - alpha u and
 * r = t - eta y - zeta A t). */
mp_status mp_gpbicg(mp_csr A, mp_vec b, mp_vec x, const mp_solve_opts* opts,
                    mp_solve_info* info, void* stream);

/* CGS and BiCGSTAB, the other product-type methods of Section 4's tables
 * (Tables 1-2).  The paper prints no algorithm for them; the textbook forms
 * with K = I and r~ = r0 are taken:
 *   CGS:      u = r + beta q, p = u + beta (q + beta p) (u = p = r0 at i = 1),
 *             v = A p, alpha = rho / (r~, v), q = u - alpha v, w = u + q,
 *             x = x + alpha w, r = r - alpha A w, beta = rho_i / rho_{i-1};
 *   BiCGSTAB: p = r + beta (p - omega v) (p = r0 at i = 1), v = A p,
 *             alpha = rho / (r~, v), s = r - alpha v, t = A s,
 *             omega = (t, s) / (t, t) (+0 when t = 0), x = x + alpha p +
 *             omega s, r = s - omega t, beta = (rho_i/rho_{i-1})(alpha/omega).
 * Every product and sum rounded left to right, inner products exact; the
 * stopping rule, options and statuses as mp_gpbicg (a zero (r~, v) or rho is
 * a breakdown; BiCGSTAB ends with MP_ERR_BREAKDOWN on omega = 0 after the
 * convergence test).  opts->transpose solves with A^T (needs
 * MP_CSR_TRANSPOSE). */
mp_status mp_cgs(mp_csr A, mp_vec b, mp_vec x, const mp_solve_opts* opts, mp_solve_info* info,
                 void* stream);
mp_status mp_bicgstab(mp_csr A, mp_vec b, mp_vec x, const mp_solve_opts* opts,
                      mp_solve_info* info, void* stream);

/* ---- ILU(0) preconditioning (Section 4's BiCGSTAB+ILU(0) rows) ----------- */

typedef struct mp_ilu_s* mp_ilu; /* opaque; owns its device storage */

/* ILU(0) of A in the textbook IKJ form (the paper prints no algorithm), all
 * steps rounded and none skipped: for each row i, for each stored (i, k),
 * k < i ascending, l_ik = RN(a_ik / u_kk) and, for each stored (i, j), j > k
 * ascending with (k, j) stored, a_ij = RN(a_ij - RN(l_ik u_kj)).  L (unit
 * lower) and U share A's pattern.  Rows run in dependency levels, one launch
 * per level (one thread per row at p <= 1024, one warp per row at p = 2048,
 * 4096, 8192, the precisions of Table 3's converging runs).  MP_ERR_DIVZERO:
 * a row without a diagonal entry or a zero pivot.  Synchronises `stream`. */
mp_status mp_ilu0_create(mp_csr A, void* stream, mp_ilu* out);
mp_status mp_ilu0_destroy(mp_ilu M);

/* Levels of the forward and backward triangular solves (launches per solve). */
mp_status mp_ilu0_info(mp_ilu M, int64_t* levels_l, int64_t* levels_u);

/* The factor values in A's CSR order (sorted columns): lu has nnz elements. */
mp_status mp_ilu0_factor(mp_ilu M, mp_vec lu, void* stream);

/* w = (LU)^{-1} r: forward y_i = r_i - RN(l_ik y_k) per step for k < i
 * ascending, then backward w_i = RN((y_i - RN(u_ik w_k) per step for k > i
 * ascending) / u_ii), one launch per level.  r and w must not alias. */
mp_status mp_ilu0_apply(mp_ilu M, mp_vec r, mp_vec w, void* stream);

/* BiCGSTAB with ILU(0) as the left preconditioner K = LU (Section 4.2 and
 * Table 3 run BiCGSTAB left-preconditioned by ILU(0); Fig. 5 names K the
 * left-preconditioning matrix and applies it by solving K w = r).  BiCGSTAB (mp_bicgstab's steps and op order) on the system
 * K^{-1} A x = K^{-1} b: r^0 = K^{-1} RN(b - A x0), v = K^{-1}(A p),
 * t = K^{-1}(A s), x = RN(RN(x + RN(alpha p)) + RN(omega s)),
 * r^ = RN(s - RN(omega t)).  The stopping rule, info->relres and the
 * history take the recursive preconditioned residual r^ against r^0; the
 * true residual b - A x is not formed.  opts->transpose must be 0; M must
 * come from mp_ilu0_create on A.  Statuses as mp_bicgstab, plus
 * MP_ERR_ARG for a preconditioner of another matrix. */
mp_status mp_bicgstab_ilu0(mp_csr A, mp_ilu M, mp_vec b, mp_vec x, const mp_solve_opts* opts,
                           mp_solve_info* info, void* stream);

/* The right-preconditioned form, kept as an option (Barrett et al.'s
 * preconditioned BiCGSTAB): p^ = K^{-1} p, v = A p^, s^ = K^{-1} s,
 * t = A s^, x = x + alpha p^ + omega s^; r remains b - A x of the original
 * system, so the stopping rule is the unpreconditioned one. */
mp_status mp_bicgstab_ilu0_right(mp_csr A, mp_ilu M, mp_vec b, mp_vec x,
                                 const mp_solve_opts* opts, mp_solve_info* info, void* stream);

/* ---- batched solves (not in the paper; its solver over a batch) ---------- */

typedef struct mp_batch_s* mp_batch; /* opaque; owns its device storage */

/* Stacks k independent instances of one precision (instance i: an n_each[i]
 * x n_each[i] CSR matrix with double values, converted exactly) into one
 * block-diagonal device matrix; several right-hand sides of one system are
 * passed as several instances with the same arrays.  Instance i owns
 * elements [off[i], off[i+1]) of the batch's concatenated vectors (see
 * mp_batch_info). */
mp_status mp_batch_create_f64(int32_t k, const int64_t* n_each, const int64_t* const* rowptrs,
                              const int32_t* const* colidxs, const double* const* values,
                              int32_t prec_bits, void* stream, mp_batch* out);

mp_status mp_batch_destroy(mp_batch B);

/* Number of instances, total length and the k+1 offsets (any may be NULL). */
mp_status mp_batch_info(mp_batch B, int32_t* k, int64_t* total_n, int64_t* offsets);

/* The batch's block-diagonal matrix, for mp_csr_set_config / mp_csr_tune /
 * mp_csr_get_config (its launch configuration is the one the batched solve
 * uses).  The handle is owned by the batch: valid until mp_batch_destroy,
 * never passed to mp_csr_destroy. */
mp_status mp_batch_matrix(mp_batch B, mp_csr* out);

/* GPBiCG on every instance at once: one SpMV launch, segmented exact inner
 * products and per-instance scalars per step, one iteration replayed as a
 * CUDA graph until every instance has exited.  Each instance's iterates
 * equal those of mp_gpbicg on that instance alone, bit for bit.  b, x are
 * concatenated vectors (x: x0 in, solutions out); infos[k] receives each
 * instance's iterations and status (relres is not computed, ms is the
 * whole batch).  opts->history must be NULL and opts->transpose 0. */
mp_status mp_batch_gpbicg(mp_batch B, mp_vec b, mp_vec x, const mp_solve_opts* opts,
                          mp_solve_info* infos, void* stream);

/* ---- mixed-precision iterative refinement (not in the paper) ------------- */

typedef struct {
  double rtol;         /* stop when max|dx| <= rtol * max|x| (the correction no
                          longer changes x at this relative level)          */
  int64_t max_outer;   /* corrections at most                                */
  double inner_rtol;   /* relative residual of each FP64 inner solve         */
  int64_t inner_maxit; /* FP64 GPBiCG iterations per inner solve             */
  int32_t equilibrate; /* 1: scale the rows of the FP64 copy by powers of two */
  int32_t poll_every;  /* inner iterations between host checks               */
} mp_refine_opts;

typedef struct {
  int64_t outer;       /* corrections applied                                */
  int64_t inner_iters; /* FP64 GPBiCG iterations over all corrections        */
  int32_t status;      /* MP_OK or MP_ERR_NOCONV                              */
  double correction;   /* last max|dx| / max|x|                              */
  double relres;       /* sqrt((r,r)/(b,b)), r = b - A x exact per row       */
  double ms;           /* wall time on the stream                            */
} mp_refine_info;

/* Solves A x = b at p bits by iterative refinement: r = RN_row(b - A x)
 * (EXACT rows, rounded once, as mp_residual), an FP64 GPBiCG solve of
 * A d = r scaled by 2^-E (E = the largest exponent of r) on a
 * row-equilibrated FP64 copy of A (built on first use and kept with the
 * matrix), then x = RN(x + 2^E d).  FP64 is used only inside the inner solve
 * and its inner products.  x holds x0 on entry.  Returns info->status. */
mp_status mp_refine(mp_csr A, mp_vec b, mp_vec x, const mp_refine_opts* opts,
                    mp_refine_info* info, void* stream);

/* Gradient on the sparsity pattern (the backward pass of a differentiated
 * solve x = A^{-1} b; not in the paper): given the solution x and the adjoint
 * lam with A^T lam = dL/dx, writes g_k = RN((-lam_i) * x_j) = dL/da_ij for
 * every stored entry k = (i, j), at the entry's position in the CSR passed to
 * mp_csr_create (g has n = nnz values).  dL/db is lam itself. */
mp_status mp_csr_grad(mp_csr A, mp_vec lam, mp_vec x, mp_vec g, void* stream);

/* ---- dense product (Section 3's comparison) ----------------------------- */

/* y = A x for a dense m x n p-bit matrix A stored column-major per plane:
 * A is an mp_vec of m*n elements (element (i, j) at index j*m + i, plane
 * stride A.ld), x has n elements, y m.  Each y_i follows the ORDERED row
 * loop of mp_spmv over all columns (y_i = +0, then y_i = RN(y_i +
 * RN(a_ij x_j)) for j ascending, zero factors skipped), so it equals the
 * ORDERED SpMV of the same matrix whether its zeros are stored or dropped
 * (Section 3 compares exactly these two).  x and y must not alias. */
mp_status mp_gemv(int64_t m, int64_t n, mp_vec A, mp_vec x, mp_vec y, void* stream);

/* ---- status -------------------------------------------------------------- */

/* Waits for `stream`, then returns and clears the device-side status word of
 * the current device (MP_OK if no kernel recorded an error). */
mp_status mp_check(void* stream);

const char* mp_status_string(mp_status s);

/* Details of the last error returned on the calling thread. */
const char* mp_last_error(void);

/* Kernels launched by this library on the calling thread since the counter
 * was last reset (reset = 1 clears it after reading). */
int64_t mp_launch_count(int32_t reset);

/* Error-path testing (no counterpart in the paper).  mp_debug_fail arms one
 * named host-side site so that, after `after` further passes through it, the
 * CUDA call there is reported as failed once (cudaErrorUnknown) without
 * being made; the library must then return MP_ERR_CUDA and release what the
 * call had allocated.  Sites: "solver poll" (the host's read of a p <= 1024
 * solver's device state) and "work memory" (each stream-ordered allocation
 * of the work space of a p <= 1024 solver or of mp_refine; a failure there
 * returns MP_ERR_CUDA before any iteration).  site = NULL or "" disarms.  Nothing reaches the
 * GPU: the fault is a fake status on the host.  mp_debug_pool_used returns
 * the bytes in use in the current device's default stream-ordered memory
 * pool (where the solvers take their work memory), to check that a failed
 * call gave them back. */
mp_status mp_debug_fail(const char* site, int64_t after);
mp_status mp_debug_pool_used(int64_t* bytes);

/* Throughput probe of the 32x32->64-bit multiply-add that the p-bit products
 * are made of: runs a dependency-free IMAD.WIDE.U32 loop on every SM and
 * returns the products per second through *rate.  Used for the roofline of
 * the integer-bound kernels. */
mp_status mp_imad_probe(double* rate, void* stream);

#ifdef __cplusplus
}
#endif
#endif
