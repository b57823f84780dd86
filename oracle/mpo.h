/* mpo.h -- CPU oracle for p-bit CSR SpMV, exact dot products and the Krylov solvers.
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, plain reference that the
 * GPU path is checked against.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it; the product library never links,
 * loads or calls it, and it shares no code with the product.
 *
 * Arithmetic follows the paper's MPFR setting (Section 2): every operation is a
 * correctly rounded binary operation at precision p, round-to-nearest with ties
 * to even (MPFR's RN).  p is one of 128, 256, 512, 1024 (libmpo.so) or also
 * 2048, 4096, 8192 (libmpo_wide.so, the same source built with -DWMAX=256;
 * the paper's solves of Tables 1-2 need up to 8192 bits).
 *
 * Value record ("interchange record"), L = p/64 uint64 words + 1 head word:
 *   rec[0]     head = exp*2 + sign   (int64; sign 1 = negative)
 *   rec[1+k]   mantissa limb k, k = 0 least significant
 * A nonzero value is (-1)^sign * M * 2^(exp-p) with 2^(p-1) <= M < 2^p (the
 * MPFR convention 0.1xxx_2 * 2^exp).  Zero has exp == MPO_EXP_ZERO and M = 0;
 * its sign is kept.  Nonzero exponents must satisfy |exp| < 2^60.
 * Vectors are arrays of records (record i at rec + i*(L+1)).
 */
#ifndef MPO_H
#define MPO_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MPO_EXP_ZERO (-(INT64_C(1) << 61))
#define MPO_EXP_LIMIT (INT64_C(1) << 60)
/* Largest exponent span (max minus min term exponent) an exact sum accepts. */
#define MPO_SPAN_CAP 16384

/* Status codes.  Numeric values agree with the product library's status
 * enumeration so that tests can compare them directly. */
enum {
  MPO_OK = 0,
  MPO_ERR_ARG = 1,
  MPO_ERR_PREC = 2,
  MPO_ERR_SPAN = 5,
  MPO_ERR_BREAKDOWN = 6,
  MPO_ERR_NOCONV = 7,
  MPO_ERR_DIVZERO = 9
};

enum { MPO_ORDERED = 0, MPO_EXACT = 1 };
enum { MPO_OP_MUL = 0, MPO_OP_ADD = 1, MPO_OP_SUB = 2, MPO_OP_DIV = 3 };

/* Elementwise r_i = RN(a_i op b_i) over n records. */
int mpo_ewise(int p, int op, int64_t n, const uint64_t *a, const uint64_t *b,
              uint64_t *r);
/* Three-way compare of two records: writes -1, 0 or 1 (zeros compare equal). */
int mpo_cmp(int p, const uint64_t *a, const uint64_t *b, int *out);
/* Exact conversion of doubles to p-bit records (53 <= p, so exact). */
int mpo_from_f64(int p, int64_t n, const double *d, uint64_t *out);
/* Nearest double of each record (for reporting only). */
int mpo_to_f64(int p, int64_t n, const uint64_t *a, double *out);

/* y = A x over rows [r0, r1) of an n x n CSR matrix (columns sorted ascending
 * within a row).  mode MPO_ORDERED or MPO_EXACT.  Rows outside the range are
 * not written.  Returns MPO_ERR_SPAN if an EXACT row exceeded the span cap
 * (that row is written as +0). */
int mpo_spmv_rows(int p, int mode, int64_t n, const int64_t *rowptr,
                  const int32_t *colidx, const uint64_t *vals, const uint64_t *x,
                  uint64_t *y, int64_t r0, int64_t r1);
int mpo_spmv(int p, int mode, int64_t n, const int64_t *rowptr,
             const int32_t *colidx, const uint64_t *vals, const uint64_t *x,
             uint64_t *y);
/* Explicit transpose by a stable counting sort: row j of A^T lists the rows i
 * of A with a_ij stored, in ascending i.  trowptr has n+1 entries. */
int mpo_transpose(int p, int64_t n, const int64_t *rowptr, const int32_t *colidx,
                  const uint64_t *vals, int64_t *trowptr, int32_t *tcolidx,
                  uint64_t *tvals);
/* y = A^T x (the SpMV above applied to the explicit transpose). */
int mpo_spmv_t(int p, int mode, int64_t n, const int64_t *rowptr,
               const int32_t *colidx, const uint64_t *vals, const uint64_t *x,
               uint64_t *y);
/* out = RN(sum_i x_i*y_i), summed exactly and rounded once. */
int mpo_dot(int p, int64_t n, const uint64_t *x, const uint64_t *y, uint64_t *out);
/* y_i = RN(y_i + RN(alpha*x_i)). */
int mpo_axpy(int p, int64_t n, const uint64_t *alpha, const uint64_t *x,
             uint64_t *y);
/* r_i = RN(b_i - sum_k a_k x_col(k)), summed exactly and rounded once. */
int mpo_residual(int p, int64_t n, const int64_t *rowptr, const int32_t *colidx,
                 const uint64_t *vals, const uint64_t *b, const uint64_t *x,
                 uint64_t *r);

/* Krylov solves.  x holds x0 on entry and the last iterate on exit.
 * hist (may be NULL) receives maxit records: (r_i, r_i) after iteration i.
 * iters receives the number of completed iterations.  Returns MPO_OK on
 * convergence, MPO_ERR_NOCONV, MPO_ERR_BREAKDOWN or an argument error. */
int mpo_bicg(int p, int mode, int64_t n, const int64_t *rowptr,
             const int32_t *colidx, const uint64_t *vals, const uint64_t *b,
             uint64_t *x, double rtol, double atol, int64_t maxit,
             int64_t *iters, uint64_t *hist);
int mpo_gpbicg(int p, int mode, int64_t n, const int64_t *rowptr,
               const int32_t *colidx, const uint64_t *vals, const uint64_t *b,
               uint64_t *x, double rtol, double atol, int64_t maxit,
               int64_t *iters, uint64_t *hist);
/* CGS and BiCGSTAB (the other product-type methods of Section 4's tables;
 * the paper prints no algorithm, the textbook forms with K = I are taken):
 * same arguments, statuses and exit order as the solvers above. */
int mpo_cgs(int p, int mode, int64_t n, const int64_t *rowptr,
            const int32_t *colidx, const uint64_t *vals, const uint64_t *b,
            uint64_t *x, double rtol, double atol, int64_t maxit,
            int64_t *iters, uint64_t *hist);
int mpo_bicgstab(int p, int mode, int64_t n, const int64_t *rowptr,
                 const int32_t *colidx, const uint64_t *vals, const uint64_t *b,
                 uint64_t *x, double rtol, double atol, int64_t maxit,
                 int64_t *iters, uint64_t *hist);

/* ILU(0) (textbook IKJ form, every operation rounded): lu receives L (unit
 * lower, left of the diagonal) and U (diagonal and right) in A's CSR order.
 * mpo_ilu0_apply computes w = (LU)^{-1} r.  mpo_bicgstab_ilu0 is BiCGSTAB
 * left-preconditioned with K = LU (Section 4.2: BiCGSTAB on K^{-1} A x =
 * K^{-1} b; the stopping rule and the history take the preconditioned
 * residual K^{-1}(b - A x)); mpo_bicgstab_ilu0_right is the right-
 * preconditioned form (r stays b - A x).  A zero pivot returns
 * MPO_ERR_DIVZERO. */
int mpo_ilu0(int p, int64_t n, const int64_t *rowptr, const int32_t *colidx,
             const uint64_t *vals, uint64_t *lu);
int mpo_ilu0_apply(int p, int64_t n, const int64_t *rowptr, const int32_t *colidx,
                   const uint64_t *lu, const uint64_t *r, uint64_t *w);
int mpo_bicgstab_ilu0(int p, int mode, int64_t n, const int64_t *rowptr,
                      const int32_t *colidx, const uint64_t *vals, const uint64_t *b,
                      uint64_t *x, double rtol, double atol, int64_t maxit,
                      int64_t *iters, uint64_t *hist);
int mpo_bicgstab_ilu0_right(int p, int mode, int64_t n, const int64_t *rowptr,
                            const int32_t *colidx, const uint64_t *vals, const uint64_t *b,
                            uint64_t *x, double rtol, double atol, int64_t maxit,
                            int64_t *iters, uint64_t *hist);

#ifdef __cplusplus
}
#endif
#endif
