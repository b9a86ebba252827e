/* sc_dense.h -- dense comparator: the original GPU assembly of the paper
 * (Sec. 3.1, "Original Schur Complement Algorithm"): dense TRSM Y = L^{-1} B^T
 * over the full n x m right-hand side, then SYRK F = Y^T Y (lower triangle),
 * both as cuBLAS FP64 library calls.  It exploits no sparsity; it is the
 * yardstick the sparsity-aware path is measured against.
 *
 * All matrices are device, column-major, caller-owned:
 *   L  -- n x n dense lower triangle of the factor (ld = n), read only
 *   Y  -- n x m: on entry the dense B^T, on exit L^{-1} B^T (ld = n)
 *   F  -- m x m: lower triangle of Y^T Y written (ld = m); upper untouched
 * emulation: 0 = native FP64 (CUBLAS_DEFAULT_MATH); 1 = cuBLAS fixed-point
 * FP64 emulation allowed eagerly (CUBLAS_FP64_EMULATED_FIXEDPOINT_MATH), where
 * the installed cuBLAS offers it for these routines.
 * Errors: nonzero return = cublasStatus_t of the failing call (or -1 for bad
 * arguments).  Asynchronous on `stream` (a cudaStream_t). */
#ifndef SC_DENSE_H
#define SC_DENSE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif
typedef struct scd_ctx scd_ctx;
int scd_create(scd_ctx **out, int32_t emulation);
int scd_trsm_syrk(scd_ctx *ctx, int32_t n, int32_t m, const double *L, double *Y, double *F, void *stream);
void scd_destroy(scd_ctx *ctx);
#ifdef __cplusplus
}
#endif
#endif
