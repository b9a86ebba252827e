// Dense cuBLAS TRSM + SYRK comparator (include/sc_dense.h): the paper's
// original GPU algorithm (Sec. 3.1), no sparsity used.
#include <cublas_v2.h>
#include <cuda_runtime.h>

#include <new>

#include "sc_dense.h"

struct scd_ctx {
  cublasHandle_t h = nullptr;
};

extern "C" {

int scd_create(scd_ctx **out, int32_t emulation) {
  if (!out) return -1;
  *out = nullptr;
  scd_ctx *c = new (std::nothrow) scd_ctx();
  if (!c) return -1;
  cublasStatus_t s = cublasCreate(&c->h);
  if (s != CUBLAS_STATUS_SUCCESS) { delete c; return (int)s; }
  if (emulation) {
    s = cublasSetMathMode(c->h, CUBLAS_FP64_EMULATED_FIXEDPOINT_MATH);
    if (s == CUBLAS_STATUS_SUCCESS) s = cublasSetEmulationStrategy(c->h, CUBLAS_EMULATION_STRATEGY_EAGER);
    if (s != CUBLAS_STATUS_SUCCESS) { cublasDestroy(c->h); delete c; return (int)s; }
  }
  *out = c;
  return 0;
}

int scd_trsm_syrk(scd_ctx *c, int32_t n, int32_t m, const double *L, double *Y, double *F, void *stream) {
  if (!c || n < 0 || m < 0) return -1;
  if (n == 0 || m == 0) return 0;
  cublasStatus_t s = cublasSetStream(c->h, static_cast<cudaStream_t>(stream));
  if (s != CUBLAS_STATUS_SUCCESS) return (int)s;
  const double one = 1.0, zero = 0.0;
  s = cublasDtrsm(c->h, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_N, CUBLAS_DIAG_NON_UNIT, n, m, &one,
                  L, n, Y, n);
  if (s != CUBLAS_STATUS_SUCCESS) return (int)s;
  s = cublasDsyrk(c->h, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_T, m, n, &one, Y, n, &zero, F, m);
  return (int)s;
}

void scd_destroy(scd_ctx *c) {
  if (!c) return;
  if (c->h) cublasDestroy(c->h);
  delete c;
}

}  // extern "C"
