// FP64 fused multiply-add rate probe (include/sc_probe.h): the measured peak
// that the FP64 kernels' roofline fraction is reported against.
#include <cuda_runtime.h>

#include <cstdint>

#include "sc_probe.h"

namespace {

constexpr int kProbeThreads = 256;

__global__ void __launch_bounds__(kProbeThreads) fp64_fma_probe(int32_t iters, double *__restrict__ out) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  // 8 independent chains hide the multiply-add latency; the multiplier and
  // addend keep the values finite and away from subnormals for any iters
  double x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = 1.0 + 1e-3 * (double)((t + k) & 1023);
  const double a = 0.99999999, c = 1e-8;
  for (int32_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  out[t] = s;
}

}  // namespace

extern "C" int sc_probe_fp64_fma(int32_t iters, int32_t blocks_per_sm, double *out_dev, double *flops,
                                 int64_t *out_len, void *stream) {
  if (iters < 1 || blocks_per_sm < 1 || blocks_per_sm > 64 || !flops || !out_len) return 1;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 3;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 3;
  const int64_t blocks = (int64_t)sms * blocks_per_sm;
  *out_len = blocks * kProbeThreads;
  *flops = 2.0 * 8.0 * (double)iters * (double)(*out_len);
  if (!out_dev) return 0;
  fp64_fma_probe<<<(unsigned)blocks, kProbeThreads, 0, static_cast<cudaStream_t>(stream)>>>(iters, out_dev);
  return cudaGetLastError() == cudaSuccess ? 0 : 3;
}
