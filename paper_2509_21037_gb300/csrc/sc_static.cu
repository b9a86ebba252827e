// sc_assemble_batch_static: the batched assembly with its workspace in a
// file-scope device array instead of caller memory (include/sc.h).
//
// Who needs it: callers that cannot call cudaMalloc -- for example a solver
// that runs under a memory manager which reserved the free device memory up
// front (a further cudaMalloc would fail), or a latency-sensitive loop where
// cudaMalloc's implicit device-wide synchronisation is not acceptable.  They
// still bring the inputs and outputs (plan tables, L values, F); only the
// temporary workspace (status word, reciprocal diagonal, sparse Y) moves
// into the library.
//
// The array below is allocated by the CUDA runtime when this module is
// loaded into a CUDA context and stays allocated until that context is
// destroyed (for the primary context of a device: until the process exits).
// Every context that loads the module has its own copy at its own address.
// In host code the array's name is only a host-side stand-in, so its device
// address is looked up with cudaGetSymbolAddress in the calling thread's
// current context on every call (a cheap host-side lookup) and then passed to
// the kernels; an address cached from another context would not be valid.
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "sc_internal.h"

using namespace sc;

namespace {

constexpr size_t kStaticScratchBytes = size_t(64) << 20;   // SC_STATIC_SCRATCH_BYTES in sc.h
static_assert(kStaticScratchBytes == SC_STATIC_SCRATCH_BYTES, "keep sc.h in step");

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

sc_status static_fail(sc_ctx *ctx, cudaError_t e, const char *where) {
  return fail(ctx, SC_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

}  // namespace

extern "C" sc_status sc_assemble_batch_static(sc_ctx *ctx, const double *L_values_dev, double *F_dev,
                                              void *stream) {
  if (!ctx) return SC_ERR_INVALID_ARG;
  if (!ctx->plan_dev && !ctx->blob.empty()) return fail(ctx, SC_ERR_STATE, "sc_upload_plan was not called");
  if (ctx->ws.total > kStaticScratchBytes)
    return fail(ctx, SC_ERR_OOM,
                "this plan needs " + std::to_string(ctx->ws.total) + " bytes of workspace, more than the " +
                    std::to_string(kStaticScratchBytes) +
                    "-byte static scratch; split the batch or use sc_assemble_batch with a caller workspace");
  if (ctx->sizes.L_values > 0 && !L_values_dev) return fail(ctx, SC_ERR_INVALID_ARG, "L_values_dev is NULL");
  if (ctx->sizes.F_doubles > 0 && (!F_dev || (reinterpret_cast<uintptr_t>(F_dev) % 8) != 0))
    return fail(ctx, SC_ERR_INVALID_ARG, "F_dev NULL or misaligned");

  // the array's address in the current context (each context has its own copy)
  void *scratch = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&scratch, g_static_scratch);
  if (e != cudaSuccess) return static_fail(ctx, e, "sc_assemble_batch_static: cudaGetSymbolAddress");

  uint8_t *ws = static_cast<uint8_t *>(scratch);
  uint32_t *status = reinterpret_cast<uint32_t *>(ws + ctx->ws.status_off);
  double *invd = reinterpret_cast<double *>(ws + ctx->ws.invd_off);
  double *Y = reinterpret_cast<double *>(ws + ctx->ws.y_off);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the array keeps the previous call's contents: only the status word must
  // start at zero (every Y entry a call reads is zeroed or written by its own
  // trsm tasks first, and every reciprocal diagonal by its prep kernel)
  e = cudaMemsetAsync(status, 0, sizeof(uint32_t), st);
  if (e != cudaSuccess) return static_fail(ctx, e, "sc_assemble_batch_static: status reset");
  int rc = launch_prep(*ctx, L_values_dev, invd, status, F_dev, ws, stream);
  if (rc) return static_fail(ctx, (cudaError_t)rc, "prep kernel launch");
  for (int w = 0; w < (int)ctx->waves.size() && !rc; ++w)
    rc = launch_groups(*ctx, w, L_values_dev, invd, ws, Y, F_dev, stream, false);   // no extra streams
  if (rc) return static_fail(ctx, (cudaError_t)rc, "assembly kernel launch");
  // report this call's device status (the caller has no handle on the scratch)
  uint32_t h = 0;
  e = cudaMemcpyAsync(&h, status, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return static_fail(ctx, e, "sc_assemble_batch_static: status read");
  if (h & kStatusNotSpd) return fail(ctx, SC_ERR_NOT_SPD, "a diagonal entry of L is not positive and finite");
  if (h & kStatusTimeout)
    return fail(ctx, SC_ERR_TIMEOUT, "a bounded device wait gave up (sc_options.poll_limit polls)");
  if (h) return fail(ctx, SC_ERR_INTERNAL, "unknown device status bits");
  return SC_OK;
}
