// C ABI entry points that touch the GPU: plan upload, batched assembly,
// device status, explicit application and export (include/sc.h).
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "sc_internal.h"

using namespace sc;

namespace {

sc_status cuda_fail(sc_ctx *ctx, int err, const char *where) {
  return fail(ctx, SC_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString((cudaError_t)err));
}

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

void destroy_events(sc_ctx *ctx) {
  for (auto &e : ctx->stage_events) {
    if (e) cudaEventDestroy(static_cast<cudaEvent_t>(e));
    e = nullptr;
  }
  ctx->stage_recorded = false;
}

void record(sc_ctx *ctx, int k, cudaStream_t st) {
  if (ctx->stage_events[k]) cudaEventRecord(static_cast<cudaEvent_t>(ctx->stage_events[k]), st);
}

}  // namespace

sc_ctx::~sc_ctx() {
  destroy_events(this);
  for (auto &e : aux_done)
    if (e) cudaEventDestroy(static_cast<cudaEvent_t>(e));
  for (auto &s : aux_streams)
    if (s) cudaStreamDestroy(static_cast<cudaStream_t>(s));
  if (fork_event) cudaEventDestroy(static_cast<cudaEvent_t>(fork_event));
}

std::vector<int> sc_ctx::groups(int w) const {
  std::vector<int> g;
  for (int v = 0; v < kNumVariants; ++v)
    if (waves[w].trsm[v][1] > 0 || waves[w].syrk[v][1] > 0) g.push_back(v);
  return g;
}

namespace sc {

int launch_groups(sc_ctx &c, int w, const double *Lv, const double *invd, void *ws, double *Y, double *F,
                  void *stream, bool aux) {
  const std::vector<int> g = c.groups(w);
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!aux || g.size() <= 1) {
    for (int v : g) {
      int e = launch_group_trsm(c, w, v, Lv, invd, ws, Y, stream);
      if (e) return e;
    }
    for (int v : g) {
      int e = launch_group_syrk(c, w, v, Y, ws, F, stream);
      if (e) return e;
    }
    return 0;
  }
  cudaError_t e;
  if (!c.fork_event) {
    cudaEvent_t ev;
    if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return (int)e;
    c.fork_event = ev;
  }
  if ((e = cudaEventRecord(static_cast<cudaEvent_t>(c.fork_event), st)) != cudaSuccess) return (int)e;
  for (int v : g) {
    if (!c.aux_streams[v]) {
      cudaStream_t s;
      cudaEvent_t ev;
      if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) return (int)e;
      c.aux_streams[v] = s;
      if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return (int)e;
      c.aux_done[v] = ev;
    }
    cudaStream_t s = static_cast<cudaStream_t>(c.aux_streams[v]);
    if ((e = cudaStreamWaitEvent(s, static_cast<cudaEvent_t>(c.fork_event), 0)) != cudaSuccess) return (int)e;
    int rc = launch_group_trsm(c, w, v, Lv, invd, ws, Y, s);
    if (!rc) rc = launch_group_syrk(c, w, v, Y, ws, F, s);
    if (rc) return rc;
    if ((e = cudaEventRecord(static_cast<cudaEvent_t>(c.aux_done[v]), s)) != cudaSuccess) return (int)e;
    if ((e = cudaStreamWaitEvent(st, static_cast<cudaEvent_t>(c.aux_done[v]), 0)) != cudaSuccess) return (int)e;
  }
  return 0;
}

}  // namespace sc

extern "C" {

sc_status sc_enable_stage_timing(sc_ctx *ctx, int32_t on) {
  if (!ctx) return SC_ERR_INVALID_ARG;
  destroy_events(ctx);
  if (on) {
    for (auto &e : ctx->stage_events) {
      cudaEvent_t ev;
      cudaError_t err = cudaEventCreate(&ev);
      if (err != cudaSuccess) { destroy_events(ctx); return cuda_fail(ctx, err, "sc_enable_stage_timing"); }
      e = ev;
    }
  }
  return SC_OK;
}

sc_status sc_stage_times(sc_ctx *ctx, float *ms, int32_t n) {
  if (!ctx || (!ms && n > 0)) return SC_ERR_INVALID_ARG;
  if (!ctx->stage_events[0] || !ctx->stage_recorded) return fail(ctx, SC_ERR_STATE, "no timed assembly recorded");
  cudaError_t e = cudaEventSynchronize(static_cast<cudaEvent_t>(ctx->stage_events[3]));
  if (e != cudaSuccess) return cuda_fail(ctx, e, "sc_stage_times");
  for (int k = 0; k < n && k < 3; ++k) {
    e = cudaEventElapsedTime(&ms[k], static_cast<cudaEvent_t>(ctx->stage_events[k]),
                             static_cast<cudaEvent_t>(ctx->stage_events[k + 1]));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "sc_stage_times elapsed");
  }
  return SC_OK;
}


sc_status sc_upload_plan(sc_ctx *ctx, void *plan_dev, size_t plan_bytes, void *stream) {
  if (!ctx) return SC_ERR_INVALID_ARG;
  if (plan_bytes < ctx->blob.size()) return fail(ctx, SC_ERR_OOM, "plan buffer smaller than sizes.plan_bytes");
  if (!ctx->blob.empty() && (!plan_dev || !aligned(plan_dev, 16)))
    return fail(ctx, SC_ERR_INVALID_ARG, "plan_dev is NULL or not 16-byte aligned");
  if (!ctx->blob.empty()) {
    cudaError_t e = cudaMemcpyAsync(plan_dev, ctx->blob.data(), ctx->blob.size(), cudaMemcpyHostToDevice,
                                    static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "sc_upload_plan");
  }
  ctx->plan_dev = plan_dev;
  ctx->plan_dev_bytes = plan_bytes;
  return SC_OK;
}

sc_status sc_assemble_batch(sc_ctx *ctx, const double *L_values_dev, double *F_dev, void *ws_dev,
                            size_t ws_bytes, void *stream) {
  if (!ctx) return SC_ERR_INVALID_ARG;
  if (!ctx->plan_dev && !ctx->blob.empty()) return fail(ctx, SC_ERR_STATE, "sc_upload_plan was not called");
  if (ws_bytes < ctx->ws.total) return fail(ctx, SC_ERR_OOM, "workspace smaller than sizes.ws_bytes");
  if (!ws_dev || !aligned(ws_dev, 256)) return fail(ctx, SC_ERR_INVALID_ARG, "ws_dev NULL or not 256-byte aligned");
  if (ctx->sizes.L_values > 0 && !L_values_dev) return fail(ctx, SC_ERR_INVALID_ARG, "L_values_dev is NULL");
  if (ctx->sizes.F_doubles > 0 && (!F_dev || !aligned(F_dev, 8)))
    return fail(ctx, SC_ERR_INVALID_ARG, "F_dev NULL or misaligned");
  uint8_t *ws = static_cast<uint8_t *>(ws_dev);
  uint32_t *status = reinterpret_cast<uint32_t *>(ws + ctx->ws.status_off);
  double *invd = reinterpret_cast<double *>(ws + ctx->ws.invd_off);
  double *Y = reinterpret_cast<double *>(ws + ctx->ws.y_off);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(uint32_t), st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "sc_assemble_batch status reset");
  record(ctx, 0, st);
  int rc = launch_prep(*ctx, L_values_dev, invd, status, F_dev, ws, stream);
  if (rc) return cuda_fail(ctx, rc, "prep kernel launch");
  record(ctx, 1, st);
  const std::vector<int> g0 = ctx->waves.empty() ? std::vector<int>() : ctx->groups(0);
  if (ctx->waves.size() == 1 && g0.size() == 1) {   // one wave, one variant: events around TRSM and SYRK
    rc = launch_group_trsm(*ctx, 0, g0[0], L_values_dev, invd, ws, Y, stream);
    if (rc) return cuda_fail(ctx, rc, "trsm kernel launch");
    record(ctx, 2, st);
    rc = launch_group_syrk(*ctx, 0, g0[0], Y, ws, F_dev, stream);
    if (rc) return cuda_fail(ctx, rc, "syrk kernel launch");
  } else {                 // waves in order, variants of a wave concurrently; stage [1] covers all
    for (int w = 0; w < (int)ctx->waves.size(); ++w) {
      rc = launch_groups(*ctx, w, L_values_dev, invd, ws, Y, F_dev, stream, true);
      if (rc) return cuda_fail(ctx, rc, "variant group launch");
    }
    record(ctx, 2, st);
  }
  record(ctx, 3, st);
  ctx->stage_recorded = ctx->stage_events[0] != nullptr;
  return SC_OK;
}

sc_status sc_device_status(sc_ctx *ctx, const void *ws_dev, void *stream) {
  if (!ctx || !ws_dev) return SC_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "sc_device_status synchronize");
  uint32_t h = 0;
  e = cudaMemcpy(&h, static_cast<const uint8_t *>(ws_dev) + ctx->ws.status_off, sizeof(h), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "sc_device_status read");
  if (h & kStatusNotSpd) return fail(ctx, SC_ERR_NOT_SPD, "a diagonal entry of L is not positive and finite");
  if (h & kStatusTimeout)
    return fail(ctx, SC_ERR_TIMEOUT, "a bounded device wait gave up (sc_options.poll_limit polls)");
  if (h) return fail(ctx, SC_ERR_INTERNAL, "unknown device status bits");
  return SC_OK;
}

sc_status sc_apply(sc_ctx *ctx, const double *F_dev, const double *lambda_dev, double *q_dev, void *stream) {
  if (!ctx) return SC_ERR_INVALID_ARG;
  if (!ctx->plan_dev && !ctx->blob.empty()) return fail(ctx, SC_ERR_STATE, "sc_upload_plan was not called");
  if (!ctx->has_lambda) return fail(ctx, SC_ERR_STATE, "planned without lambda_map");
  if (ctx->n_dual > 0 && (!lambda_dev || !q_dev)) return fail(ctx, SC_ERR_INVALID_ARG, "lambda_dev or q_dev is NULL");
  if (ctx->sizes.F_doubles > 0 && !F_dev) return fail(ctx, SC_ERR_INVALID_ARG, "F_dev is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (ctx->n_dual > 0) {
    cudaError_t e = cudaMemsetAsync(q_dev, 0, sizeof(double) * (size_t)ctx->n_dual, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "sc_apply zero q");
  }
  int rc = launch_apply(*ctx, F_dev, lambda_dev, q_dev, stream);
  if (rc) return cuda_fail(ctx, rc, "apply kernel launch");
  return SC_OK;
}

sc_status sc_export_F(sc_ctx *ctx, const double *F_dev, int32_t i, double *dst_dev, int32_t ld, void *stream) {
  if (!ctx) return SC_ERR_INVALID_ARG;
  if (!ctx->plan_dev && !ctx->blob.empty()) return fail(ctx, SC_ERR_STATE, "sc_upload_plan was not called");
  if (i < 0 || i >= ctx->nsub) return fail(ctx, SC_ERR_INVALID_ARG, "subdomain index out of range");
  if (ld < ctx->m[i] || ld < 1) return fail(ctx, SC_ERR_INVALID_ARG, "ld < m_i");
  if (ctx->m[i] > 0 && (!F_dev || !dst_dev)) return fail(ctx, SC_ERR_INVALID_ARG, "NULL device pointer");
  int rc = launch_export(*ctx, F_dev, i, dst_dev, ld, stream);
  if (rc) return cuda_fail(ctx, rc, "export kernel launch");
  return SC_OK;
}

}  // extern "C"
