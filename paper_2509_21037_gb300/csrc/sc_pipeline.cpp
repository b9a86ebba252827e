// CPU/GPU pipeline of the numeric assembly stage (include/sc_pipeline.h):
// host numeric factorisation of chunk c+1 overlapped with the host->device
// copy and the GPU assembly of chunk c.  The symbolic stage of every
// subdomain's factorisation (scf_analyze) runs once in scp_create; scp_run
// runs only the numeric stage (scf_numeric), straight into the pinned
// staging buffer.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <mutex>
#include <new>
#include <stdexcept>
#include <string>
#include <thread>
#include <vector>

#include "sc.h"
#include "sc_factor.h"
#include "sc_pipeline.h"

struct scp_ctx {
  std::string err;
  std::vector<scp_subdomain> subs;
  std::vector<scp_chunk> chunks;
  std::vector<scf_factor *> sym;              // per subdomain: the analysed ordering and pattern of L
  std::vector<std::vector<int64_t>> L_off;   // per chunk: the plan's L offsets (hi - lo + 1)
  int32_t nthreads = 1;
  size_t stage_doubles = 0;
  double *stage[2] = {nullptr, nullptr};      // pinned
  cudaStream_t copy = nullptr;
  std::vector<cudaEvent_t> ev_copy0, ev_copy1, ev_asm0, ev_asm1;
  ~scp_ctx() {
    for (scf_factor *f : sym) scf_free(f);
    for (double *p : stage)
      if (p) cudaFreeHost(p);
    for (auto *v : {&ev_copy0, &ev_copy1, &ev_asm0, &ev_asm1})
      for (cudaEvent_t e : *v)
        if (e) cudaEventDestroy(e);
    if (copy) cudaStreamDestroy(copy);
  }
};

namespace {

sc_status pfail(scp_ctx *c, sc_status st, const std::string &m) {
  if (c) c->err = m;
  return st;
}

sc_status cuda_fail(scp_ctx *c, cudaError_t e, const char *where) {
  return pfail(c, SC_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// Numeric factorisation of subdomains [lo, hi) into dst (the chunk's
// concatenated L values), on the analysed patterns.
sc_status factor_chunk(scp_ctx *ctx, int32_t c, double *dst) {
  const scp_chunk &ch = ctx->chunks[c];
  const std::vector<int64_t> &off = ctx->L_off[c];
  const int32_t cnt = ch.hi - ch.lo;
  const int32_t T = std::max(1, std::min(ctx->nthreads, cnt));
  std::atomic<int32_t> next{0};
  std::atomic<int> status{SC_OK};
  std::mutex mu;
  std::string msg;
  auto work = [&]() {
    for (;;) {
      const int32_t k = next.fetch_add(1);
      if (k >= cnt || status.load() != SC_OK) return;
      const int32_t i = ch.lo + k;
      const int rc = scf_numeric(ctx->sym[i], ctx->subs[i].K_val, dst + off[k]);
      sc_status st = SC_OK;
      std::string m;
      if (rc != SCF_OK) {
        st = rc == SCF_ERR_NOT_SPD ? SC_ERR_NOT_SPD : rc == SCF_ERR_OOM ? SC_ERR_INTERNAL : SC_ERR_INVALID_ARG;
        m = "subdomain " + std::to_string(i) + ": host numeric factorisation failed (code " + std::to_string(rc) + ")";
      }
      if (st != SC_OK) {
        int expected = SC_OK;
        if (status.compare_exchange_strong(expected, st)) {
          std::lock_guard<std::mutex> g(mu);
          msg = m;
        }
        return;
      }
    }
  };
  std::vector<std::thread> pool;
  for (int32_t t = 1; t < T; ++t) pool.emplace_back(work);
  work();
  for (auto &th : pool) th.join();
  if (status.load() != SC_OK) return pfail(ctx, (sc_status)status.load(), msg);
  return SC_OK;
}

sc_status create_impl(scp_ctx *ctx, int32_t nsub, const scp_subdomain *subs, int32_t nchunks,
                      const scp_chunk *chunks, int32_t nthreads);
sc_status run_impl(scp_ctx *ctx, void *stream, scp_times *times);

}  // namespace

extern "C" {

sc_status scp_create(scp_ctx **out, int32_t nsub, const scp_subdomain *subs, int32_t nchunks,
                     const scp_chunk *chunks, int32_t nthreads) {
  if (!out) return SC_ERR_INVALID_ARG;
  scp_ctx *ctx = new (std::nothrow) scp_ctx();
  *out = ctx;
  if (!ctx) return SC_ERR_INTERNAL;
  try {
    return create_impl(ctx, nsub, subs, nchunks, chunks, nthreads);
  } catch (const std::exception &e) {
    return pfail(ctx, SC_ERR_INTERNAL, std::string("scp_create: ") + e.what());
  }
}

sc_status scp_run(scp_ctx *ctx, void *stream, scp_times *times) {
  if (!ctx) return SC_ERR_INVALID_ARG;
  try {
    return run_impl(ctx, stream, times);
  } catch (const std::exception &e) {
    return pfail(ctx, SC_ERR_INTERNAL, std::string("scp_run: ") + e.what());
  }
}

}  // extern "C"

namespace {

sc_status create_impl(scp_ctx *ctx, int32_t nsub, const scp_subdomain *subs, int32_t nchunks,
                      const scp_chunk *chunks, int32_t nthreads) {
  if (nsub < 0 || nchunks < 0 || (nsub > 0 && !subs) || (nchunks > 0 && !chunks))
    return pfail(ctx, SC_ERR_INVALID_ARG, "negative counts or NULL arrays");
  ctx->subs.assign(subs, subs + nsub);
  ctx->chunks.assign(chunks, chunks + nchunks);
  ctx->nthreads = nthreads > 0 ? nthreads : (int32_t)std::max(1u, std::thread::hardware_concurrency());
  std::vector<int> covered(nsub, 0);
  for (int32_t c = 0; c < nchunks; ++c) {
    const scp_chunk &ch = ctx->chunks[c];
    if (ch.lo < 0 || ch.hi > nsub || ch.lo > ch.hi || !ch.plan)
      return pfail(ctx, SC_ERR_INVALID_ARG, "chunk " + std::to_string(c) + ": bad range or NULL plan");
    sc_sizes sz{};
    if (sc_get_sizes(ch.plan, &sz) != SC_OK || sz.nsub != ch.hi - ch.lo)
      return pfail(ctx, SC_ERR_INVALID_ARG, "chunk " + std::to_string(c) + ": plan does not hold hi - lo subdomains");
    std::vector<int64_t> F_off(sz.nsub + 1), L_off(sz.nsub + 1);
    sc_get_offsets(ch.plan, F_off.data(), L_off.data());
    ctx->L_off.push_back(L_off);
    ctx->stage_doubles = std::max(ctx->stage_doubles, (size_t)L_off[sz.nsub]);
    if ((sz.L_values > 0 && !ch.L_dev) || (sz.F_doubles > 0 && !ch.F_dev) || !ch.ws_dev || ch.ws_bytes < sz.ws_bytes)
      return pfail(ctx, SC_ERR_INVALID_ARG, "chunk " + std::to_string(c) + ": device buffers missing or too small");
    for (int32_t i = ch.lo; i < ch.hi; ++i) {
      const scp_subdomain &s = ctx->subs[i];
      if (s.n < 0 || (s.n > 0 && (!s.K_colptr || !s.K_rowind || !s.K_val || !s.perm)) || (s.nfixed > 0 && !s.fixed))
        return pfail(ctx, SC_ERR_INVALID_ARG, "subdomain " + std::to_string(i) + ": NULL or negative input");
      covered[i]++;
    }
  }
  for (int32_t i = 0; i < nsub; ++i)
    if (covered[i] != 1) return pfail(ctx, SC_ERR_INVALID_ARG, "every subdomain must lie in exactly one chunk");
  // symbolic stage of every subdomain, on the host threads; its L pattern must be the plan's
  ctx->sym.assign(nsub, nullptr);
  std::vector<int32_t> chunk_of(nsub), index_in(nsub);
  for (int32_t c = 0; c < nchunks; ++c)
    for (int32_t i = ctx->chunks[c].lo; i < ctx->chunks[c].hi; ++i) {
      chunk_of[i] = c;
      index_in[i] = i - ctx->chunks[c].lo;
    }
  std::vector<std::string> why(nsub);
  {
    std::atomic<int32_t> next{0};
    auto work = [&]() {
      for (int32_t i; (i = next.fetch_add(1)) < nsub;) {
        const scp_subdomain &s = ctx->subs[i];
        const int rc = scf_analyze(s.n, s.K_colptr, s.K_rowind, s.nfixed, s.fixed, s.perm, 0, &ctx->sym[i]);
        const std::vector<int64_t> &off = ctx->L_off[chunk_of[i]];
        const int64_t want = off[index_in[i] + 1] - off[index_in[i]];
        if (rc != SCF_OK)
          why[i] = "subdomain " + std::to_string(i) + ": host symbolic factorisation failed (code " +
                   std::to_string(rc) + ")";
        else if (scf_nnz(ctx->sym[i]) != want)
          why[i] = "subdomain " + std::to_string(i) + ": factor has " + std::to_string(scf_nnz(ctx->sym[i])) +
                   " entries, the plan expects " + std::to_string(want);
      }
    };
    const int32_t T = std::max(1, std::min(ctx->nthreads, nsub));
    std::vector<std::thread> pool;
    for (int32_t t = 1; t < T; ++t) pool.emplace_back(work);
    work();
    for (auto &th : pool) th.join();
  }
  for (int32_t i = 0; i < nsub; ++i)
    if (!why[i].empty()) return pfail(ctx, SC_ERR_INVALID_ARG, why[i]);
  cudaError_t e = cudaStreamCreateWithFlags(&ctx->copy, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "copy stream");
  for (int b = 0; b < 2; ++b) {
    e = cudaHostAlloc(reinterpret_cast<void **>(&ctx->stage[b]), std::max<size_t>(1, ctx->stage_doubles) * 8,
                      cudaHostAllocDefault);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "pinned staging buffer");
  }
  for (auto *v : {&ctx->ev_copy0, &ctx->ev_copy1, &ctx->ev_asm0, &ctx->ev_asm1}) {
    v->assign(nchunks, nullptr);
    for (int32_t c = 0; c < nchunks; ++c) {
      e = cudaEventCreate(&(*v)[c]);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "event");
    }
  }
  return SC_OK;
}

sc_status run_impl(scp_ctx *ctx, void *stream, scp_times *times) {
  if (!ctx->copy) return pfail(ctx, SC_ERR_STATE, "scp_create did not complete");
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int32_t nc = (int32_t)ctx->chunks.size();
  double factor_ms = 0.0;
  int64_t h2d = 0;
  const auto t0 = std::chrono::steady_clock::now();
  for (int32_t c = 0; c < nc; ++c) {
    double *buf = ctx->stage[c & 1];
    // the staging buffer is free once the copy that read it two chunks ago is done
    if (c >= 2) {
      const cudaError_t e = cudaEventSynchronize(ctx->ev_copy1[c - 2]);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "staging buffer wait");
    }
    const auto f0 = std::chrono::steady_clock::now();
    const sc_status fs = factor_chunk(ctx, c, buf);
    factor_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - f0).count();
    if (fs != SC_OK) {
      cudaStreamSynchronize(st);
      cudaStreamSynchronize(ctx->copy);
      return fs;
    }
    const scp_chunk &ch = ctx->chunks[c];
    const size_t bytes = (size_t)ctx->L_off[c].back() * 8;
    h2d += (int64_t)bytes;
    cudaError_t e = cudaSuccess;
    // the L buffer may be the one of the chunk two before: wait for its assembly
    if (c >= 2) e = cudaStreamWaitEvent(ctx->copy, ctx->ev_asm1[c - 2], 0);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_copy0[c], ctx->copy);
    if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(ch.L_dev, buf, bytes, cudaMemcpyHostToDevice, ctx->copy);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_copy1[c], ctx->copy);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ctx->ev_copy1[c], 0);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_asm0[c], st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "chunk copy");
    const sc_status as = sc_assemble_batch(ch.plan, ch.L_dev, ch.F_dev, ch.ws_dev, ch.ws_bytes, stream);
    if (as != SC_OK) return pfail(ctx, as, std::string("chunk ") + std::to_string(c) + ": " + sc_last_error(ch.plan));
    e = cudaEventRecord(ctx->ev_asm1[c], st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "event record");
  }
  cudaError_t e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->copy);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "pipeline drain");
  const double wall = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (times) {
    double h2d_ms = 0.0, asm_ms = 0.0;
    for (int32_t c = 0; c < nc; ++c) {
      float a = 0.f, b = 0.f;
      cudaEventElapsedTime(&a, ctx->ev_copy0[c], ctx->ev_copy1[c]);
      cudaEventElapsedTime(&b, ctx->ev_asm0[c], ctx->ev_asm1[c]);
      h2d_ms += a;
      asm_ms += b;
    }
    times->wall_ms = wall;
    times->factor_ms = factor_ms;
    times->h2d_ms = h2d_ms;
    times->assembly_ms = asm_ms;
    times->serial_ms = factor_ms + h2d_ms + asm_ms;
    times->h2d_bytes = h2d;
  }
  return SC_OK;
}

}  // namespace

extern "C" {

const char *scp_last_error(const scp_ctx *ctx) { return ctx ? ctx->err.c_str() : "NULL context"; }

void scp_destroy(scp_ctx *ctx) { delete ctx; }

}  // extern "C"
