// The learned per-subdomain variant choice through the C ABI (include/sc.h,
// sc_subdomain_features / sc_select): plan features on the host, the MLP's
// forward pass in the library's own kernels (include/sc_mlp.h), and the
// choice of the fastest variant predicted to meet an error target.  The
// paper has no learned component; this is the selection of row a9.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "sc_internal.h"
#include "sc_mlp.h"

using namespace sc;

namespace {

float log2p(double x) { return (float)std::log2(std::max(x, 1.0)); }

int n_split(const sc_selector *sel) {
  int k = 0;
  for (int v = 0; v < sel->n_variants; ++v) k += sel->slices[v] != 0;
  return k;
}

sc_status check_selector(sc_ctx *ctx, const sc_selector *sel) {
  if (!sel || sel->n_variants < 1 || sel->n_variants > 64 || !sel->slices || !sel->tiles || !sel->params_dev ||
      sel->n_hidden < 1 || !sel->x_shift || !sel->x_scale || !sel->y_shift || !sel->y_scale)
    return fail(ctx, SC_ERR_INVALID_ARG, "sc_selector: NULL array or bad sizes");
  bool fp64 = false;
  for (int v = 0; v < sel->n_variants; ++v) {
    const int S = sel->slices[v], t = sel->tiles[v];
    if ((S != 0 && (S < 3 || S > 7)) || (t != SC_TILE_32 && t != SC_TILE_TC128) || (S == 0 && t != SC_TILE_32))
      return fail(ctx, SC_ERR_INVALID_ARG, "sc_selector: variant " + std::to_string(v) + " is not (0, 32) or (3..7, 0/1)");
    fp64 = fp64 || S == 0;
  }
  if (!fp64) return fail(ctx, SC_ERR_INVALID_ARG, "sc_selector: the FP64 variant must be among the variants");
  return SC_OK;
}

}  // namespace

extern "C" {

sc_status sc_subdomain_features(const sc_ctx *ctx, const double *L_values_host, float *out) {
  if (!ctx || (!out && ctx->nsub > 0)) return SC_ERR_INVALID_ARG;
  int64_t col = 0;
  for (int32_t i = 0; i < ctx->nsub; ++i) {
    const SubFeat &f = ctx->sub_feat[i];
    float *o = out + (size_t)i * SC_NUM_FEATURES;
    o[0] = log2p(f.n); o[1] = log2p(f.m); o[2] = log2p(f.nnzL); o[3] = log2p(f.supernodes);
    o[4] = log2p(f.max_supernode); o[5] = log2p(f.flops_trsm); o[6] = log2p(f.flops_syrk);
    o[7] = log2p(f.flops_dense); o[8] = log2p(f.y_doubles); o[9] = 0.f;
    if (L_values_host && f.n > 0) {
      double lo = INFINITY, hi = 0.0;
      for (int32_t c = 0; c < (int32_t)f.n; ++c) {
        const double d = L_values_host[ctx->diag_index[col + c]];
        lo = std::min(lo, d);
        hi = std::max(hi, d);
      }
      if (lo > 0.0 && std::isfinite(hi)) o[9] = (float)std::log2(hi / lo);
    }
    col += (int64_t)f.n;
  }
  return SC_OK;
}

sc_status sc_select_workspace(const sc_ctx *ctx, const sc_selector *sel, size_t *ws_floats) {
  if (!ctx || !sel || !ws_floats || sel->n_variants < 1 || sel->n_hidden < 1 || !sel->slices) return SC_ERR_INVALID_ARG;
  sc_mlp_shape sh{SC_NUM_FEATURES, sel->n_hidden, sel->n_variants + n_split(sel)};
  const int64_t B = std::max<int32_t>(ctx->nsub, 1);
  *ws_floats = (size_t)(B * (sh.n_in + sh.n_out) + sc_mlp_workspace_floats(&sh, (int32_t)B));
  return SC_OK;
}

sc_status sc_select(sc_ctx *ctx, const sc_selector *sel, const double *L_values_host, double tol, double margin,
                    float *ws_dev, size_t ws_floats, int8_t *sub_slices, int8_t *sub_tile, void *stream) {
  if (!ctx) return SC_ERR_INVALID_ARG;
  sc_status st = check_selector(ctx, sel);
  if (st != SC_OK) return st;
  if (!(tol > 0.0) || !(margin >= 1.0)) return fail(ctx, SC_ERR_INVALID_ARG, "sc_select: tol <= 0 or margin < 1");
  if (ctx->nsub > 0 && (!sub_slices || !sub_tile)) return fail(ctx, SC_ERR_INVALID_ARG, "sc_select: NULL outputs");
  size_t need = 0;
  sc_select_workspace(ctx, sel, &need);
  if (ws_floats < need || (!ws_dev && ctx->nsub > 0)) return fail(ctx, SC_ERR_OOM, "sc_select: workspace too small");
  if (ctx->nsub == 0) return SC_OK;
  const int B = ctx->nsub, nin = SC_NUM_FEATURES, nsp = n_split(sel), nout = sel->n_variants + nsp;
  sc_mlp_shape sh{nin, sel->n_hidden, nout};
  std::vector<float> X((size_t)B * nin), Y((size_t)B * nout);
  sc_subdomain_features(ctx, L_values_host, X.data());
  for (int i = 0; i < B; ++i)
    for (int k = 0; k < nin; ++k) X[(size_t)i * nin + k] = (X[(size_t)i * nin + k] - sel->x_shift[k]) / sel->x_scale[k];
  float *Xd = ws_dev, *Yd = ws_dev + (size_t)B * nin, *mws = Yd + (size_t)B * nout;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(Xd, X.data(), sizeof(float) * X.size(), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return fail(ctx, SC_ERR_CUDA, std::string("sc_select: ") + cudaGetErrorString(e));
  const int rc = sc_mlp_forward(&sh, sel->params_dev, Xd, B, Yd, mws, stream);
  if (rc != 0) return fail(ctx, SC_ERR_CUDA, "sc_select: MLP forward launch failed");
  e = cudaMemcpyAsync(Y.data(), Yd, sizeof(float) * Y.size(), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(ctx, SC_ERR_CUDA, std::string("sc_select: ") + cudaGetErrorString(e));
  // outputs: log10 time of every variant, then log10 error of every split variant (in variant order)
  for (int i = 0; i < B; ++i) {
    const float *y = Y.data() + (size_t)i * nout;
    int best = -1, k = 0;
    double best_t = INFINITY;
    for (int v = 0; v < sel->n_variants; ++v) {
      const double t = std::pow(10.0, (double)y[v] * sel->y_scale[v] + sel->y_shift[v]);
      bool ok = true;
      if (sel->slices[v] != 0) {
        const int j = sel->n_variants + k++;
        const double err = std::pow(10.0, (double)y[j] * sel->y_scale[j] + sel->y_shift[j]);
        ok = err * margin <= tol;
      }
      if (ok && t < best_t) { best_t = t; best = v; }
    }
    if (best < 0) {                      // only possible with non-finite predictions: FP64
      for (int v = 0; v < sel->n_variants; ++v)
        if (sel->slices[v] == 0) { best = v; break; }
    }
    sub_slices[i] = sel->slices[best];
    sub_tile[i] = sel->tiles[best];
  }
  return SC_OK;
}

}  // extern "C"
