/* C client of the library's C ABI (compiled and run by tests/test_c_abi.py):
 * every public header must compile as C, and the host-side entry points must
 * work from C without a GPU.  One subdomain: the 1D chain of n nodes, whose
 * factor L (tridiagonal lower) has the pattern {c, c+1} per column, glued at
 * two dofs; the host factor's two stages on the same chain's stiffness. */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "sc.h"
#include "sc_dense.h"
#include "sc_factor.h"
#include "sc_implicit.h"
#include "sc_mlp.h"
#include "sc_pipeline.h"

#define CHECK(cond, msg)                        \
  do {                                          \
    if (!(cond)) {                              \
      fprintf(stderr, "FAIL: %s\n", msg);       \
      return 1;                                 \
    }                                           \
  } while (0)

int main(void) {
  enum { n = 10, m = 2 };
  int64_t colptr[n + 1];
  int32_t rowind[2 * n - 1];
  int64_t e = 0;
  for (int c = 0; c < n; ++c) {
    colptr[c] = e;
    rowind[e++] = c;
    if (c + 1 < n) rowind[e++] = c + 1;
  }
  colptr[n] = e;
  const int32_t bt_colptr[m + 1] = {0, 1, 2};
  const int32_t bt_rowind[m] = {3, 8};
  const int8_t bt_sign[m] = {1, -1};
  const int32_t lambda_map[m] = {0, 1};
  sc_subdomain_desc d;
  memset(&d, 0, sizeof d);
  d.n = n;
  d.m = m;
  d.L_colptr = colptr;
  d.L_rowind = rowind;
  d.Bt_colptr = bt_colptr;
  d.Bt_rowind = bt_rowind;
  d.Bt_sign = bt_sign;
  d.lambda_map = lambda_map;

  sc_options opt;
  memset(&opt, 0, sizeof opt);
  opt.precision = SC_FP64;
  sc_ctx *ctx = NULL;
  CHECK(sc_plan(&ctx, 1, &d, 2, &opt) == SC_OK, sc_last_error(ctx));
  sc_sizes sz;
  CHECK(sc_get_sizes(ctx, &sz) == SC_OK, "sc_get_sizes");
  CHECK(sz.nsub == 1 && sz.L_values == (int64_t)(2 * n - 1) && sz.F_doubles == 32 * 32, "sizes");
  sc_stats st;
  CHECK(sc_get_stats(ctx, &st) == SC_OK && st.n_supernodes >= 1, "stats");
  void *blob = malloc(sz.plan_bytes);
  CHECK(blob && sc_export_plan(ctx, blob, sz.plan_bytes) == SC_OK, "export plan");
  CHECK(memcmp(blob, "SCPL", 4) == 0, "plan magic");
  free(blob);
  sc_destroy(ctx);

  /* a bad pattern is reported, with a message, not a crash */
  ctx = NULL;
  int32_t bad_rowind[2 * n - 1];
  memcpy(bad_rowind, rowind, sizeof rowind);
  bad_rowind[0] = 1;                                 /* column 0 no longer starts with its diagonal */
  d.L_rowind = bad_rowind;
  CHECK(sc_plan(&ctx, 1, &d, 2, &opt) == SC_ERR_INVALID_ARG, "invalid pattern accepted");
  CHECK(strstr(sc_last_error(ctx), "diagonal") != NULL, sc_last_error(ctx));
  sc_destroy(ctx);
  d.L_rowind = rowind;

  /* the options added to sc_options (tile, sub_tile, poll_limit) are validated on the host */
  {
    sc_options o2;
    memset(&o2, 0, sizeof o2);
    o2.precision = SC_SPLIT_BF16;
    o2.n_slices = 5;
    o2.tile = SC_TILE_TC128;
    o2.poll_limit = 1000;
    CHECK(sc_plan(&ctx, 1, &d, 2, &o2) == SC_OK, sc_last_error(ctx));
    float feat[SC_NUM_FEATURES];
    CHECK(sc_subdomain_features(ctx, NULL, feat) == SC_OK && feat[0] > 0.f && feat[9] == 0.f, "features");
    sc_destroy(ctx);
    const int8_t bad_tile[1] = {2};
    o2.sub_tile = bad_tile;
    CHECK(sc_plan(&ctx, 1, &d, 2, &o2) == SC_ERR_INVALID_ARG, "sub_tile 2 accepted");
    sc_destroy(ctx);
    o2.sub_tile = NULL;
    o2.poll_limit = -1;
    CHECK(sc_plan(&ctx, 1, &d, 2, &o2) == SC_ERR_INVALID_ARG, "negative poll_limit accepted");
    sc_destroy(ctx);
    /* general B^T values in place of the signs */
    const double bt_val[2] = {0.5, -3.0};
    sc_subdomain_desc dv = d;
    dv.Bt_sign = NULL;
    dv.Bt_val = bt_val;
    CHECK(sc_plan(&ctx, 1, &dv, 2, NULL) == SC_OK, sc_last_error(ctx));
    sc_destroy(ctx);
    const double bt_nan[2] = {0.5, NAN};
    dv.Bt_val = bt_nan;
    CHECK(sc_plan(&ctx, 1, &dv, 2, NULL) == SC_ERR_INVALID_ARG, "non-finite B^T value accepted");
    sc_destroy(ctx);
    ctx = NULL;
  }

  sci_ctx *ic = NULL;
  CHECK(sci_plan(&ic, 1, &d, 2, NULL) == SC_OK, sci_last_error(ic));
  sci_sizes is;
  CHECK(sci_get_sizes(ic, &is) == SC_OK, "sci_get_sizes");
  CHECK(is.L_values == (int64_t)(2 * n - 1) && is.nnz_visited > 0 && is.flops == 4.0 * (double)is.nnz_visited,
        "implicit sizes");
  sci_destroy(ic);

  /* host factor from C: the chain's stiffness (full symmetric CSC, node 0
   * fixed), symbolic stage once, numeric stage into caller memory, equal to
   * the one-call factorisation; then K -> 4 K gives L -> 2 L on free columns */
  {
    int64_t kcp[n + 1];
    int32_t kri[3 * n - 2];
    double kv[3 * n - 2], k4[3 * n - 2];
    int64_t q = 0;
    for (int c = 0; c < n; ++c) {
      kcp[c] = q;
      if (c > 0) { kri[q] = c - 1; kv[q++] = -1.0; }
      kri[q] = c; kv[q++] = (c == 0 || c == n - 1) ? 1.0 : 2.0;
      if (c + 1 < n) { kri[q] = c + 1; kv[q++] = -1.0; }
    }
    kcp[n] = q;
    for (int64_t k = 0; k < q; ++k) k4[k] = 4.0 * kv[k];
    const int32_t fixed0[1] = {0};
    scf_factor *sym = NULL, *one = NULL;
    CHECK(scf_analyze(n, kcp, kri, 1, fixed0, NULL, 0, &sym) == SCF_OK, "scf_analyze");
    CHECK(scf_factorize(n, kcp, kri, kv, 1, fixed0, NULL, 0, &one) == SCF_OK, "scf_factorize");
    const int64_t nnz = scf_nnz(sym);
    CHECK(nnz == scf_nnz(one) && nnz == 2 * n - 2, "factor pattern size"); /* node 0: unit column */
    double a[2 * n - 1], b[2 * n - 1], c4[2 * n - 1];
    CHECK(scf_numeric(sym, kv, a) == SCF_OK && scf_numeric(sym, k4, c4) == SCF_OK, "scf_numeric");
    CHECK(scf_export(one, NULL, NULL, b, NULL) == SCF_OK, "scf_export");
    CHECK(memcmp(a, b, sizeof(double) * (size_t)nnz) == 0, "numeric stage differs from scf_factorize");
    for (int64_t k = 1; k < nnz; ++k) CHECK(c4[k] == 2.0 * a[k], "K -> 4K must give L -> 2L");
    CHECK(c4[0] == 1.0, "fixed dof keeps its unit column");
    CHECK(scf_numeric(NULL, kv, a) == SCF_ERR_INVALID_ARG, "NULL handle accepted");
    for (int64_t k = 0; k < q; ++k) k4[k] = -kv[k];
    CHECK(scf_numeric(sym, k4, a) == SCF_ERR_NOT_SPD, "indefinite matrix accepted");
    /* host implicit apply from C: planned and column by column agree */
    {
      double lv[2 * n - 1];
      CHECK(scf_numeric(sym, kv, lv) == SCF_OK, "scf_numeric for the implicit apply");
      int64_t lcp[n + 1];
      int32_t lri[2 * n - 1];
      CHECK(scf_export(sym, lcp, lri, NULL, NULL) == SCF_OK, "scf_export pattern");
      scf_apply_subdomain as;
      memset(&as, 0, sizeof as);
      as.n = n;
      as.m = m;
      as.L_colptr = lcp;
      as.L_rowind = lri;
      as.L_val = lv;
      as.Bt_colptr = bt_colptr;
      as.Bt_rowind = bt_rowind;
      as.Bt_sign = bt_sign;
      as.lambda_map = lambda_map;
      const double lam[m] = {0.75, -1.5};
      double q1[m], q2[m];
      scf_implicit *ip = NULL;
      CHECK(scf_implicit_apply(1, &as, m, lam, q1, 1) == SCF_OK, "scf_implicit_apply");
      CHECK(scf_implicit_plan(1, &as, m, &ip) == SCF_OK && ip, "scf_implicit_plan");
      CHECK(scf_implicit_run(ip, lam, q2, 1) == SCF_OK, "scf_implicit_run");
      for (int j = 0; j < m; ++j) CHECK(fabs(q1[j] - q2[j]) <= 1e-14 * (fabs(q1[j]) + 1.0), "planned apply differs");
      CHECK(scf_implicit_run(NULL, lam, q2, 1) == SCF_ERR_INVALID_ARG, "NULL plan accepted");
      scf_implicit_free(ip);
    }
    scf_free(sym);
    scf_free(one);
  }

  sc_mlp_shape shape = {10, 64, 8};
  CHECK(sc_mlp_param_count(&shape) == 64 * 10 + 64 + 64 * 64 + 64 + 8 * 64 + 8, "mlp parameter count");

  printf("C ABI OK: %lld plan bytes, %lld supernodes, %lld visited entries\n", (long long)sz.plan_bytes,
         (long long)st.n_supernodes, (long long)is.nnz_visited);
  return 0;
}
