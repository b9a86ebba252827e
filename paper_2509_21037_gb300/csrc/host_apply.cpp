// Implicit application of the dual operator on the host (paper Sec. 2.2,
// Eq. "dualop_apply_impl"): per subdomain, x = B_i^T p_i (sparse scatter),
// two triangular solves with the sparse factor (L y = x, L^T z = y), then
// q_i = B_i z (sparse gather), summed into the global dual vector.  This is
// the per-iteration cost the explicit F*lambda saves; with the assembly time
// it gives the amortisation point.  FP64, host threads over subdomains, each
// thread accumulating into its own dual vector (summed at the end), so the
// result does not depend on thread timing.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

#include "sc_factor.h"

namespace {

void apply_one(const scf_apply_subdomain &s, const double *lambda, double *q, std::vector<double> &x) {
  const int32_t n = s.n;
  x.assign(n, 0.0);
  for (int32_t j = 0; j < s.m; ++j) {
    const double pj = lambda[s.lambda_map[j]];
    for (int32_t e = s.Bt_colptr[j]; e < s.Bt_colptr[j + 1]; ++e) x[s.Bt_rowind[e]] += s.Bt_sign[e] * pj;
  }
  // forward: L y = x, column oriented
  for (int32_t c = 0; c < n; ++c) {
    const int64_t a = s.L_colptr[c], b = s.L_colptr[c + 1];
    const double yc = x[c] / s.L_val[a];
    x[c] = yc;
    for (int64_t e = a + 1; e < b; ++e) x[s.L_rowind[e]] -= s.L_val[e] * yc;
  }
  // backward: L^T z = y, row oriented over the columns of L
  for (int32_t c = n - 1; c >= 0; --c) {
    const int64_t a = s.L_colptr[c], b = s.L_colptr[c + 1];
    double acc = x[c];
    for (int64_t e = a + 1; e < b; ++e) acc -= s.L_val[e] * x[s.L_rowind[e]];
    x[c] = acc / s.L_val[a];
  }
  for (int32_t j = 0; j < s.m; ++j) {
    double v = 0.0;
    for (int32_t e = s.Bt_colptr[j]; e < s.Bt_colptr[j + 1]; ++e) v += s.Bt_sign[e] * x[s.Bt_rowind[e]];
    q[s.lambda_map[j]] += v;
  }
}

}  // namespace

extern "C" int scf_implicit_apply(int32_t nsub, const scf_apply_subdomain *subs, int64_t n_dual,
                                  const double *lambda, double *q, int32_t nthreads) {
  if (nsub < 0 || n_dual < 0 || (nsub > 0 && !subs) || (n_dual > 0 && (!lambda || !q))) return SCF_ERR_INVALID_ARG;
  for (int32_t i = 0; i < nsub; ++i) {
    const scf_apply_subdomain &s = subs[i];
    if (s.n < 0 || s.m < 0 || (s.n > 0 && (!s.L_colptr || !s.L_rowind || !s.L_val))) return SCF_ERR_INVALID_ARG;
    for (int32_t j = 0; j < s.m; ++j)
      if (s.lambda_map[j] < 0 || s.lambda_map[j] >= n_dual) return SCF_ERR_INVALID_ARG;
  }
  int32_t T = nthreads > 0 ? nthreads : (int32_t)std::max(1u, std::thread::hardware_concurrency());
  T = std::max(1, std::min(T, nsub));
  std::vector<std::vector<double>> qs(T, std::vector<double>(n_dual, 0.0));
  std::vector<std::thread> pool;
  for (int32_t t = 0; t < T; ++t) {
    pool.emplace_back([&, t]() {
      std::vector<double> x;
      for (int32_t i = t; i < nsub; i += T) apply_one(subs[i], lambda, qs[t].data(), x);
    });
  }
  for (auto &th : pool) th.join();
  std::memset(q, 0, sizeof(double) * (size_t)n_dual);
  for (int32_t t = 0; t < T; ++t)
    for (int64_t k = 0; k < n_dual; ++k) q[k] += qs[t][k];
  return SCF_OK;
}
