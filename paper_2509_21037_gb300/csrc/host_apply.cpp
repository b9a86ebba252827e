// Implicit application of the dual operator on the host (paper Sec. 2.2,
// Eq. "dualop_apply_impl"): per subdomain, x = B_i^T p_i (sparse scatter),
// two triangular solves with the sparse factor (L y = x, L^T z = y), then
// q_i = B_i z (sparse gather), summed into the global dual vector.  This is
// the per-iteration cost the explicit F*lambda saves; with the assembly time
// it gives the amortisation point.  FP64, host threads over subdomains, each
// thread accumulating into its own dual vector (summed at the end), so the
// result does not depend on thread timing.
#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstring>
#include <new>
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

struct SubPlan {
  std::vector<int32_t> sn;        // supernode starts, sn.back() == n
  std::vector<int32_t> visit;     // supernodes on the etree paths from B^T's rows, ascending
  int64_t max_below = 0;          // largest row count below a supernode's diagonal block
};

// Supernodes (runs of columns f..l-1 where column c+1's pattern is column
// c's minus c, checked entry by entry) and the ones the solves need: those
// holding B^T's rows and, transitively, every supernode holding a row that a
// needed one updates (for a Cholesky pattern: the etree paths from B^T's rows
// to the root).  The forward right-hand side is zero elsewhere, and the
// backward solve is read only at B^T's rows, which depend on those alone.
void plan_one(const scf_apply_subdomain &s, SubPlan &P) {
  const int32_t n = s.n;
  const int64_t *cp = s.L_colptr;
  const int32_t *ri = s.L_rowind;
  P.sn.assign(1, 0);
  for (int32_t c = 1; c < n; ++c) {
    const int64_t la = cp[c] - cp[c - 1], lb = cp[c + 1] - cp[c];
    const bool merge = la == lb + 1 && la > 1 && ri[cp[c - 1] + 1] == c &&
                       std::equal(ri + cp[c - 1] + 1, ri + cp[c], ri + cp[c]);
    if (!merge) P.sn.push_back(c);
  }
  if (n > 0) P.sn.push_back(n);
  const int32_t nsn = (int32_t)P.sn.size() - 1;
  std::vector<int32_t> sn_of(n);
  for (int32_t J = 0; J < nsn; ++J)
    for (int32_t c = P.sn[J]; c < P.sn[J + 1]; ++c) sn_of[c] = J;
  std::vector<char> mark(std::max(nsn, 0), 0);
  for (int32_t j = 0; j < s.m; ++j)
    for (int32_t e = s.Bt_colptr[j]; e < s.Bt_colptr[j + 1]; ++e) mark[sn_of[s.Bt_rowind[e]]] = 1;
  P.visit.clear();
  P.max_below = 0;
  for (int32_t J = 0; J < nsn; ++J) {            // a parent supernode comes after its children
    const int32_t f = P.sn[J], ns = P.sn[J + 1] - f;
    const int64_t nr = cp[f + 1] - cp[f];
    if (!mark[J]) continue;
    P.visit.push_back(J);
    P.max_below = std::max(P.max_below, nr - ns);
    // every supernode whose rows J updates (for a Cholesky pattern these are
    // J's etree ancestors; marking all of them also covers any other lower pattern)
    for (int64_t e = cp[f] + ns; e < cp[f + 1]; ++e) mark[sn_of[ri[e]]] = 1;
  }
}

// The two solves over the visited supernodes.  Forward, per supernode: its
// diagonal triangle on the contiguous rows f..l-1 of x, then the rows below
// accumulated column by column into a dense buffer (contiguous L values, no
// row indices) and scattered once.  Backward, per supernode: the solved
// values of the rows below gathered once, then per column (last first) the
// dot product of its contiguous L values with them and the triangle.
void run_one(const scf_apply_subdomain &s, const SubPlan &P, const double *lambda, double *q,
             std::vector<double> &x, std::vector<double> &buf) {
  const int32_t n = s.n;
  const int64_t *cp = s.L_colptr;
  const int32_t *ri = s.L_rowind;
  const double *Lv = s.L_val;
  x.assign(n, 0.0);
  buf.resize(std::max<int64_t>(P.max_below, 1));
  for (int32_t j = 0; j < s.m; ++j) {
    const double pj = lambda[s.lambda_map[j]];
    for (int32_t e = s.Bt_colptr[j]; e < s.Bt_colptr[j + 1]; ++e) x[s.Bt_rowind[e]] += s.Bt_sign[e] * pj;
  }
  for (int32_t J : P.visit) {
    const int32_t f = P.sn[J], ns = P.sn[J + 1] - f;
    const int64_t nr = cp[f + 1] - cp[f], nb = nr - ns;
    double *xs = x.data() + f;
    double *tmp = buf.data();
    std::fill(tmp, tmp + nb, 0.0);
    for (int32_t t = 0; t < ns; ++t) {
      const double *Lc = Lv + cp[f + t];        // rows f+t .. of the panel
      const double yt = xs[t] / Lc[0];
      xs[t] = yt;
      for (int32_t a = t + 1; a < ns; ++a) xs[a] -= Lc[a - t] * yt;
      const double *Lb = Lc + (ns - t);
      for (int64_t k = 0; k < nb; ++k) tmp[k] -= Lb[k] * yt;
    }
    const int32_t *Rb = ri + cp[f] + ns;
    for (int64_t k = 0; k < nb; ++k) x[Rb[k]] += tmp[k];
  }
  for (size_t v = P.visit.size(); v-- > 0;) {
    const int32_t J = P.visit[v];
    const int32_t f = P.sn[J], ns = P.sn[J + 1] - f;
    const int64_t nr = cp[f + 1] - cp[f], nb = nr - ns;
    double *xs = x.data() + f;
    double *g = buf.data();
    const int32_t *Rb = ri + cp[f] + ns;
    for (int64_t k = 0; k < nb; ++k) g[k] = x[Rb[k]];
    for (int32_t t = ns - 1; t >= 0; --t) {
      const double *Lc = Lv + cp[f + t];
      const double *Lb = Lc + (ns - t);
      double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
      int64_t k = 0;
      for (; k + 4 <= nb; k += 4) {
        a0 += Lb[k] * g[k];
        a1 += Lb[k + 1] * g[k + 1];
        a2 += Lb[k + 2] * g[k + 2];
        a3 += Lb[k + 3] * g[k + 3];
      }
      for (; k < nb; ++k) a0 += Lb[k] * g[k];
      double acc = xs[t] - ((a0 + a1) + (a2 + a3));
      for (int32_t a = t + 1; a < ns; ++a) acc -= Lc[a - t] * xs[a];
      xs[t] = acc / Lc[0];
    }
  }
  for (int32_t j = 0; j < s.m; ++j) {
    double v = 0.0;
    for (int32_t e = s.Bt_colptr[j]; e < s.Bt_colptr[j + 1]; ++e) v += s.Bt_sign[e] * x[s.Bt_rowind[e]];
    q[s.lambda_map[j]] += v;
  }
}

// Every index the solves form stays in range: L is CSC lower with the
// diagonal first and rows strictly ascending below it, B^T's column pointers
// start at 0 and do not decrease, its rows and the multiplier map are in
// range.
bool check_one(const scf_apply_subdomain &s, int64_t n_dual) {
  if (s.n < 0 || s.m < 0 || (s.n > 0 && (!s.L_colptr || !s.L_rowind || !s.L_val))) return false;
  if (s.m > 0 && (!s.Bt_colptr || !s.Bt_rowind || !s.Bt_sign || !s.lambda_map)) return false;
  if (s.n > 0) {
    if (s.L_colptr[0] != 0) return false;
    for (int32_t c = 0; c < s.n; ++c) {
      const int64_t a = s.L_colptr[c], b = s.L_colptr[c + 1];
      if (b <= a || s.L_rowind[a] != c) return false;
      for (int64_t e = a + 1; e < b; ++e)
        if (s.L_rowind[e] <= s.L_rowind[e - 1] || s.L_rowind[e] >= s.n) return false;
    }
  }
  if (s.m > 0) {
    if (s.Bt_colptr[0] != 0) return false;
    for (int32_t j = 0; j < s.m; ++j)
      if (s.Bt_colptr[j + 1] < s.Bt_colptr[j]) return false;
  }
  for (int32_t j = 0; j < s.m; ++j)
    if (s.lambda_map[j] < 0 || s.lambda_map[j] >= n_dual) return false;
  for (int32_t j = 0; j < s.m; ++j)
    for (int32_t e = s.Bt_colptr[j]; e < s.Bt_colptr[j + 1]; ++e)
      if (s.Bt_rowind[e] < 0 || s.Bt_rowind[e] >= s.n) return false;
  return true;
}

int32_t thread_count(int32_t nthreads, int32_t nsub) {
  const int32_t T = nthreads > 0 ? nthreads : (int32_t)std::max(1u, std::thread::hardware_concurrency());
  return std::max(1, std::min(T, std::max(nsub, 1)));
}

// check_one for every subdomain, on the host threads.
int check_subs(int32_t nsub, const scf_apply_subdomain *subs, int64_t n_dual, int32_t nthreads) {
  if (nsub < 0 || n_dual < 0 || (nsub > 0 && !subs)) return SCF_ERR_INVALID_ARG;
  std::atomic<bool> ok{true};
  std::atomic<int32_t> next{0};
  auto work = [&]() {
    for (int32_t i; ok && (i = next.fetch_add(1)) < nsub;)
      if (!check_one(subs[i], n_dual)) ok = false;
  };
  try {
    const int32_t T = thread_count(nthreads, nsub);
    std::vector<std::thread> pool;
    for (int32_t t = 1; t < T; ++t) pool.emplace_back(work);
    work();
    for (auto &th : pool) th.join();
  } catch (const std::bad_alloc &) {
    return SCF_ERR_OOM;
  }
  return ok ? SCF_OK : SCF_ERR_INVALID_ARG;
}

// Threads over subdomains, each summing into its own dual vector; the vectors
// are added in thread order, so the result does not depend on timing.
// Returns SCF_ERR_OOM (q untouched) if a host allocation fails.
template <class F>
int over_threads(int32_t nsub, int64_t n_dual, double *q, int32_t nthreads, F &&body) {
  try {
    const int32_t T = thread_count(nthreads, nsub);
    std::vector<std::vector<double>> qs(T, std::vector<double>(n_dual, 0.0));
    std::atomic<bool> oom{false};
    std::vector<std::thread> pool;
    for (int32_t t = 0; t < T; ++t)
      pool.emplace_back([&, t]() {
        try {
          body(t, T, qs[t].data());
        } catch (const std::bad_alloc &) {
          oom = true;
        }
      });
    for (auto &th : pool) th.join();
    if (oom) return SCF_ERR_OOM;
    std::memset(q, 0, sizeof(double) * (size_t)n_dual);
    for (int32_t t = 0; t < T; ++t)
      for (int64_t k = 0; k < n_dual; ++k) q[k] += qs[t][k];
  } catch (const std::bad_alloc &) {
    return SCF_ERR_OOM;
  }
  return SCF_OK;
}

}  // namespace

struct scf_implicit {
  int64_t n_dual = 0;
  std::vector<scf_apply_subdomain> subs;
  std::vector<SubPlan> plans;
};

extern "C" {

int scf_implicit_apply(int32_t nsub, const scf_apply_subdomain *subs, int64_t n_dual, const double *lambda,
                       double *q, int32_t nthreads) {
  if (n_dual > 0 && (!lambda || !q)) return SCF_ERR_INVALID_ARG;
  const int rc = check_subs(nsub, subs, n_dual, nthreads);
  if (rc != SCF_OK) return rc;
  return over_threads(nsub, n_dual, q, nthreads, [&](int32_t t, int32_t T, double *qt) {
    std::vector<double> x;
    for (int32_t i = t; i < nsub; i += T) apply_one(subs[i], lambda, qt, x);
  });
}

int scf_implicit_plan(int32_t nsub, const scf_apply_subdomain *subs, int64_t n_dual, scf_implicit **out) {
  if (!out) return SCF_ERR_INVALID_ARG;
  *out = nullptr;
  const int rc = check_subs(nsub, subs, n_dual, 0);
  if (rc != SCF_OK) return rc;
  scf_implicit *p = new (std::nothrow) scf_implicit();
  if (!p) return SCF_ERR_OOM;
  try {
    p->n_dual = n_dual;
    p->subs.assign(subs, subs + nsub);
    p->plans.resize(nsub);
    for (int32_t i = 0; i < nsub; ++i) plan_one(p->subs[i], p->plans[i]);
  } catch (const std::bad_alloc &) {
    delete p;
    return SCF_ERR_OOM;
  }
  *out = p;
  return SCF_OK;
}

int scf_implicit_run(const scf_implicit *p, const double *lambda, double *q, int32_t nthreads) {
  if (!p || (p->n_dual > 0 && (!lambda || !q))) return SCF_ERR_INVALID_ARG;
  const int32_t nsub = (int32_t)p->subs.size();
  return over_threads(nsub, p->n_dual, q, nthreads, [&](int32_t t, int32_t T, double *qt) {
    std::vector<double> x, buf;
    for (int32_t i = t; i < nsub; i += T) run_one(p->subs[i], p->plans[i], lambda, qt, x, buf);
  });
}

void scf_implicit_free(scf_implicit *p) { delete p; }

int scf_solve(int32_t n, const int64_t *L_colptr, const int32_t *L_rowind, const double *L_val, const double *b,
              double *x) {
  if (n < 0 || (n > 0 && (!L_colptr || !L_rowind || !L_val || !b || !x))) return SCF_ERR_INVALID_ARG;
  scf_apply_subdomain s;
  std::memset(&s, 0, sizeof s);
  s.n = n;
  s.L_colptr = L_colptr;
  s.L_rowind = L_rowind;
  s.L_val = L_val;
  if (!check_one(s, 0)) return SCF_ERR_INVALID_ARG;
  if (x != b) std::memcpy(x, b, sizeof(double) * (size_t)n);
  for (int32_t c = 0; c < n; ++c) {                       // L y = b, column oriented
    const int64_t a = L_colptr[c], e1 = L_colptr[c + 1];
    const double yc = x[c] / L_val[a];
    x[c] = yc;
    for (int64_t e = a + 1; e < e1; ++e) x[L_rowind[e]] -= L_val[e] * yc;
  }
  for (int32_t c = n - 1; c >= 0; --c) {                   // L^T x = y, row oriented over L's columns
    const int64_t a = L_colptr[c], e1 = L_colptr[c + 1];
    double acc = x[c];
    for (int64_t e = a + 1; e < e1; ++e) acc -= L_val[e] * x[L_rowind[e]];
    x[c] = acc / L_val[a];
  }
  return SCF_OK;
}

}  // extern "C"
