// Host sparse Cholesky that produces the library's input factor L (FP64).
//
// Paper Sec. 2.2: the two-stage factorisation K_reg = L L^T -- a symbolic
// stage that fixes the fill-reducing permutation and the nonzero pattern of L,
// then a numeric stage -- whose factor the Schur-complement assembly consumes.
// This file is the input producer only; it is not part of the GPU hot path.
//
// Steps:
//   1. K_reg from K (full symmetric CSC, original order) and the fixed dofs
//      (rows/columns of fixed dofs replaced by the identity), permuted by P;
//   2. elimination tree (Liu's algorithm with path compression);
//   3. optional etree postorder, composed into P (an equivalent ordering:
//      same fill, L relabelled);
//   4. column patterns of L: pattern(j) = struct(A(j:,j)) united with the
//      patterns of j's etree children (minus the child itself);
//   5. numeric left-looking column Cholesky with per-row linked lists of the
//      columns that update each row.  Each column's updates are accumulated in
//      double-double (exact products by fma, error-free sums), because the
//      last pivots of a floating subdomain fixed at few dofs are small
//      differences of large sums (the near-kernel mode); plain sequential FP64
//      accumulation loses about log10(kappa) digits there.
// Built with floating-point contraction off, so x86 and Arm produce the same
// factor bit for bit.
// The output L is CSC lower, rows ascending, diagonal first in every column.

#include "sc_factor.h"

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

struct scf_factor {
  int32_t n = 0;
  std::vector<int64_t> colptr;
  std::vector<int32_t> rowind;
  std::vector<double> val;
  std::vector<int32_t> perm;  // new -> old
};

namespace {

// Lower-triangular pattern+values of A = P K_reg P^T in CSC (rows >= col).
void permuted_lower(int32_t n, const int64_t *cp, const int32_t *ri, const double *v,
                    const std::vector<char> &is_fixed, const std::vector<int32_t> &perm,
                    std::vector<int64_t> &acp, std::vector<int32_t> &ari, std::vector<double> &av) {
  std::vector<int32_t> inv(n);
  for (int32_t i = 0; i < n; ++i) inv[perm[i]] = i;
  std::vector<int64_t> cnt(n + 1, 0);
  for (int32_t oc = 0; oc < n; ++oc) {
    int32_t nc = inv[oc];
    if (is_fixed[oc]) { cnt[nc + 1]++; continue; }
    for (int64_t e = cp[oc]; e < cp[oc + 1]; ++e) {
      int32_t orow = ri[e];
      if (is_fixed[orow]) continue;
      int32_t nr = inv[orow];
      if (nr >= nc) cnt[nc + 1]++;
    }
  }
  acp.assign(n + 1, 0);
  for (int32_t c = 0; c < n; ++c) acp[c + 1] = acp[c] + cnt[c + 1];
  ari.assign(acp[n], 0);
  av.assign(acp[n], 0.0);
  std::vector<int64_t> pos(acp.begin(), acp.end() - 1);
  for (int32_t oc = 0; oc < n; ++oc) {
    int32_t nc = inv[oc];
    if (is_fixed[oc]) { ari[pos[nc]] = nc; av[pos[nc]] = 1.0; pos[nc]++; continue; }
    for (int64_t e = cp[oc]; e < cp[oc + 1]; ++e) {
      int32_t orow = ri[e];
      if (is_fixed[orow]) continue;
      int32_t nr = inv[orow];
      if (nr >= nc) { ari[pos[nc]] = nr; av[pos[nc]] = v[e]; pos[nc]++; }
    }
  }
  // sort rows within each column
  std::vector<std::pair<int32_t, double>> tmp;
  for (int32_t c = 0; c < n; ++c) {
    tmp.clear();
    for (int64_t e = acp[c]; e < acp[c + 1]; ++e) tmp.emplace_back(ari[e], av[e]);
    std::sort(tmp.begin(), tmp.end(), [](auto &a, auto &b) { return a.first < b.first; });
    // merge duplicates
    int64_t w = acp[c];
    for (size_t k = 0; k < tmp.size(); ++k) {
      if (w > acp[c] && ari[w - 1] == tmp[k].first) { av[w - 1] += tmp[k].second; continue; }
      ari[w] = tmp[k].first; av[w] = tmp[k].second; ++w;
    }
    for (int64_t e = w; e < acp[c + 1]; ++e) { ari[e] = -1; }
  }
  // compact (duplicates removed)
  std::vector<int64_t> ncp(n + 1, 0);
  int64_t w = 0;
  for (int32_t c = 0; c < n; ++c) {
    for (int64_t e = acp[c]; e < acp[c + 1]; ++e)
      if (ari[e] >= 0) { ari[w] = ari[e]; av[w] = av[e]; ++w; }
    ncp[c + 1] = w;
  }
  ari.resize(w); av.resize(w); acp.swap(ncp);
}

// Elimination tree from the lower pattern (row r > c in column c means
// A(c, r) != 0 in the upper triangle, i.e. entry of "column r, row c").
void etree_from_lower(int32_t n, const std::vector<int64_t> &acp, const std::vector<int32_t> &ari,
                      std::vector<int32_t> &parent) {
  // transpose to get, per column k, the rows i < k with A(i,k) != 0
  std::vector<int64_t> ucp(n + 1, 0);
  for (int32_t c = 0; c < n; ++c)
    for (int64_t e = acp[c]; e < acp[c + 1]; ++e) if (ari[e] > c) ucp[ari[e] + 1]++;
  for (int32_t k = 0; k < n; ++k) ucp[k + 1] += ucp[k];
  std::vector<int32_t> uri(ucp[n]);
  std::vector<int64_t> pos(ucp.begin(), ucp.end() - 1);
  for (int32_t c = 0; c < n; ++c)
    for (int64_t e = acp[c]; e < acp[c + 1]; ++e) if (ari[e] > c) uri[pos[ari[e]]++] = c;
  parent.assign(n, -1);
  std::vector<int32_t> anc(n, -1);
  for (int32_t k = 0; k < n; ++k) {
    for (int64_t e = ucp[k]; e < ucp[k + 1]; ++e) {
      int32_t i = uri[e];
      while (i != -1 && i < k) {
        int32_t nxt = anc[i];
        anc[i] = k;
        if (nxt == -1) parent[i] = k;
        i = nxt;
      }
    }
  }
}

void postorder(int32_t n, const std::vector<int32_t> &parent, std::vector<int32_t> &post) {
  std::vector<int32_t> head(n, -1), next(n, -1);
  for (int32_t j = n - 1; j >= 0; --j) {          // children in increasing order
    if (parent[j] >= 0) { next[j] = head[parent[j]]; head[parent[j]] = j; }
  }
  post.clear();
  std::vector<int32_t> stack;
  for (int32_t r = 0; r < n; ++r) {
    if (parent[r] != -1) continue;
    stack.push_back(r);
    while (!stack.empty()) {
      int32_t p = stack.back();
      int32_t c = head[p];
      if (c == -1) { stack.pop_back(); post.push_back(p); }
      else { head[p] = next[c]; stack.push_back(c); }
    }
  }
}

}  // namespace

extern "C" {

int scf_factorize(int32_t n, const int64_t *K_colptr, const int32_t *K_rowind, const double *K_val,
                  int32_t nfixed, const int32_t *fixed, const int32_t *perm_in, int32_t do_postorder,
                  scf_factor **out) {
  if (!out || n < 0 || (n > 0 && (!K_colptr || !K_rowind || !K_val))) return SCF_ERR_INVALID_ARG;
  *out = nullptr;
  scf_factor *F = new (std::nothrow) scf_factor();
  if (!F) return SCF_ERR_OOM;
  F->n = n;
  std::vector<char> is_fixed(n, 0);
  for (int32_t k = 0; k < nfixed; ++k) {
    if (fixed[k] < 0 || fixed[k] >= n) { delete F; return SCF_ERR_INVALID_ARG; }
    is_fixed[fixed[k]] = 1;
  }
  std::vector<int32_t> perm(n);
  if (perm_in) {
    std::vector<char> seen(n, 0);
    for (int32_t i = 0; i < n; ++i) {
      if (perm_in[i] < 0 || perm_in[i] >= n || seen[perm_in[i]]) { delete F; return SCF_ERR_INVALID_ARG; }
      seen[perm_in[i]] = 1; perm[i] = perm_in[i];
    }
  } else {
    for (int32_t i = 0; i < n; ++i) perm[i] = i;
  }
  std::vector<int64_t> acp; std::vector<int32_t> ari; std::vector<double> av;
  permuted_lower(n, K_colptr, K_rowind, K_val, is_fixed, perm, acp, ari, av);
  std::vector<int32_t> parent;
  etree_from_lower(n, acp, ari, parent);
  if (do_postorder) {
    std::vector<int32_t> post;
    postorder(n, parent, post);
    std::vector<int32_t> p2(n);
    for (int32_t i = 0; i < n; ++i) p2[i] = perm[post[i]];
    perm.swap(p2);
    permuted_lower(n, K_colptr, K_rowind, K_val, is_fixed, perm, acp, ari, av);
    etree_from_lower(n, acp, ari, parent);
  }
  F->perm = perm;

  // symbolic: column patterns via children
  std::vector<std::vector<int32_t>> children(n);
  for (int32_t j = 0; j < n; ++j) if (parent[j] >= 0) children[parent[j]].push_back(j);
  std::vector<int32_t> mark(n, -1);
  std::vector<int64_t> cp(n + 1, 0);
  std::vector<int32_t> ri;
  ri.reserve(acp[n] * 4);
  std::vector<int32_t> buf;
  for (int32_t j = 0; j < n; ++j) {
    buf.clear();
    mark[j] = j; buf.push_back(j);
    for (int64_t e = acp[j]; e < acp[j + 1]; ++e) {
      int32_t r = ari[e];
      if (mark[r] != j) { mark[r] = j; buf.push_back(r); }
    }
    for (int32_t c : children[j]) {
      for (int64_t e = cp[c] + 1; e < cp[c + 1]; ++e) {     // skip child's diagonal
        int32_t r = ri[e];
        if (r > j && mark[r] != j) { mark[r] = j; buf.push_back(r); }
      }
    }
    std::sort(buf.begin() + 1, buf.end());
    ri.insert(ri.end(), buf.begin(), buf.end());
    cp[j + 1] = (int64_t)ri.size();
  }
  // numeric: left-looking with row lists
  std::vector<double> L(ri.size(), 0.0);
  std::vector<double> x(n, 0.0), xl(n, 0.0);   // double-double work column
  std::vector<int32_t> head(n, -1), link(n, -1);
  std::vector<int64_t> nextpos(n, 0);
  for (int32_t j = 0; j < n; ++j) {
    for (int64_t e = acp[j]; e < acp[j + 1]; ++e) x[ari[e]] = av[e];
    int32_t k = head[j];
    while (k != -1) {
      int32_t knext = link[k];
      int64_t p = nextpos[k];            // position of row j in column k
      const double ljk = L[p];
      for (int64_t e = p; e < cp[k + 1]; ++e) {
        const int32_t i = ri[e];
        const double a = L[e] * ljk;
        const double ae = std::fma(L[e], ljk, -a);   // a + ae == L[e] * ljk exactly
        const double s = x[i] - a;                     // two-sum of x[i] and -a
        const double bb = s - x[i];
        const double err = (x[i] - (s - bb)) + (-a - bb);
        x[i] = s;
        xl[i] += err - ae;
      }
      // re-link k under its next row
      if (p + 1 < cp[k + 1]) {
        nextpos[k] = p + 1;
        int32_t r = ri[p + 1];
        link[k] = head[r]; head[r] = k;
      }
      k = knext;
    }
    head[j] = -1;
    double d = x[j] + xl[j];
    if (!(d > 0.0) || !std::isfinite(d)) {
      delete F;
      return SCF_ERR_NOT_SPD;
    }
    double ljj = std::sqrt(d);
    L[cp[j]] = ljj;
    x[j] = 0.0;
    xl[j] = 0.0;
    for (int64_t e = cp[j] + 1; e < cp[j + 1]; ++e) {
      const int32_t i = ri[e];
      L[e] = (x[i] + xl[i]) / ljj;
      x[i] = 0.0;
      xl[i] = 0.0;
    }
    if (cp[j] + 1 < cp[j + 1]) {
      nextpos[j] = cp[j] + 1;
      int32_t r = ri[cp[j] + 1];
      link[j] = head[r]; head[r] = j;
    }
  }
  F->colptr.swap(cp);
  F->rowind.swap(ri);
  F->val.swap(L);
  *out = F;
  return SCF_OK;
}

int64_t scf_nnz(const scf_factor *F) { return F ? (int64_t)F->rowind.size() : -1; }

int scf_export(const scf_factor *F, int64_t *colptr, int32_t *rowind, double *val, int32_t *perm) {
  if (!F) return SCF_ERR_INVALID_ARG;
  if (colptr) std::memcpy(colptr, F->colptr.data(), sizeof(int64_t) * (F->n + 1));
  if (rowind) std::memcpy(rowind, F->rowind.data(), sizeof(int32_t) * F->rowind.size());
  if (val) std::memcpy(val, F->val.data(), sizeof(double) * F->val.size());
  if (perm) std::memcpy(perm, F->perm.data(), sizeof(int32_t) * F->n);
  return SCF_OK;
}

void scf_free(scf_factor *F) { delete F; }

}  // extern "C"
