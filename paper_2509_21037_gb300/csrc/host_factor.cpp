// Host sparse Cholesky that produces the library's input factor L (FP64).
//
// Paper Sec. 2.2: the two-stage factorisation K_reg = L L^T -- a symbolic
// stage that fixes the fill-reducing permutation and the nonzero pattern of L,
// then a numeric stage -- whose factor the Schur-complement assembly consumes.
// This file is the input producer only; it is not part of the GPU hot path.
//
// Symbolic stage (scf_analyze):
//   1. the lower pattern of A = P K_reg P^T (K_reg: K with the rows and
//      columns of the fixed dofs replaced by the identity) and the map from
//      each stored entry of K to its place in A;
//   2. elimination tree (Liu's algorithm with path compression);
//   3. optional etree postorder, composed into P (an equivalent ordering:
//      same fill, L relabelled);
//   4. column patterns of L: pattern(j) = struct(A(j:,j)) united with the
//      patterns of j's etree children (minus the child itself);
//   5. supernodes: maximal runs of columns f..l-1 in which column j+1 is
//      column j's etree parent and has column j's pattern minus j itself.
// Numeric stage (scf_numeric, any number of times per analysis): A's values
// through the entry map, then supernodal left-looking Cholesky (dense
// panels, updated by the finished supernodes through per-supernode linked
// lists).  Every update is accumulated in double-double (exact products by
// fma, error-free sums), because the last pivots of a floating subdomain
// fixed at few dofs are small differences of large sums (the near-kernel
// mode); plain sequential FP64 accumulation loses about log10(kappa) digits
// there.  Each entry of L is the correctly rounded result of its column step
// given the finished entries it depends on (up to the rare double-double sum
// that is not correctly rounded itself).
// Built with floating-point contraction off, so x86 and Arm produce the same
// factor bit for bit.
// The output L is CSC lower, rows ascending, diagonal first in every column.

#include "sc_factor.h"

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <utility>
#include <vector>

struct scf_factor {
  int32_t n = 0;
  int64_t nnzK = 0;               // stored entries of K the analysis was made for
  std::vector<int64_t> colptr;    // pattern of L
  std::vector<int32_t> rowind;
  std::vector<double> val;        // values of L (zero after scf_analyze alone)
  std::vector<int32_t> perm;      // new -> old
  // symbolic data of the numeric stage
  std::vector<int64_t> acp;       // lower pattern of A = P K_reg P^T, CSC
  std::vector<int32_t> ari;
  std::vector<int64_t> kmap;      // K entry -> position in A's values, -1 if dropped
  std::vector<int64_t> ident;     // positions of the fixed dofs' unit diagonals
  std::vector<int32_t> sn;        // supernode starts, sn.back() == n
  std::vector<int32_t> sn_of;     // column -> supernode
  size_t max_panel = 0, max_rows = 0, max_width = 0;
};

namespace {

// Lower pattern of A = P K_reg P^T in CSC (rows >= column, ascending,
// duplicates merged) and the map from K's stored entries into it.  Entries of
// fixed rows or columns, and of the upper triangle of A, map to -1; a fixed
// dof gets a unit diagonal (listed in ident).
void lower_map(int32_t n, const int64_t *cp, const int32_t *ri, const std::vector<char> &is_fixed,
               const std::vector<int32_t> &perm, std::vector<int64_t> &acp, std::vector<int32_t> &ari,
               std::vector<int64_t> &kmap, std::vector<int64_t> &ident) {
  std::vector<int32_t> inv(n);
  for (int32_t i = 0; i < n; ++i) inv[perm[i]] = i;
  std::vector<int64_t> cnt(n + 1, 0);
  for (int32_t oc = 0; oc < n; ++oc) {
    const int32_t nc = inv[oc];
    if (is_fixed[oc]) { cnt[nc + 1]++; continue; }
    for (int64_t e = cp[oc]; e < cp[oc + 1]; ++e)
      if (!is_fixed[ri[e]] && inv[ri[e]] >= nc) cnt[nc + 1]++;
  }
  for (int32_t c = 0; c < n; ++c) cnt[c + 1] += cnt[c];
  // (row, K entry) per new column; the unit diagonal of a fixed dof has entry -1
  std::vector<std::pair<int32_t, int64_t>> ent(cnt[n]);
  std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
  for (int32_t oc = 0; oc < n; ++oc) {
    const int32_t nc = inv[oc];
    if (is_fixed[oc]) { ent[fill[nc]++] = {nc, -1}; continue; }
    for (int64_t e = cp[oc]; e < cp[oc + 1]; ++e) {
      const int32_t nr = inv[ri[e]];
      if (!is_fixed[ri[e]] && nr >= nc) ent[fill[nc]++] = {nr, e};
    }
  }
  kmap.assign(n > 0 ? cp[n] : 0, -1);
  ident.clear();
  acp.assign(n + 1, 0);
  ari.clear();
  ari.reserve(ent.size());
  for (int32_t c = 0; c < n; ++c) {
    std::sort(ent.begin() + cnt[c], ent.begin() + cnt[c + 1]);
    for (int64_t k = cnt[c]; k < cnt[c + 1]; ++k) {
      if (ari.size() == (size_t)acp[c] || ari.back() != ent[k].first) ari.push_back(ent[k].first);
      const int64_t at = (int64_t)ari.size() - 1;
      if (ent[k].second < 0) ident.push_back(at);
      else kmap[ent[k].second] = at;
    }
    acp[c + 1] = (int64_t)ari.size();
  }
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

// w + wl += sum_s v_s * b_s over len entries, each product exact (fma gives
// its rounding error) and added with an error-free two-sum; the errors go to
// wl.  Four columns per pass, so that w and wl are loaded and stored once for
// four products; the accumulation order is that of four single passes.
// Init: w and wl start from zero instead of being read (the same numbers:
// 0 + p is p exactly and its two-sum error is 0).
template <bool Init>
void dd_axpy4(double *__restrict w, double *__restrict wl, const double *__restrict v0,
              const double *__restrict v1, const double *__restrict v2, const double *__restrict v3,
              double b0, double b1, double b2, double b3, int64_t len) {
  for (int64_t a = 0; a < len; ++a) {
    double h = Init ? 0.0 : w[a], l = Init ? 0.0 : wl[a];
    const double x[4] = {v0[a], v1[a], v2[a], v3[a]};
    const double b[4] = {b0, b1, b2, b3};
    for (int u = 0; u < 4; ++u) {
      const double p = x[u] * b[u];
      const double pe = std::fma(x[u], b[u], -p);
      const double s = h + p;
      const double bb = s - h;
      l += ((h - (s - bb)) + (p - bb)) + pe;
      h = s;
    }
    w[a] = h;
    wl[a] = l;
  }
}

template <bool Init>
void dd_axpy1(double *__restrict w, double *__restrict wl, const double *__restrict v, double b, int64_t len) {
  for (int64_t a = 0; a < len; ++a) {
    const double h = Init ? 0.0 : w[a];
    const double p = v[a] * b;
    const double pe = std::fma(v[a], b, -p);
    const double s = h + p;
    const double bb = s - h;
    wl[a] = (Init ? 0.0 : wl[a]) + (((h - (s - bb)) + (p - bb)) + pe);
    w[a] = s;
  }
}

// w + wl += sign * sum_{s < ns} V[s] * V[s][off], V[s] = cols[s] (rows off..off+len);
// with init (ns >= 1) w + wl is the sum alone, its previous contents unread.
void dd_update(double *w, double *wl, const double *const *cols, int32_t ns, int64_t off, int64_t len, double sign,
               bool init = false) {
  int32_t s = 0;
  for (; s + 4 <= ns; s += 4) {
    const double *const v[4] = {cols[s] + off, cols[s + 1] + off, cols[s + 2] + off, cols[s + 3] + off};
    const double b[4] = {sign * cols[s][off], sign * cols[s + 1][off], sign * cols[s + 2][off], sign * cols[s + 3][off]};
    if (init && s == 0) dd_axpy4<true>(w, wl, v[0], v[1], v[2], v[3], b[0], b[1], b[2], b[3], len);
    else dd_axpy4<false>(w, wl, v[0], v[1], v[2], v[3], b[0], b[1], b[2], b[3], len);
  }
  for (; s < ns; ++s) {
    if (init && s == 0) dd_axpy1<true>(w, wl, cols[s] + off, sign * cols[s][off], len);
    else dd_axpy1<false>(w, wl, cols[s] + off, sign * cols[s][off], len);
  }
}

// Numeric stage, supernodal left-looking, into L (nnz values, CSC layout of
// f's pattern).  Supernode J = columns f..l-1 has nr shared rows R (the first
// ns = l-f of them f..l-1), so its columns form a dense nr x ns panel, held
// here in double-double (Ph + Pl):
//   1. the panel takes A's columns f..l-1;
//   2. every finished supernode K with rows in [f, l) (found through per-
//      supernode lists keyed by K's next row) contributes
//      -L_K(rows >= f) L_K(rows in [f, l))^T: accumulated per target column
//      in a dense double-double vector and then subtracted into the panel
//      through the row map R -> panel position;
//   3. the panel is factored column by column, each column first updated by
//      the finished columns to its left (same double-double arithmetic) and
//      then scaled by its pivot.
// Returns false on a non-positive or non-finite pivot.
bool numeric_supernodal(const scf_factor &F, const std::vector<double> &av, double *L) {
  const int32_t n = F.n, nsn = (int32_t)F.sn.size() - 1;
  const std::vector<int64_t> &cp = F.colptr, &acp = F.acp;
  const std::vector<int32_t> &ri = F.rowind, &ari = F.ari, &sn = F.sn, &sn_of = F.sn_of;
  std::vector<double> Ph(F.max_panel), Pl(F.max_panel), wh(F.max_rows), wl(F.max_rows);
  std::vector<const double *> cols(F.max_width);
  std::vector<int32_t> pos(n, 0), head(std::max(nsn, 0), -1), link(std::max(nsn, 0), -1);
  std::vector<int64_t> next(std::max(nsn, 0), 0);     // position in K's rows of the next row K updates
  for (int32_t J = 0; J < nsn; ++J) {
    const int32_t f = sn[J], l = sn[J + 1], ns = l - f;
    const int32_t *R = ri.data() + cp[f];
    const int64_t nr = cp[f + 1] - cp[f];
    for (int64_t a = 0; a < nr; ++a) pos[R[a]] = (int32_t)a;
    std::fill(Ph.begin(), Ph.begin() + nr * ns, 0.0);
    std::fill(Pl.begin(), Pl.begin() + nr * ns, 0.0);
    for (int32_t t = 0; t < ns; ++t)
      for (int64_t e = acp[f + t]; e < acp[f + t + 1]; ++e) Ph[t * nr + pos[ari[e]]] = av[e];
    // 2. updates from finished supernodes
    int32_t K = head[J];
    head[J] = -1;
    while (K != -1) {
      const int32_t knext = link[K];
      const int32_t fk = sn[K], nsk = sn[K + 1] - fk;
      const int32_t *RK = ri.data() + cp[fk];
      const int64_t nrk = cp[fk + 1] - cp[fk];
      const int64_t p = next[K];
      int64_t p2 = p;
      while (p2 < nrk && RK[p2] < l) ++p2;
      for (int32_t s = 0; s < nsk; ++s) cols[s] = L + cp[fk + s] + (p - s);   // rows RK[p..nrk)
      const int64_t len = nrk - p;
      for (int64_t b = 0; b < p2 - p; ++b) {
        dd_update(wh.data() + b, wl.data() + b, cols.data(), nsk, b, len - b, 1.0, true);   // nsk >= 1
        double *ph = Ph.data() + (int64_t)(RK[p + b] - f) * nr, *pl = Pl.data() + (int64_t)(RK[p + b] - f) * nr;
        for (int64_t a = b; a < len; ++a) {
          const int32_t i = pos[RK[p + a]];
          const double h = ph[i], q = -wh[a];
          const double s = h + q;
          const double bb = s - h;
          pl[i] += ((h - (s - bb)) + (q - bb)) - wl[a];
          ph[i] = s;
        }
      }
      if (p2 < nrk) {
        next[K] = p2;
        const int32_t S = sn_of[RK[p2]];
        link[K] = head[S];
        head[S] = K;
      }
      K = knext;
    }
    // 3. the panel's own columns
    for (int32_t t = 0; t < ns; ++t) {
      double *ph = Ph.data() + (int64_t)t * nr, *pl = Pl.data() + (int64_t)t * nr;
      for (int32_t s = 0; s < t; ++s) cols[s] = Ph.data() + (int64_t)s * nr;
      dd_update(ph + t, pl + t, cols.data(), t, t, nr - t, -1.0);
      const double d = ph[t] + pl[t];
      if (!(d > 0.0) || !std::isfinite(d)) return false;
      const double ljj = std::sqrt(d);
      ph[t] = ljj;
      for (int64_t a = t + 1; a < nr; ++a) ph[a] = (ph[a] + pl[a]) / ljj;
      double *out = L + cp[f + t];
      for (int64_t a = t; a < nr; ++a) out[a - t] = ph[a];
    }
    if (nr > ns) {
      next[J] = ns;
      const int32_t S = sn_of[R[ns]];
      link[J] = head[S];
      head[S] = J;
    }
  }
  return true;
}

// Symbolic stage into F (steps 1-5 of the header); F's vectors are filled here.
int analyze_into(scf_factor *F, int32_t n, const int64_t *K_colptr, const int32_t *K_rowind, int32_t nfixed,
                 const int32_t *fixed, const int32_t *perm_in, int32_t do_postorder) {
  F->n = n;
  F->nnzK = n > 0 ? K_colptr[n] : 0;
  std::vector<char> is_fixed(n, 0);
  for (int32_t k = 0; k < nfixed; ++k) {
    if (fixed[k] < 0 || fixed[k] >= n) return SCF_ERR_INVALID_ARG;
    is_fixed[fixed[k]] = 1;
  }
  std::vector<int32_t> perm(n);
  if (perm_in) {
    std::vector<char> seen(n, 0);
    for (int32_t i = 0; i < n; ++i) {
      if (perm_in[i] < 0 || perm_in[i] >= n || seen[perm_in[i]]) return SCF_ERR_INVALID_ARG;
      seen[perm_in[i]] = 1; perm[i] = perm_in[i];
    }
  } else {
    for (int32_t i = 0; i < n; ++i) perm[i] = i;
  }
  lower_map(n, K_colptr, K_rowind, is_fixed, perm, F->acp, F->ari, F->kmap, F->ident);
  std::vector<int32_t> parent;
  etree_from_lower(n, F->acp, F->ari, parent);
  if (do_postorder) {
    std::vector<int32_t> post;
    postorder(n, parent, post);
    std::vector<int32_t> p2(n);
    for (int32_t i = 0; i < n; ++i) p2[i] = perm[post[i]];
    perm.swap(p2);
    lower_map(n, K_colptr, K_rowind, is_fixed, perm, F->acp, F->ari, F->kmap, F->ident);
    etree_from_lower(n, F->acp, F->ari, parent);
  }
  F->perm = perm;
  const std::vector<int64_t> &acp = F->acp;
  const std::vector<int32_t> &ari = F->ari;

  // column patterns via children
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
  // supernodes
  F->sn.assign(1, 0);
  for (int32_t j = 1; j < n; ++j)
    if (!(parent[j - 1] == j && cp[j] - cp[j - 1] == cp[j + 1] - cp[j] + 1)) F->sn.push_back(j);
  if (n > 0) F->sn.push_back(n);
  F->sn_of.assign(n, 0);
  for (int32_t J = 0; J + 1 < (int32_t)F->sn.size(); ++J) {
    const int32_t f = F->sn[J], l = F->sn[J + 1];
    for (int32_t j = f; j < l; ++j) F->sn_of[j] = J;
    const size_t nr = (size_t)(cp[f + 1] - cp[f]), ns = (size_t)(l - f);
    F->max_panel = std::max(F->max_panel, nr * ns);
    F->max_rows = std::max(F->max_rows, nr);
    F->max_width = std::max(F->max_width, ns);
  }
  F->colptr.swap(cp);
  F->rowind.swap(ri);
  F->val.assign(F->rowind.size(), 0.0);
  return SCF_OK;
}

}  // namespace

extern "C" {

int scf_analyze(int32_t n, const int64_t *K_colptr, const int32_t *K_rowind, int32_t nfixed, const int32_t *fixed,
                const int32_t *perm_in, int32_t do_postorder, scf_factor **out) {
  if (!out) return SCF_ERR_INVALID_ARG;
  *out = nullptr;
  if (n < 0 || nfixed < 0 || (nfixed > 0 && !fixed) || (n > 0 && (!K_colptr || !K_rowind)))
    return SCF_ERR_INVALID_ARG;
  if (n > 0) {
    if (K_colptr[0] != 0) return SCF_ERR_INVALID_ARG;
    for (int32_t c = 0; c < n; ++c)
      if (K_colptr[c + 1] < K_colptr[c]) return SCF_ERR_INVALID_ARG;
    for (int64_t e = 0; e < K_colptr[n]; ++e)
      if (K_rowind[e] < 0 || K_rowind[e] >= n) return SCF_ERR_INVALID_ARG;
  }
  scf_factor *F = new (std::nothrow) scf_factor();
  if (!F) return SCF_ERR_OOM;
  try {
    const int rc = analyze_into(F, n, K_colptr, K_rowind, nfixed, fixed, perm_in, do_postorder);
    if (rc != SCF_OK) {
      delete F;
      return rc;
    }
  } catch (const std::bad_alloc &) {
    delete F;
    return SCF_ERR_OOM;
  }
  *out = F;
  return SCF_OK;
}

int scf_numeric(const scf_factor *F, const double *K_val, double *L_val) {
  if (!F || (F->nnzK > 0 && !K_val) || (!F->rowind.empty() && !L_val)) return SCF_ERR_INVALID_ARG;
  std::vector<double> av;
  try {
    av.assign(F->ari.size(), 0.0);
    for (int64_t at : F->ident) av[at] = 1.0;
    for (int64_t e = 0; e < F->nnzK; ++e)
      if (F->kmap[e] >= 0) av[F->kmap[e]] += K_val[e];
    return numeric_supernodal(*F, av, L_val) ? SCF_OK : SCF_ERR_NOT_SPD;
  } catch (const std::bad_alloc &) {
    return SCF_ERR_OOM;
  }
}

int scf_factorize(int32_t n, const int64_t *K_colptr, const int32_t *K_rowind, const double *K_val,
                  int32_t nfixed, const int32_t *fixed, const int32_t *perm_in, int32_t do_postorder,
                  scf_factor **out) {
  if (!out) return SCF_ERR_INVALID_ARG;
  *out = nullptr;
  if (n > 0 && K_colptr && K_colptr[n] > 0 && !K_val) return SCF_ERR_INVALID_ARG;
  scf_factor *F = nullptr;
  int rc = scf_analyze(n, K_colptr, K_rowind, nfixed, fixed, perm_in, do_postorder, &F);
  if (rc != SCF_OK) return rc;
  rc = scf_numeric(F, K_val, F->val.data());
  if (rc != SCF_OK) {
    delete F;
    return rc;
  }
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
