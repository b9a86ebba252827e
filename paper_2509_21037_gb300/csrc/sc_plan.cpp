// Host planner: the symbolic ("initialization") stage of the Schur-complement
// assembly (paper Sec. 2.2 stages; Sec. 3 column permutation; Sec. 3.2 factor
// splitting with pruning; Sec. 3.3 SYRK input splitting).
//
// Per subdomain, from the patterns of L and B^T only:
//   1. validate the CSC patterns;
//   2. elimination tree of L (parent(c) = first off-diagonal row of column c)
//      and its postorder rank;
//   3. fundamental supernodes: column c+1 continues c's supernode when c+1 is
//      c's parent, c is its only child and pattern(c) \ {c} == pattern(c+1);
//      a supernode's pruned rows are the rows of its last column below the
//      diagonal block (paper Sec. 3.2, "pruning": only nonempty rows);
//   4. sort B^T's columns by their pivot (first nonzero, compared through the
//      postorder rank; for a postordered L this is the pivot row itself),
//      giving the stepped shape of paper Sec. 3;
//   5. the sorted column range [jlo, jhi) on which Y = L^{-1} P B^T is nonzero
//      on each supernode: column j is nonzero on the etree path from each of
//      its nonzero rows to the root (zeros above pivots are preserved, paper
//      Sec. 3.2), and a subtree's columns are contiguous after the sort;
//   6. the task lists: TRSM tasks over (subdomain, 32-column chunk) walking the
//      supernodes the chunk touches, SYRK tasks over (subdomain, chunk pair)
//      walking the supernodes active on both chunks;
//   7. flop and byte counters.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <limits>
#include <new>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "sc_internal.h"

using namespace sc;

namespace sc {

sc_status fail(sc_ctx *ctx, sc_status st, const std::string &msg) {
  if (ctx) ctx->err = msg;
  return st;
}

}  // namespace sc

namespace {

// cut for local rows [kb, kb + 32): one past the last sorted column that is
// nonzero somewhere in those rows (columns at or after it are zero there)
static int32_t block_cut(const SubPlan &P, int32_t s, int32_t kb) {
  int32_t c = P.maxq0[s];
  for (const auto &qe : P.inner[s])
    if (qe.second <= kb + 31 && qe.first > c) c = qe.first;
  return c + 1;
}

template <class T>
size_t add_section(std::vector<uint8_t> &blob, Section &s, const std::vector<T> &v) {
  size_t off = (blob.size() + 255) & ~size_t(255);
  blob.resize(off + v.size() * sizeof(T));
  if (!v.empty()) std::memcpy(blob.data() + off, v.data(), v.size() * sizeof(T));
  s.off = off;
  s.bytes = v.size() * sizeof(T);
  return off;
}

std::string sub_msg(int32_t i, const std::string &m) { return "subdomain " + std::to_string(i) + ": " + m; }

}  // namespace

// Steps 1-5 for one subdomain.  Returns empty string on success.
std::string sc::analyze(int32_t idx, const sc_subdomain_desc &d, SubPlan &P) {
  const int32_t n = d.n, m = d.m;
  if (n < 0 || m < 0) return sub_msg(idx, "negative n or m");
  if (n == 0 && m > 0) return sub_msg(idx, "m > 0 with n == 0");
  if (n > 0 && (!d.L_colptr || !d.L_rowind)) return sub_msg(idx, "L pattern pointers are NULL");
  if (m > 0 && (!d.Bt_colptr || !d.Bt_rowind || (!d.Bt_sign && !d.Bt_val))) return sub_msg(idx, "B^T pointers are NULL");
  const int64_t *cp = d.L_colptr;
  const int32_t *ri = d.L_rowind;
  if (n > 0 && cp[0] != 0) return sub_msg(idx, "L_colptr[0] != 0");
  for (int32_t c = 0; c < n; ++c) {
    if (cp[c + 1] <= cp[c]) return sub_msg(idx, "L column " + std::to_string(c) + " is empty");
    if (ri[cp[c]] != c) return sub_msg(idx, "L column " + std::to_string(c) + " does not start with its diagonal");
    for (int64_t e = cp[c] + 1; e < cp[c + 1]; ++e) {
      if (ri[e] <= ri[e - 1] || ri[e] >= n)
        return sub_msg(idx, "L column " + std::to_string(c) + " rows not strictly ascending / in range");
    }
  }
  if (m > 0) {
    if (d.Bt_colptr[0] != 0) return sub_msg(idx, "Bt_colptr[0] != 0");
    for (int32_t j = 0; j < m; ++j) {
      if (d.Bt_colptr[j + 1] < d.Bt_colptr[j]) return sub_msg(idx, "Bt_colptr not monotone");
      for (int32_t e = d.Bt_colptr[j]; e < d.Bt_colptr[j + 1]; ++e) {
        if (d.Bt_rowind[e] < 0 || d.Bt_rowind[e] >= n) return sub_msg(idx, "B^T row out of range");
        if (e > d.Bt_colptr[j] && d.Bt_rowind[e] <= d.Bt_rowind[e - 1])
          return sub_msg(idx, "B^T rows not strictly ascending in column " + std::to_string(j));
        if (d.Bt_val) {
          if (!std::isfinite(d.Bt_val[e])) return sub_msg(idx, "B^T value is not finite");
        } else if (d.Bt_sign[e] != 1 && d.Bt_sign[e] != -1) {
          return sub_msg(idx, "B^T entry is not +1/-1");
        }
      }
    }
  }
  // etree
  std::vector<int32_t> parent(n, -1), nchild(n, 0);
  for (int32_t c = 0; c < n; ++c) {
    if (cp[c + 1] - cp[c] > 1) {
      parent[c] = ri[cp[c] + 1];
      nchild[parent[c]]++;
    }
  }
  // postorder rank
  std::vector<int32_t> head(n, -1), next(n, -1), post_rank(n, 0);
  for (int32_t c = n - 1; c >= 0; --c)
    if (parent[c] >= 0) { next[c] = head[parent[c]]; head[parent[c]] = c; }
  {
    int32_t k = 0;
    std::vector<int32_t> stack;
    for (int32_t r = 0; r < n; ++r) {
      if (parent[r] != -1) continue;
      stack.push_back(r);
      while (!stack.empty()) {
        int32_t p = stack.back();
        int32_t ch = head[p];
        if (ch == -1) { stack.pop_back(); post_rank[p] = k++; }
        else { head[p] = next[ch]; stack.push_back(ch); }
      }
    }
  }
  // fundamental supernodes
  P.snode_of.assign(n, -1);
  for (int32_t c = 0; c < n; ++c) {
    bool cont = false;
    if (c > 0 && parent[c - 1] == c && nchild[c] == 1) {
      int64_t a = cp[c - 1], b = cp[c];
      int64_t la = cp[c] - cp[c - 1], lb = cp[c + 1] - cp[c];
      if (la == lb + 1) {
        cont = std::equal(ri + a + 1, ri + a + la, ri + b);
      }
    }
    if (!cont) {
      P.sn_c0.push_back(c);
      P.sn_ns.push_back(0);
      P.sn_rows_off.push_back(cp[c]);
    }
    int32_t s = (int32_t)P.sn_c0.size() - 1;
    P.snode_of[c] = s;
    P.sn_ns[s]++;
  }
  const int32_t nsn = (int32_t)P.sn_c0.size();
  P.sn_rs.resize(nsn);
  P.sparent.assign(nsn, -1);
  for (int32_t s = 0; s < nsn; ++s) {
    int32_t c1 = P.sn_c0[s] + P.sn_ns[s] - 1;
    P.sn_rs[s] = (int32_t)(cp[c1 + 1] - cp[c1] - 1);
    if (parent[c1] >= 0) P.sparent[s] = P.snode_of[parent[c1]];
  }
  // pivot sort (stable, by postorder rank of the first nonzero row)
  std::vector<int64_t> key(m);
  for (int32_t j = 0; j < m; ++j) {
    if (d.Bt_colptr[j + 1] > d.Bt_colptr[j]) {
      int32_t best = std::numeric_limits<int32_t>::max();
      for (int32_t e = d.Bt_colptr[j]; e < d.Bt_colptr[j + 1]; ++e) best = std::min(best, post_rank[d.Bt_rowind[e]]);
      key[j] = best;
    } else {
      key[j] = std::numeric_limits<int64_t>::max();   // empty column: last
    }
  }
  P.perm_cols.resize(m);
  std::iota(P.perm_cols.begin(), P.perm_cols.end(), 0);
  std::stable_sort(P.perm_cols.begin(), P.perm_cols.end(), [&](int32_t a, int32_t b) { return key[a] < key[b]; });
  // active ranges
  P.sn_jlo.assign(nsn, std::numeric_limits<int32_t>::max());
  P.sn_jhi.assign(nsn, -1);
  P.maxq0.assign(nsn, -1);
  P.inner.assign(nsn, {});
  std::vector<int32_t> mark(nsn, -1);
  for (int32_t q = 0; q < m; ++q) {
    int32_t j = P.perm_cols[q];
    for (int32_t e = d.Bt_colptr[j]; e < d.Bt_colptr[j + 1]; ++e) {
      const int32_t r = d.Bt_rowind[e];
      int32_t s = P.snode_of[r];
      bool first = true;
      while (s != -1 && mark[s] != q) {
        mark[s] = q;
        P.sn_jlo[s] = std::min(P.sn_jlo[s], q);
        P.sn_jhi[s] = std::max(P.sn_jhi[s], q + 1);
        const int32_t entry = first ? r - P.sn_c0[s] : 0;
        if (entry == 0) P.maxq0[s] = std::max(P.maxq0[s], q);
        else P.inner[s].emplace_back(q, entry);
        first = false;
        s = P.sparent[s];
      }
    }
  }
  for (int32_t s = 0; s < nsn; ++s)
    if (P.sn_jhi[s] < 0) { P.sn_jlo[s] = 0; P.sn_jhi[s] = 0; }
  return std::string();
}


sc_status build_plan(sc_ctx *ctx, int32_t nsub, const sc_subdomain_desc *d) {
  std::vector<SubPlan> P(nsub);
  // steps 1-5 of every subdomain on the host threads (each writes only its
  // own SubPlan); errors are reported for the lowest failing index
  std::vector<std::string> err(nsub);
  {
    std::atomic<int32_t> next{0};
    std::atomic<bool> oom{false};
    auto work = [&]() {
      for (int32_t i; (i = next.fetch_add(1)) < nsub;) {
        try {
          err[i] = analyze(i, d[i], P[i]);
        } catch (const std::bad_alloc &) {
          oom = true;
          return;
        }
      }
    };
    const int32_t T = std::max(1, std::min<int32_t>((int32_t)std::thread::hardware_concurrency(), nsub));
    std::vector<std::thread> pool;
    for (int32_t t = 1; t < T; ++t) pool.emplace_back(work);
    work();
    for (auto &th : pool) th.join();
    if (oom) throw std::bad_alloc();
  }
  for (int32_t i = 0; i < nsub; ++i) {
    if (!err[i].empty()) return fail(ctx, SC_ERR_INVALID_ARG, err[i]);
    if (d[i].m > 0 && !d[i].lambda_map) ctx->has_lambda = false;
    for (int32_t j = 0; j < d[i].m && d[i].lambda_map; ++j)
      if (d[i].lambda_map[j] < 0 || d[i].lambda_map[j] >= ctx->n_dual)
        return fail(ctx, SC_ERR_INVALID_ARG, sub_msg(i, "lambda_map entry out of [0, n_dual)"));
  }
  std::vector<SubDev> subs(nsub);
  std::vector<SnDev> sns;
  std::vector<int64_t> lcp, rmap;
  std::vector<TrsmTask> trsm;
  std::vector<int32_t> trsm_list;
  std::vector<SyrkTask> syrk;
  std::vector<int32_t> syrk_list;
  std::vector<Seed> seeds;
  std::vector<int32_t> perm, lam;
  std::vector<ApplyTask> apply;
  std::vector<int32_t> active_cols;
  std::vector<int32_t> cuts;
  std::vector<int32_t> sblk_v[kNumVariants], sblk_w[kNumVariants];
  std::vector<double> trsm_cost, syrk_cost;
  std::vector<int8_t> trsm_var, syrk_var;
  std::vector<int32_t> trsm_wave, syrk_wave;

  // temporary data of each subdomain and its packing into waves
  ctx->sub_wave.assign(nsub, 0);
  {
    const double Smax = ctx->n_slices;
    double cur = 0.0;
    int32_t w = 0;
    bool any = false;
    for (int32_t i = 0; i < nsub; ++i) {
      const SubPlan &S = P[i];
      double y = 0, yd = 0, ld = 0;
      for (size_t s = 0; s < S.sn_c0.size(); ++s) {
        const double ws = S.sn_jhi[s] - S.sn_jlo[s];
        if (ws <= 0) continue;
        y += S.sn_ns[s] * ws;
        yd += ws * ((S.sn_ns[s] + 31) / 32 * 32);
        for (int32_t kb = 0; kb < S.sn_ns[s]; kb += 32) ld += S.sn_ns[s] + S.sn_rs[s] - kb - std::min(32, S.sn_ns[s] - kb);
      }
      const double need = 8.0 * y + (ctx->sub_var[i] ? Smax * (2.0 * yd + 64.0 * ld) + 2.0 * ld : 0.0) + 4096.0;
      if (ctx->ws_limit > 0) {
        if (need > (double)ctx->ws_limit)
          return fail(ctx, SC_ERR_OOM, sub_msg(i, "needs " + std::to_string((int64_t)need) +
                                                      " workspace bytes, more than ws_limit"));
        if (any && cur + need > (double)ctx->ws_limit) { ++w; cur = 0.0; }
      }
      cur += need;
      any = true;
      ctx->sub_wave[i] = w;
    }
    ctx->waves.assign((size_t)w + 1, sc_ctx::WaveGroups());
  }

  ctx->F_offsets.assign(nsub + 1, 0);
  ctx->L_offsets.assign(nsub + 1, 0);
  ctx->n.resize(nsub);
  ctx->m.resize(nsub);
  int64_t y_total = 0, col_total = 0, lcp_total = 0, ld_rows_total = 0, yd_total = 0;
  int64_t y_max = 0, ld_max = 0, yd_max = 0, y_all = 0;  // per-wave offsets restart at 0
  sc_stats st{};
  int32_t max_m = 0;

  for (int32_t i = 0; i < nsub; ++i) {
    const sc_subdomain_desc &D = d[i];
    SubPlan &S = P[i];
    const int32_t n = D.n, m = D.m, nt = (m + kTile - 1) / kTile;
    if (i > 0 && ctx->sub_wave[i] != ctx->sub_wave[i - 1]) {   // a new wave reuses the workspace
      y_all += y_total;
      y_total = ld_rows_total = yd_total = 0;
    }
    ctx->n[i] = n;
    ctx->m[i] = m;
    max_m = std::max(max_m, m);
    const sc_stats st0 = st;                      // per-subdomain counters: differences at the end
    const int64_t y0 = y_all + y_total, nsn0 = (int64_t)sns.size();
    SubDev sd{};
    sd.F_off = ctx->F_offsets[i];
    sd.L_off = ctx->L_offsets[i];
    sd.n = n; sd.m = m; sd.nt = nt;
    sd.col_off = (int32_t)col_total;
    sd.lcp_off = (int32_t)lcp_total;
    subs[i] = sd;
    ctx->F_offsets[i + 1] = ctx->F_offsets[i] + (int64_t)nt * (nt + 1) / 2 * kTile * kTile;
    ctx->L_offsets[i + 1] = ctx->L_offsets[i] + (n > 0 ? D.L_colptr[n] : 0);
    for (int32_t c = 0; c < n; ++c) lcp.push_back(sd.L_off + D.L_colptr[c]);
    for (int32_t q = 0; q < m; ++q) {
      perm.push_back(S.perm_cols[q]);
      lam.push_back(D.lambda_map ? D.lambda_map[q] : 0);
    }
    // active supernodes -> global index, Y offsets
    const int32_t nsn = (int32_t)S.sn_c0.size();
    std::vector<int32_t> gidx(nsn, -1);
    std::vector<int64_t> yoff(nsn, 0);
    for (int32_t s = 0; s < nsn; ++s) {
      int32_t ws = S.sn_jhi[s] - S.sn_jlo[s];
      if (ws <= 0) continue;
      gidx[s] = (int32_t)sns.size();
      yoff[s] = y_total;
      y_total += (int64_t)S.sn_ns[s] * ws;
      SnDev sn{};
      sn.y_off = yoff[s];
      sn.sub = i;
      sn.c0 = S.sn_c0[s]; sn.ns = S.sn_ns[s]; sn.rs = S.sn_rs[s];
      sn.jlo = S.sn_jlo[s]; sn.jhi = S.sn_jhi[s];
      sn.lcp_off = (int32_t)(lcp_total + S.sn_c0[s]);
      const int var = ctx->sub_var[i];
      if (var) {
        sn.ld_off = ld_rows_total;
        for (int32_t kb = 0; kb < sn.ns; kb += 32)
          ld_rows_total += (sn.ns + sn.rs) - kb - std::min(32, sn.ns - kb);
        sn.yd_off = yd_total;
        yd_total += (int64_t)ws * ((sn.ns + 31) / 32 * 32);
      }
      sn.cut_off = (int32_t)cuts.size();
      for (int32_t kb = 0; kb < sn.ns; kb += 32) {
        cuts.push_back(std::max(sn.jlo, block_cut(S, s, kb)));
        if (var) {
          sblk_v[var].push_back((int32_t)sns.size());
          sblk_v[var].push_back(kb / 32);
          sblk_w[var].push_back(ctx->sub_wave[i]);
        }
      }
      sns.push_back(sn);
      y_max = std::max(y_max, y_total);
      ld_max = std::max(ld_max, ld_rows_total);
      yd_max = std::max(yd_max, yd_total);
      st.max_supernode = std::max<int64_t>(st.max_supernode, sn.ns);
      for (int32_t c = 0; c < sn.ns; ++c) active_cols.push_back(sn.lcp_off + c);
    }
    // pruned-row targets
    for (int32_t s = 0; s < nsn; ++s) {
      if (gidx[s] < 0) continue;
      SnDev &sn = sns[gidx[s]];
      sn.rmap_off = (int64_t)rmap.size();
      int32_t c1 = sn.c0 + sn.ns - 1;
      for (int32_t k = 0; k < sn.rs; ++k) {
        int32_t r = D.L_rowind[D.L_colptr[c1] + 1 + k];
        int32_t a = S.snode_of[r];
        if (gidx[a] < 0 || S.sn_jlo[a] > sn.jlo || S.sn_jhi[a] < sn.jhi)
          return fail(ctx, SC_ERR_INTERNAL, sub_msg(i, "ancestor range does not nest"));
        int32_t wa = S.sn_jhi[a] - S.sn_jlo[a];
        rmap.push_back(yoff[a] + (int64_t)(r - S.sn_c0[a]) * wa + (sn.jlo - S.sn_jlo[a]));
      }
    }
    // seeds, by sorted column
    std::vector<int32_t> seed_ptr(m + 1, 0);
    int32_t seed_base = (int32_t)seeds.size();
    for (int32_t q = 0; q < m; ++q) {
      int32_t j = S.perm_cols[q];
      seed_ptr[q] = (int32_t)seeds.size();
      for (int32_t e = D.Bt_colptr[j]; e < D.Bt_colptr[j + 1]; ++e) {
        int32_t r = D.Bt_rowind[e];
        int32_t s = S.snode_of[r];
        int32_t ws = S.sn_jhi[s] - S.sn_jlo[s];
        Seed sdd;
        sdd.y_off = yoff[s] + (int64_t)(r - S.sn_c0[s]) * ws + (q - S.sn_jlo[s]);
        sdd.value = D.Bt_val ? D.Bt_val[e] : (double)D.Bt_sign[e];
        seeds.push_back(sdd);
      }
    }
    seed_ptr[m] = (int32_t)seeds.size();
    (void)seed_base;
    // chunk lists
    const int32_t nchunk = nt;
    std::vector<std::vector<int32_t>> clist(nchunk);
    for (int32_t s = 0; s < nsn; ++s) {
      if (gidx[s] < 0) continue;
      for (int32_t q = S.sn_jlo[s] / kChunk; q <= (S.sn_jhi[s] - 1) / kChunk; ++q) clist[q].push_back(s);
    }
    for (int32_t q = 0; q < nchunk; ++q) {
      TrsmTask t{};
      t.sub = i;
      t.c_lo = q * kChunk;
      t.w = std::min(kChunk, m - t.c_lo);
      t.list_off = (int32_t)trsm_list.size();
      t.list_len = (int32_t)clist[q].size();
      t.seed_lo = seed_ptr[t.c_lo];
      t.seed_hi = seed_ptr[t.c_lo + t.w];
      double cost = 0, exec = 0;
      for (int32_t s : clist[q]) {
        trsm_list.push_back(gidx[s]);
        const SnDev &sn = sns[gidx[s]];
        int32_t a = std::max(S.sn_jlo[s], t.c_lo), b = std::min(S.sn_jhi[s], t.c_lo + t.w);
        const int32_t nrow = sn.ns + sn.rs;
        for (int32_t kb = 0; kb < sn.ns; kb += 32) {
          const int32_t wkb = std::min(b, cuts[sn.cut_off + kb / 32]) - a;
          if (wkb <= 0) continue;
          const double kw = std::min(32, sn.ns - kb);
          const double blk = kw * kw + 2.0 * kw * (nrow - kb - kw);
          cost += wkb * blk;
          exec += kChunk * blk;
        }
      }
      st.flops_trsm += cost;
      st.flops_trsm_exec += exec;
      trsm.push_back(t);
      trsm_cost.push_back(exec + 1e3 * t.list_len);
      trsm_var.push_back(ctx->sub_var[i]);
      trsm_wave.push_back(ctx->sub_wave[i]);
    }
    // 128x32 tiles for the tcgen05 SYRK: rows = chunks q1 .. q1 + 3 (q1 = 4 Q), columns = chunk q2;
    // supernodes = the union of the chunk pairs' common lists (lower triangle only)
    for (int32_t q1 = 0; (ctx->sub_var[i] & kVarTile) && q1 < nchunk; q1 += 4) {
      for (int32_t q2 = 0; q2 <= std::min(q1 + 3, nchunk - 1); ++q2) {
        SyrkTask t{};
        t.sub = i; t.q1 = q1; t.q2 = q2;
        t.list_off = (int32_t)syrk_list.size();
        std::vector<int32_t> uni;
        for (int32_t qa = std::max(q1, q2); qa <= std::min(q1 + 3, nchunk - 1); ++qa) {
          const auto &A = clist[qa], &B = clist[q2];
          size_t ia = 0, ib = 0;
          while (ia < A.size() && ib < B.size()) {
            if (A[ia] < B[ib]) ++ia;
            else if (B[ib] < A[ia]) ++ib;
            else { uni.push_back(A[ia]); ++ia; ++ib; }
          }
        }
        std::sort(uni.begin(), uni.end());
        uni.erase(std::unique(uni.begin(), uni.end()), uni.end());
        double exec = 0;
        const int32_t j1min = std::max(q1, q2) * kChunk;
        for (int32_t s : uni) {
          const SnDev &sn = sns[gidx[s]];
          syrk_list.push_back(gidx[s]);
          for (int32_t k0 = 0; k0 < sn.ns; k0 += 32)
            if (j1min < cuts[sn.cut_off + k0 / 32]) exec += 2.0 * 128 * kChunk * 32;
        }
        t.list_len = (int32_t)syrk_list.size() - t.list_off;
        st.flops_syrk_exec += exec;
        syrk.push_back(t);
        syrk_cost.push_back(exec + 1e3 * (t.list_len + 1));
        syrk_var.push_back(ctx->sub_var[i]);
        syrk_wave.push_back(ctx->sub_wave[i]);
      }
    }
    // chunk-pair lists (lower triangle of sorted chunks)
    for (int32_t q1 = 0; !(ctx->sub_var[i] & kVarTile) && q1 < nchunk; ++q1) {
      for (int32_t q2 = 0; q2 <= q1; ++q2) {
        SyrkTask t{};
        t.sub = i; t.q1 = q1; t.q2 = q2;
        t.list_off = (int32_t)syrk_list.size();
        const auto &A = clist[q1], &B = clist[q2];
        size_t ia = 0, ib = 0;
        double exec = 0;
        while (ia < A.size() && ib < B.size()) {
          if (A[ia] < B[ib]) ++ia;
          else if (B[ib] < A[ia]) ++ib;
          else {
            const SnDev &sn = sns[gidx[A[ia]]];
            syrk_list.push_back(gidx[A[ia]]);
            for (int32_t k0 = 0; k0 < sn.ns; k0 += 32)
              if (q1 * kChunk < cuts[sn.cut_off + k0 / 32]) exec += 2.0 * kChunk * kChunk * std::min(32, sn.ns - k0);
            ++ia; ++ib;
          }
        }
        t.list_len = (int32_t)syrk_list.size() - t.list_off;
        st.flops_syrk_exec += exec;
        syrk.push_back(t);
        syrk_cost.push_back(exec + 1e3 * (t.list_len + 1));
        syrk_var.push_back(ctx->sub_var[i]);
        syrk_wave.push_back(ctx->sub_wave[i]);
      }
    }
    for (int32_t s = 0; s < nsn; ++s) {
      if (gidx[s] < 0) continue;
      const SnDev &sn = sns[gidx[s]];
      for (int32_t k0 = 0; k0 < sn.ns; k0 += 32) {
        // lower triangle incl. diagonal of the nonzero columns of this row block, 2 flops per row
        const double wc = cuts[sn.cut_off + k0 / 32] - sn.jlo;
        st.flops_syrk += wc * (wc + 1.0) * std::min(32, sn.ns - k0);
      }
    }
    for (int32_t I = 0; I < nt; ++I) apply.push_back(ApplyTask{i, I});
    st.flops_dense += (double)n * n * m + (double)n * m * (m + 1.0);
    st.bytes_assembly += 12.0 * (n > 0 ? (double)D.L_colptr[n] : 0.0) + 8.0 * m * (m + 1.0) / 2.0;
    st.bytes_apply += 8.0 * m * (m + 1.0) / 2.0 + 16.0 * m;
    {
      SubFeat f{};
      f.n = n; f.m = m;
      f.nnzL = n > 0 ? (double)D.L_colptr[n] : 0.0;
      f.supernodes = (double)((int64_t)sns.size() - nsn0);
      for (int64_t k = nsn0; k < (int64_t)sns.size(); ++k) f.max_supernode = std::max(f.max_supernode, (double)sns[k].ns);
      f.flops_trsm = st.flops_trsm - st0.flops_trsm;
      f.flops_syrk = st.flops_syrk - st0.flops_syrk;
      f.flops_dense = st.flops_dense - st0.flops_dense;
      f.y_doubles = (double)(y_all + y_total - y0);
      ctx->sub_feat.push_back(f);
    }
    col_total += m;
    lcp_total += n;
  }
  // grouped by wave and variant (one launch per group), largest tasks first
  // inside a group: the block scheduler hands out CTAs roughly in index order
  auto order_by = [](const std::vector<double> &cost, const std::vector<int8_t> &var,
                     const std::vector<int32_t> &wave) {
    std::vector<int32_t> o(cost.size());
    std::iota(o.begin(), o.end(), 0);
    std::stable_sort(o.begin(), o.end(), [&](int32_t a, int32_t b) {
      if (wave[a] != wave[b]) return wave[a] < wave[b];
      return var[a] != var[b] ? var[a] < var[b] : cost[a] > cost[b];
    });
    return o;
  };
  auto groups = [&](const std::vector<int8_t> &var, const std::vector<int32_t> &wave, const std::vector<int32_t> &o,
                    int which) {
    for (size_t k = 0; k < o.size(); ++k) {
      const int v = var[o[k]];
      auto &g = which == 0 ? ctx->waves[wave[o[k]]].trsm[v] : ctx->waves[wave[o[k]]].syrk[v];
      if (g[1] == 0) g[0] = (int64_t)k;
      g[1]++;
    }
  };
  {
    auto o = order_by(trsm_cost, trsm_var, trsm_wave);
    // The TRSM of a batch is about one wave of resident CTAs, so what the launch
    // costs is its busiest SM.  With CTAs handed to the SMs in index order, a
    // largest-first list gives the low-numbered SMs the larger task of every
    // round; reversing every other round of kGridSMs tasks (a snake) pairs
    // larger with smaller ones.  Results do not depend on the order.
    for (size_t g0 = 0; g0 < o.size();) {
      size_t g1 = g0;
      while (g1 < o.size() && trsm_wave[o[g1]] == trsm_wave[o[g0]] && trsm_var[o[g1]] == trsm_var[o[g0]]) ++g1;
      for (size_t r0 = g0, rnd = 0; r0 < g1; r0 += kGridSMs, ++rnd)
        if (rnd & 1) std::reverse(o.begin() + r0, o.begin() + std::min(g1, r0 + (size_t)kGridSMs));
      g0 = g1;
    }
    groups(trsm_var, trsm_wave, o, 0);
    std::vector<TrsmTask> t2(trsm.size());
    for (size_t k = 0; k < o.size(); ++k) t2[k] = trsm[o[k]];
    trsm.swap(t2);
  }
  {
    auto o = order_by(syrk_cost, syrk_var, syrk_wave);
    groups(syrk_var, syrk_wave, o, 1);
    std::vector<SyrkTask> t2(syrk.size());
    for (size_t k = 0; k < o.size(); ++k) t2[k] = syrk[o[k]];
    syrk.swap(t2);
  }
  std::vector<int32_t> sblk;
  for (size_t w = 0; w < ctx->waves.size(); ++w) {
    for (int v = 0; v < kNumVariants; ++v) {
      auto &g = ctx->waves[w].sblk[v];
      g[0] = (int64_t)sblk.size() / 2;
      for (size_t k = 0; k < sblk_w[v].size(); ++k) {
        if (sblk_w[v][k] != (int32_t)w) continue;
        sblk.push_back(sblk_v[v][2 * k]);
        sblk.push_back(sblk_v[v][2 * k + 1]);
      }
      g[1] = (int64_t)sblk.size() / 2 - g[0];
    }
  }
  ctx->diag_index = lcp;
  ctx->blob.assign(kHeaderBytes, 0);
  add_section(ctx->blob, ctx->s_subs, subs);
  add_section(ctx->blob, ctx->s_sns, sns);
  add_section(ctx->blob, ctx->s_lcp, lcp);
  add_section(ctx->blob, ctx->s_rmap, rmap);
  add_section(ctx->blob, ctx->s_trsm, trsm);
  add_section(ctx->blob, ctx->s_trsm_list, trsm_list);
  add_section(ctx->blob, ctx->s_syrk, syrk);
  add_section(ctx->blob, ctx->s_syrk_list, syrk_list);
  add_section(ctx->blob, ctx->s_seeds, seeds);
  add_section(ctx->blob, ctx->s_perm, perm);
  add_section(ctx->blob, ctx->s_lambda, lam);
  add_section(ctx->blob, ctx->s_apply, apply);
  add_section(ctx->blob, ctx->s_active, active_cols);
  add_section(ctx->blob, ctx->s_cuts, cuts);
  add_section(ctx->blob, ctx->s_sblk, sblk);
  ctx->blob.resize((ctx->blob.size() + 255) & ~size_t(255));
  ctx->n_sns = (int64_t)sns.size();
  ctx->n_trsm = (int64_t)trsm.size();
  ctx->n_syrk = (int64_t)syrk.size();
  ctx->n_apply = (int64_t)apply.size();
  ctx->n_cols = lcp_total;
  ctx->n_active_cols = (int64_t)active_cols.size();
  ctx->n_sblk = (int64_t)sblk.size() / 2;
  {
    PlanHeader h{};
    h.magic = 0x4C504353u;  // "SCPL"
    h.version = 1;
    h.nsub = nsub;
    h.chunk = kChunk;
    h.n_sns = ctx->n_sns; h.n_trsm = ctx->n_trsm; h.n_syrk = ctx->n_syrk; h.n_apply = ctx->n_apply;
    h.n_cols = ctx->n_cols; h.n_active_cols = ctx->n_active_cols;
    const Section *secs[kNumSections] = {&ctx->s_subs, &ctx->s_sns, &ctx->s_lcp, &ctx->s_rmap, &ctx->s_trsm,
                                         &ctx->s_trsm_list, &ctx->s_syrk, &ctx->s_syrk_list, &ctx->s_seeds,
                                         &ctx->s_perm, &ctx->s_lambda, &ctx->s_apply, &ctx->s_active,
                                         &ctx->s_cuts, &ctx->s_sblk};
    for (int k = 0; k < kNumSections; ++k) { h.sec_off[k] = secs[k]->off; h.sec_bytes[k] = secs[k]->bytes; }
    std::memcpy(ctx->blob.data(), &h, sizeof(h));
  }

  ctx->ws.status_off = 0;
  ctx->ws.invd_off = 256;
  ctx->ws.y_off = (ctx->ws.invd_off + sizeof(double) * (size_t)lcp_total + 255) & ~size_t(255);
  ctx->ws.total = ctx->ws.y_off + sizeof(double) * (size_t)y_max;
  if (ctx->n_slices > 0) {
    const size_t S = (size_t)ctx->n_slices;
    auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
    ctx->ws.colexp_off = up(ctx->ws.total);
    ctx->ws.yd_off = up(ctx->ws.colexp_off + sizeof(int32_t) * (size_t)col_total);
    ctx->ws.yd_plane = yd_max;
    ctx->ws.ld_off = up(ctx->ws.yd_off + 2 * S * (size_t)yd_max);
    ctx->ws.ld_rows = ld_max;
    ctx->ws.lexp_off = up(ctx->ws.ld_off + 2 * 32 * S * (size_t)ld_max);
    ctx->ws.total = up(ctx->ws.lexp_off + sizeof(int16_t) * (size_t)ld_max);
  }

  ctx->sizes.plan_bytes = ctx->blob.size();
  ctx->sizes.ws_bytes = ctx->ws.total;
  ctx->sizes.F_doubles = ctx->F_offsets[nsub];
  ctx->sizes.L_values = ctx->L_offsets[nsub];
  ctx->sizes.nsub = nsub;
  ctx->sizes.max_m = max_m;

  st.n_supernodes = (int64_t)sns.size();
  st.n_trsm_tasks = ctx->n_trsm;
  st.n_syrk_tasks = ctx->n_syrk;
  st.n_apply_tasks = ctx->n_apply;
  st.y_doubles = y_all + y_total;
  st.n_waves = (int64_t)ctx->waves.size();
  ctx->stats = st;
  return SC_OK;
}

sc::PlanPtrs sc_ctx::ptrs() const {
  const uint8_t *b = static_cast<const uint8_t *>(plan_dev);
  PlanPtrs p;
  p.subs = reinterpret_cast<const SubDev *>(b + s_subs.off);
  p.sns = reinterpret_cast<const SnDev *>(b + s_sns.off);
  p.lcp = reinterpret_cast<const int64_t *>(b + s_lcp.off);
  p.rmap = reinterpret_cast<const int64_t *>(b + s_rmap.off);
  p.trsm_tasks = reinterpret_cast<const TrsmTask *>(b + s_trsm.off);
  p.trsm_list = reinterpret_cast<const int32_t *>(b + s_trsm_list.off);
  p.syrk_tasks = reinterpret_cast<const SyrkTask *>(b + s_syrk.off);
  p.syrk_list = reinterpret_cast<const int32_t *>(b + s_syrk_list.off);
  p.seeds = reinterpret_cast<const Seed *>(b + s_seeds.off);
  p.perm_cols = reinterpret_cast<const int32_t *>(b + s_perm.off);
  p.lambda = reinterpret_cast<const int32_t *>(b + s_lambda.off);
  p.apply_tasks = reinterpret_cast<const ApplyTask *>(b + s_apply.off);
  p.active_cols = reinterpret_cast<const int32_t *>(b + s_active.off);
  p.cuts = reinterpret_cast<const int32_t *>(b + s_cuts.off);
  p.sblk = reinterpret_cast<const int32_t *>(b + s_sblk.off);
  return p;
}

extern "C" {

sc_status sc_plan(sc_ctx **out, int32_t nsub, const sc_subdomain_desc *subdomains, int64_t n_dual,
                  const sc_options *opt) {
  if (!out) return SC_ERR_INVALID_ARG;
  *out = nullptr;
  sc_ctx *ctx = new (std::nothrow) sc_ctx();
  if (!ctx) return SC_ERR_OOM;
  sc_status st = SC_OK;
  if (nsub < 0 || (nsub > 0 && !subdomains) || n_dual < 0) {
    st = fail(ctx, SC_ERR_INVALID_ARG, "nsub < 0, NULL subdomain array or n_dual < 0");
  } else if (opt && opt->precision != SC_FP64 && opt->precision != SC_SPLIT_BF16) {
    st = fail(ctx, SC_ERR_INVALID_ARG, "unsupported precision");
  } else if (opt && opt->precision == SC_SPLIT_BF16 && opt->n_slices != 0 &&
             (opt->n_slices < 3 || opt->n_slices > 7)) {
    st = fail(ctx, SC_ERR_INVALID_ARG, "n_slices must be 3..7 (or 0 for 7)");
  } else {
    const int8_t dflt = (opt && opt->precision == SC_SPLIT_BF16) ? (int8_t)(opt->n_slices ? opt->n_slices : 7) : 0;
    ctx->sub_var.assign(nsub > 0 ? nsub : 0, dflt);
    for (int32_t i = 0; i < nsub && opt && opt->sub_slices; ++i) {
      const int8_t v = opt->sub_slices[i];
      if (v != 0 && (v < 3 || v > 7)) {
        st = fail(ctx, SC_ERR_INVALID_ARG, "sub_slices entries must be 0 or 3..7");
        break;
      }
      ctx->sub_var[i] = v;
    }
    if (st == SC_OK && opt && opt->tile != SC_TILE_32 && opt->tile != SC_TILE_TC128)
      st = fail(ctx, SC_ERR_INVALID_ARG, "tile must be SC_TILE_32 or SC_TILE_TC128");
    for (int32_t i = 0; i < nsub && st == SC_OK && opt; ++i) {
      const int tile = opt->sub_tile ? opt->sub_tile[i] : opt->tile;
      if (tile != SC_TILE_32 && tile != SC_TILE_TC128) {
        st = fail(ctx, SC_ERR_INVALID_ARG, "sub_tile entries must be 0 or 1");
        break;
      }
      if (tile == SC_TILE_TC128 && ctx->sub_var[i] != 0) ctx->sub_var[i] = (int8_t)(ctx->sub_var[i] | kVarTile);
    }
    if (st == SC_OK && opt && opt->poll_limit < 0) st = fail(ctx, SC_ERR_INVALID_ARG, "poll_limit < 0");
    ctx->poll_limit = opt ? opt->poll_limit : 0;
    for (int8_t v : ctx->sub_var) ctx->n_slices = std::max<int32_t>(ctx->n_slices, var_digits(v));
    ctx->precision = ctx->n_slices > 0 ? SC_SPLIT_BF16 : SC_FP64;
    if (opt && opt->ws_limit < 0) st = fail(ctx, SC_ERR_INVALID_ARG, "ws_limit < 0");
    ctx->ws_limit = opt ? opt->ws_limit : 0;
    if (opt && opt->persistent != 0 && opt->persistent != 1) st = fail(ctx, SC_ERR_INVALID_ARG, "persistent must be 0 or 1");
    ctx->persistent = opt ? opt->persistent : 0;
  }
  if (st == SC_OK && !(nsub < 0 || (nsub > 0 && !subdomains) || n_dual < 0)) {
    ctx->nsub = nsub;
    ctx->n_dual = n_dual;
    try {
      st = build_plan(ctx, nsub, subdomains);
    } catch (const std::bad_alloc &) {
      st = fail(ctx, SC_ERR_OOM, "host allocation failed while planning");
    } catch (...) {
      st = fail(ctx, SC_ERR_INTERNAL, "unexpected exception while planning");
    }
  }
  *out = ctx;  // the context carries the error message even on failure
  return st;
}

sc_status sc_get_sizes(const sc_ctx *ctx, sc_sizes *o) {
  if (!ctx || !o) return SC_ERR_INVALID_ARG;
  *o = ctx->sizes;
  return SC_OK;
}

sc_status sc_get_stats(const sc_ctx *ctx, sc_stats *o) {
  if (!ctx || !o) return SC_ERR_INVALID_ARG;
  *o = ctx->stats;
  return SC_OK;
}

sc_status sc_get_offsets(const sc_ctx *ctx, int64_t *F_offsets, int64_t *L_offsets) {
  if (!ctx) return SC_ERR_INVALID_ARG;
  if (F_offsets) std::memcpy(F_offsets, ctx->F_offsets.data(), sizeof(int64_t) * ctx->F_offsets.size());
  if (L_offsets) std::memcpy(L_offsets, ctx->L_offsets.data(), sizeof(int64_t) * ctx->L_offsets.size());
  return SC_OK;
}

sc_status sc_export_plan(const sc_ctx *ctx, void *dst, size_t bytes) {
  if (!ctx || (!dst && bytes)) return SC_ERR_INVALID_ARG;
  if (bytes < ctx->blob.size()) return SC_ERR_OOM;
  if (!ctx->blob.empty()) std::memcpy(dst, ctx->blob.data(), ctx->blob.size());
  return SC_OK;
}

sc_status sc_workspace_layout(const sc_ctx *ctx, size_t *status_off, size_t *invdiag_off, size_t *y_off) {
  if (!ctx) return SC_ERR_INVALID_ARG;
  if (status_off) *status_off = ctx->ws.status_off;
  if (invdiag_off) *invdiag_off = ctx->ws.invd_off;
  if (y_off) *y_off = ctx->ws.y_off;
  return SC_OK;
}

const char *sc_last_error(const sc_ctx *ctx) { return ctx ? ctx->err.c_str() : "NULL context"; }

void sc_destroy(sc_ctx *ctx) { delete ctx; }

}  // extern "C"
