// Implicit application of the dual operator on the GPU (include/sc_implicit.h):
// per subdomain q += B L^{-T} L^{-1} B^T lambda with two sparse triangular
// solves over the supernodes of L (paper Sec. 2.2, Eq. "dualop_apply_impl").
//
// Host side (sci_plan): the symbolic analysis of sc_plan (fundamental
// supernodes, the supernodes reached from B^T's rows), then per subdomain a
// level schedule of the reached supernodes by etree height (leaves 0; a
// parent is at least one level above each child), B^T grouped by row for the
// gather and by entry for the scatter.
//
// Device side: one CTA per subdomain (largest first).  Forward solve level by
// level upwards, backward solve level by level downwards, the warps sharing
// the supernodes of a level; a barrier between levels.  A warp solves its
// supernode in 32-column blocks:
//   forward   the block's triangle with lane = row (32 shuffle steps, the
//             block's L entries prefetched into registers), then the panel
//             below (the supernode's remaining diagonal rows and its pruned
//             rows) updated with lane = row and coalesced column reads;
//             updates of ancestor rows are FP64 atomic additions (other
//             warps of the level may hit the same ancestor row);
//   backward  blocks in descending order; the panel's contribution
//             sum_t L(t, k) z_t per block column k accumulated per lane
//             (lane = row, coalesced column reads) and summed across the warp
//             by a 31-step transpose-reduce (lane k ends with column k), then
//             the transposed triangle with lane = column.
// Levels with fewer than four supernodes (the top of the tree, where the
// large separators are) run each supernode on the whole CTA instead: warp 0
// solves the triangle, all warps share the panel rows.
// A fundamental supernode's CSC columns are its dense trapezoidal panel
// columns: local column t (0-based) holds rows t..ns-1 of the diagonal block
// then the rs pruned rows, and starts off(t) = t (ns + rs) - t (t - 1) / 2
// entries after column 0's diagonal.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <new>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "sc_implicit.h"
#include "sc_internal.h"

namespace {

namespace cg = cooperative_groups;

// 16 warps per CTA and one CTA per SM while a batch has at most one
// subdomain per SM: a subdomain that a CTA solves alone gets twice the warps
// for the wide lower levels of its elimination tree (many small supernodes,
// one warp each); 8 warps and two CTAs per SM for larger batches
constexpr int kWarps = 16;      // warps per CTA at most (the planner picks 8 or 16 per batch)
constexpr int kCluster = 8;     // CTAs per cluster (portable maximum)
constexpr int64_t kCtaSlots = 152;   // resident CTAs on a GB300 (152 SMs, 1 CTA each)
constexpr int kThreadsI = 32 * kWarps;
constexpr uint32_t kFull = 0xffffffffu;

struct ISub {
  int64_t x_off;                // doubles, this subdomain's n-vector in the workspace
  int32_t n, sn_lo, sn_hi;      // supernodes [sn_lo, sn_hi), ordered by (level, first column)
  int32_t lev_lo, n_lev;        // level boundaries levptr[lev_lo .. lev_lo + n_lev]
  int32_t g_lo, g_hi;           // gather rows
  int32_t s_lo, s_hi;           // scatter entries
  // solved by a CTA pair (item kind 2): the levels are those of subtree part
  // A (n_lev_a), then part B (n_lev_b), then the top chain above the split;
  // scatter entries [s_lo, s_mid1) lie in part A, [s_mid1, s_mid2) in B, the
  // rest in the top.  Otherwise n_lev_a = n_lev_b = 0, s_mid1 = s_mid2 = s_lo.
  int32_t n_lev_a, n_lev_b, s_mid1, s_mid2;
  int32_t pad;
};
static_assert(sizeof(ISub) == 64, "ISub layout");

struct ISn {
  int64_t lval;      // absolute index of L(c0, c0) in the concatenated values
  int64_t rows_off;  // first of the rs pruned rows in `rows`
  int32_t c0, ns, rs, sub;
};
static_assert(sizeof(ISn) == 32, "ISn layout");

struct IRow {
  int32_t r, e_lo, e_hi, pad;   // local row r of B^T, its entries [e_lo, e_hi) in gent
};
struct IEnt {
  int32_t gj, sign;             // global multiplier, +1 / -1
};
struct ISEnt {
  int32_t r, gj, sign, pad;     // one B^T entry: local row, global multiplier, sign
};

struct IItem {
  int32_t kind;                 // 0: sub[0] on the whole cluster; 1: sub[r] on CTA r, r < n;
                                // 2: sub[j] on the CTA pair (2j, 2j + 1), j < n <= kCluster / 2
  int32_t n;
  int32_t sub[kCluster];        // indices into the subdomain table
};
static_assert(sizeof(IItem) == 40, "IItem layout");

constexpr int kSections = 8;
struct IHeader {
  uint32_t magic;     // 'SCIP'
  uint32_t version;   // 1
  int32_t nsub, pad;
  int64_t n_sn, n_levptr, n_rows, n_grow, n_gent, n_sent, n_items;
  uint64_t sec_off[kSections];   // subs sns levptr rows grow gent sent items
};
constexpr size_t kIHeaderBytes = 256;
static_assert(sizeof(IHeader) <= kIHeaderBytes, "implicit plan header");

struct IPtrs {
  const ISub *subs;
  const ISn *sns;
  const int32_t *levptr;
  const int32_t *rows;
  const IRow *grow;
  const IEnt *gent;
  const ISEnt *sent;
  const IItem *items;
  int64_t rd_off;      // doubles from a subdomain's x to its reciprocal diagonals (workspace)
};

__device__ __forceinline__ int col_off(int t, int nr) {
  // 32-bit: the planner checks that every visited panel holds fewer than 2^31 entries
  return t * nr - t * (t - 1) / 2;
}

// Loads of x: when a subdomain spans a cluster, x is written by several SMs
// and read after cluster barriers, so reads bypass the (non-coherent) L1.
template <bool CL>
__device__ __forceinline__ double ldx(const double *p) {
  if constexpr (CL) return __ldcg(p);
  else return *p;
}

// Forward triangle of one 32-column block (one warp, lane = row): y = L_bb^{-1} x_b,
// written to x; returns the lane's y (0 for lanes >= w).
template <bool CL>
__device__ __forceinline__ double forward_triangle(const double *__restrict__ L, int nr, int kb, int w, double *xs,
                                                   int64_t rd_off, int lane) {
  const double inv = lane < w ? ldx<CL>(xs + rd_off + kb + lane) : 0.0;   // 1 / L(c, c), computed per call
  // lane i: L(kb + i, kb + k) for k < i, entry (i - k) of column kb + k, at
  // col_off(kb + k) + i - k: one offset stepped by nr - (kb + k) - 1 per column
  double lv[32];
  int o = col_off(kb, nr) + lane;
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    lv[k] = (k < w && k < lane && lane < w) ? L[o] : 0.0;
    o += nr - (kb + k) - 1;
  }
  double xi = lane < w ? ldx<CL>(xs + kb + lane) : 0.0;
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    if (k < w) {   // uniform
      const double yk = __shfl_sync(kFull, xi, k) * __shfl_sync(kFull, inv, k);
      xi = lane == k ? yk : fma(-lv[k], yk, xi);
    }
  }
  if (lane < w) xs[kb + lane] = xi;
  return xi;
}

// Forward panel update for local rows t0 + lane (one warp):
// x_t -= sum_k L(t, kb + k) y_k.  Rows of the supernode's own diagonal block
// belong to this warp alone; rows below are ancestors' rows that other warps
// (or SMs) may update at the same level: atomic.
template <bool CL>
__device__ __forceinline__ void forward_panel_chunk(const double *__restrict__ L, const int32_t *__restrict__ R,
                                                    int ns, int nr, int kb, int w, int t0, const double *ys,
                                                    double *xs, double *x, int lane) {
  const int t = t0 + lane;
  const bool ok = t < nr;
  double lv[32];
#pragma unroll
  // entry (t, c) of the panel at col_off(c) + t - c, and col_off(c + 1) = col_off(c) + nr - c
  int o = col_off(kb, nr) + (t - kb);
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    lv[k] = (k < w && ok) ? L[o] : 0.0;
    o += nr - (kb + k) - 1;
  }
  double acc = 0.0;
#pragma unroll
  for (int k = 0; k < 32; ++k)
    if (k < w) acc = fma(lv[k], ys[k], acc);
  if (!ok) return;
  if (t < ns) xs[t] = ldx<CL>(xs + t) - acc;
  else atomicAdd(x + R[t - ns], -acc);
}

// Backward: per-lane partial sums acc[k] += L(t, kb + k) z_t over local rows t0 + lane.
template <bool CL>
__device__ __forceinline__ void backward_panel_chunk(const double *__restrict__ L, const int32_t *__restrict__ R,
                                                     int ns, int nr, int kb, int w, int t0, const double *xs,
                                                     const double *x, double (&acc)[32], int lane) {
  const int t = t0 + lane;
  const bool ok = t < nr;
  const double zt = ok ? (t < ns ? ldx<CL>(xs + t) : ldx<CL>(x + R[t - ns])) : 0.0;
  int o = col_off(kb, nr) + (t - kb);
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    if (k < w && ok) acc[k] = fma(L[o], zt, acc[k]);
    o += nr - (kb + k) - 1;
  }
}

// Warp transpose-reduce: on return lane k holds the sum over the warp's lanes
// of acc[k] (31 shuffle-add steps; acc is destroyed).
__device__ __forceinline__ double transpose_reduce(double (&acc)[32], int lane) {
#pragma unroll
  for (int h = 16; h >= 1; h >>= 1) {
    const bool up = (lane & h) != 0;
#pragma unroll
    for (int j = 0; j < h; ++j) {
      const double send = up ? acc[j] : acc[j + h];
      const double keep = up ? acc[j + h] : acc[j];
      acc[j] = keep + __shfl_xor_sync(kFull, send, h);
    }
  }
  return acc[0];
}

// The same for the first w < 32 columns (acc[k] = 0 for k >= w): a
// transpose-reduce over groups of P lanes (P the power of two >= w), then a
// butterfly across the 32 / P groups: P - 1 + 5 - log2 P additions instead of 31.
__device__ __forceinline__ double transpose_reduce_w(double (&acc)[32], int lane, int w) {
  if (w > 16) return transpose_reduce(acc, lane);
  const int P = w <= 1 ? 1 : w <= 2 ? 2 : w <= 4 ? 4 : w <= 8 ? 8 : 16;
#pragma unroll
  for (int h = 8; h >= 1; h >>= 1) {
    if (h < P) {   // uniform
      const bool up = (lane & h) != 0;
#pragma unroll
      for (int j = 0; j < h; ++j) {
        const double send = up ? acc[j] : acc[j + h];
        const double keep = up ? acc[j + h] : acc[j];
        acc[j] = keep + __shfl_xor_sync(kFull, send, h);
      }
    }
  }
  double v = acc[0];
  for (int m = P; m < 32; m <<= 1) v += __shfl_xor_sync(kFull, v, m);
  return v;
}

// Backward triangle of one block (one warp, lane = column): z = L_bb^{-T} rhs, written to x.
template <bool CL>
__device__ __forceinline__ void backward_triangle(const double *__restrict__ L, int nr, int kb, int w, double rhs,
                                                  double *xs, int64_t rd_off, int lane) {
  const double inv = lane < w ? ldx<CL>(xs + rd_off + kb + lane) : 0.0;
  // lane k: L(kb + i, kb + k) for i > k, entry (i - k) of its own column
  const double *pc = L + (lane < w ? col_off(kb + lane, nr) - lane : 0);
  double lc[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) lc[i] = (i > lane && i < w) ? pc[i] : 0.0;
#pragma unroll
  for (int i = 31; i >= 0; --i) {
    if (i < w) {   // uniform
      if (lane == i) rhs *= inv;
      const double zi = __shfl_sync(kFull, rhs, i);
      rhs = fma(-lc[i], zi, rhs);
    }
  }
  if (lane < w) xs[kb + lane] = rhs;
}

// A group of warps solving supernodes together: the whole cluster, one CTA,
// or a subgroup of a CTA's warps (consecutive warps w0 .. w0 + nwl - 1 with
// their own named barrier `bar`).  warp: the warp's index in its CTA; gw,
// nw: its index and the warp count across the group; slot: the group's row
// of the CTA's 32-double reduction buffer.
struct Group {
  int rank, size, warp, lane, gw, nw;
  bool cluster;
  int w0, nwl, bar, slot;
  // the warps of the group in this CTA
  __device__ void sync_cta() const {
    if (bar == 0) __syncthreads();
    else asm volatile("bar.sync %0, %1;\n" ::"r"(bar), "r"(32 * nwl) : "memory");
  }
  __device__ void sync() const {
    if (cluster) cg::this_cluster().sync();
    else sync_cta();
  }
};

__device__ __forceinline__ int nwarps() { return (int)(blockDim.x >> 5); }

__device__ __forceinline__ Group cta_group(int warp, int lane) {
  return Group{0, 1, warp, lane, warp, nwarps(), false, 0, nwarps(), 0, 0};
}

// warps [w0, w0 + nwl) of this CTA, named barrier 1 + slot (slot < kWarps - 1)
__device__ __forceinline__ Group sub_group(int warp, int lane, int w0, int nwl, int slot) {
  return Group{0, 1, warp, lane, warp - w0, nwl, false, w0, nwl, nwl == nwarps() ? 0 : 1 + slot, slot};
}

__device__ __forceinline__ Group cluster_group(int warp, int lane) {
  cg::cluster_group c = cg::this_cluster();
  const int r = (int)c.block_rank(), n = (int)c.num_blocks();
  return Group{r, n, warp, lane, r * nwarps() + warp, n * nwarps(), true, 0, nwarps(), 0, 0};
}

// One supernode by one warp.
template <bool CL>
__device__ void forward_warp(const ISn &sn, const double *__restrict__ Lv, const int32_t *__restrict__ rows,
                             double *x, double *ys, int64_t rd_off, int lane) {
  const int ns = sn.ns, nr = ns + sn.rs;
  const double *L = Lv + sn.lval;
  const int32_t *R = rows + sn.rows_off;
  double *xs = x + sn.c0;
  for (int kb = 0; kb < ns; kb += 32) {
    const int w = min(32, ns - kb);
    ys[lane] = forward_triangle<CL>(L, nr, kb, w, xs, rd_off, lane);
    __syncwarp();
    for (int t0 = kb + w; t0 < nr; t0 += 32) forward_panel_chunk<CL>(L, R, ns, nr, kb, w, t0, ys, xs, x, lane);
    __syncwarp();
  }
}

template <bool CL>
__device__ void backward_warp(const ISn &sn, const double *__restrict__ Lv, const int32_t *__restrict__ rows,
                              double *x, int64_t rd_off, int lane) {
  const int ns = sn.ns, nr = ns + sn.rs;
  const double *L = Lv + sn.lval;
  const int32_t *R = rows + sn.rows_off;
  double *xs = x + sn.c0;
  for (int kb = ((ns - 1) / 32) * 32; kb >= 0; kb -= 32) {
    const int w = min(32, ns - kb);
    double acc[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) acc[k] = 0.0;
    for (int t0 = kb + w; t0 < nr; t0 += 32) backward_panel_chunk<CL>(L, R, ns, nr, kb, w, t0, xs, x, acc, lane);
    const double part = transpose_reduce_w(acc, lane, w);
    const double rhs = lane < w ? ldx<CL>(xs + kb + lane) - part : 0.0;
    backward_triangle<CL>(L, nr, kb, w, rhs, xs, rd_off, lane);
    __syncwarp();
  }
}

// Two supernodes of at most 16 columns on one warp, one per 16-lane half
// (lane & 15 = row or column within the half).  Every loop runs to the
// larger of the two halves' bounds and every shuffle and __syncwarp is taken
// by the whole warp; a half's rows and columns past its own supernode stay
// zero, so they add nothing.  valid = false: the half has no supernode.  A
// supernode of at most 16 columns is one block, and every row below it is a
// pruned row (an ancestor's).
template <bool CL>
__device__ void forward_half(const ISn &sn, bool valid, const double *__restrict__ Lv,
                             const int32_t *__restrict__ rows, double *x, double *ys, int64_t rd_off, int lane) {
  const int hl = lane & 15, h = lane >> 4;
  const int ns = valid ? sn.ns : 0, nr = valid ? sn.ns + sn.rs : 0;
  const double *L = Lv + (valid ? sn.lval : 0);
  const int32_t *R = rows + (valid ? sn.rows_off : 0);
  double *xs = x + (valid ? sn.c0 : 0);
  const int wmax = max(ns, __shfl_xor_sync(kFull, ns, 16));
  const int nch = (nr - ns + 15) >> 4, chmax = max(nch, __shfl_xor_sync(kFull, nch, 16));
  const double inv = hl < ns ? ldx<CL>(xs + rd_off + hl) : 0.0;
  // lane i: L(i, k) for k < i, entry (i - k) of column k (offsets stepped column to column)
  double lv[16];
  int o = hl;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    lv[k] = (k < ns && k < hl && hl < ns) ? L[o] : 0.0;
    o += nr - k - 1;
  }
  double xi = hl < ns ? ldx<CL>(xs + hl) : 0.0;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    if (k < wmax) {   // uniform
      const double yk = __shfl_sync(kFull, xi, k, 16) * __shfl_sync(kFull, inv, k, 16);
      xi = hl == k ? yk : fma(-lv[k], yk, xi);
    }
  }
  if (hl < ns) xs[hl] = xi;
  ys[16 * h + hl] = hl < ns ? xi : 0.0;
  __syncwarp();
  for (int ch = 0; ch < chmax; ++ch) {
    const int t = ns + 16 * ch + hl;
    const bool ok = t < nr;
    int oo = t;
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      if (k < wmax) {   // uniform
        const double l = (k < ns && ok) ? L[oo] : 0.0;
        acc = fma(l, ys[16 * h + k], acc);
      }
      oo += nr - k - 1;
    }
    if (ok) atomicAdd(x + R[t - ns], -acc);
  }
  __syncwarp();
}

template <bool CL>
__device__ void backward_half(const ISn &sn, bool valid, const double *__restrict__ Lv,
                              const int32_t *__restrict__ rows, double *x, int64_t rd_off, int lane) {
  const int hl = lane & 15;
  const int ns = valid ? sn.ns : 0, nr = valid ? sn.ns + sn.rs : 0;
  const double *L = Lv + (valid ? sn.lval : 0);
  const int32_t *R = rows + (valid ? sn.rows_off : 0);
  double *xs = x + (valid ? sn.c0 : 0);
  const int wmax = max(ns, __shfl_xor_sync(kFull, ns, 16));
  const int nch = (nr - ns + 15) >> 4, chmax = max(nch, __shfl_xor_sync(kFull, nch, 16));
  double acc[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) acc[k] = 0.0;
  for (int ch = 0; ch < chmax; ++ch) {
    const int t = ns + 16 * ch + hl;
    const bool ok = t < nr;
    const double zt = ok ? ldx<CL>(x + R[t - ns]) : 0.0;
    int oo = t;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      if (k < wmax && k < ns && ok) acc[k] = fma(L[oo], zt, acc[k]);
      oo += nr - k - 1;
    }
  }
  // sum of acc[k] over the half's lanes, lane k of the half ending with column k: a
  // transpose-reduce over groups of P lanes (P the power of two >= wmax), then a butterfly
  // across the half's 16 / P groups (xor distances below 16 stay inside the half)
  const int P = wmax <= 1 ? 1 : wmax <= 2 ? 2 : wmax <= 4 ? 4 : wmax <= 8 ? 8 : 16;
#pragma unroll
  for (int hh = 8; hh >= 1; hh >>= 1) {
    if (hh < P) {   // uniform
      const bool up = (lane & hh) != 0;
#pragma unroll
      for (int j = 0; j < hh; ++j) {
        const double send = up ? acc[j] : acc[j + hh];
        const double keep = up ? acc[j + hh] : acc[j];
        acc[j] = keep + __shfl_xor_sync(kFull, send, hh);
      }
    }
  }
  double part = acc[0];
  for (int m = P; m < 16; m <<= 1) part += __shfl_xor_sync(kFull, part, m);
  double rhs = hl < ns ? ldx<CL>(xs + hl) - part : 0.0;
  const double inv = hl < ns ? ldx<CL>(xs + rd_off + hl) : 0.0;
  // lane k: L(i, k) for i > k, entry (i - k) of its own column
  const double *pc = L + (hl < ns ? col_off(hl, nr) - hl : 0);
  double lc[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) lc[i] = (i > hl && i < ns) ? pc[i] : 0.0;
#pragma unroll
  for (int i = 15; i >= 0; --i) {
    if (i < wmax) {   // uniform
      if (hl == i) rhs *= inv;
      const double zi = __shfl_sync(kFull, rhs, i, 16);
      rhs = fma(-lc[i], zi, rhs);
    }
  }
  if (hl < ns) xs[hl] = rhs;
  __syncwarp();
}

// One supernode by a CTA (CL = false; warps of this CTA) or by the whole
// cluster (CL = true): the triangle by the group's first warp, the panel rows
// spread over all the group's warps.
template <bool CL>
__device__ void forward_group(const Group &g, const ISn &sn, const double *__restrict__ Lv,
                              const int32_t *__restrict__ rows, double *x, double *ys, int64_t rd_off) {
  const int ns = sn.ns, nr = ns + sn.rs;
  const double *L = Lv + sn.lval;
  const int32_t *R = rows + sn.rows_off;
  double *xs = x + sn.c0;
  for (int kb = 0; kb < ns; kb += 32) {
    const int w = min(32, ns - kb);
    if (g.gw == 0) forward_triangle<CL>(L, nr, kb, w, xs, rd_off, g.lane);
    g.sync();
    ys[g.lane] = g.lane < w ? ldx<CL>(xs + kb + g.lane) : 0.0;
    __syncwarp();
    for (int t0 = kb + w + 32 * g.gw; t0 < nr; t0 += 32 * g.nw)
      forward_panel_chunk<CL>(L, R, ns, nr, kb, w, t0, ys, xs, x, g.lane);
    g.sync();
  }
}

// red: this CTA's kWarps x 32 doubles; red_cta: its 32-double sum (read by
// the group's first CTA through distributed shared memory when CL).
template <bool CL>
__device__ void backward_group(const Group &g, const ISn &sn, const double *__restrict__ Lv,
                               const int32_t *__restrict__ rows, double *x, int64_t rd_off, double *red,
                               double *red_cta) {
  const int ns = sn.ns, nr = ns + sn.rs;
  const double *L = Lv + sn.lval;
  const int32_t *R = rows + sn.rows_off;
  double *xs = x + sn.c0;
  for (int kb = ((ns - 1) / 32) * 32; kb >= 0; kb -= 32) {
    const int w = min(32, ns - kb);
    double acc[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) acc[k] = 0.0;
    for (int t0 = kb + w + 32 * g.gw; t0 < nr; t0 += 32 * g.nw)
      backward_panel_chunk<CL>(L, R, ns, nr, kb, w, t0, xs, x, acc, g.lane);
    red[g.warp * 32 + g.lane] = transpose_reduce_w(acc, g.lane, w);
    g.sync_cta();
    if (g.warp == g.w0) {
      double s = 0.0;
      for (int v = g.w0; v < g.w0 + g.nwl; ++v) s += red[v * 32 + g.lane];
      red_cta[32 * g.slot + g.lane] = s;
    }
    g.sync();
    if (g.gw == 0) {
      double part = red_cta[32 * g.slot + g.lane];
      if (g.cluster) {
        cg::cluster_group c = cg::this_cluster();
        for (int r = 1; r < g.size; ++r) part += c.map_shared_rank(red_cta, r)[g.lane];
      }
      const double rhs = g.lane < w ? ldx<CL>(xs + kb + g.lane) - part : 0.0;
      backward_triangle<CL>(L, nr, kb, w, rhs, xs, rd_off, g.lane);
    }
    g.sync();
  }
}

// L2 prefetch of what level `lev` reads first (its supernodes' descriptors,
// L panels and pruned-row lists), spread over the group's warps: issued at
// the top of the level before, so that the level's dependent loads (a
// descriptor, then its panel, then the rows it updates) hit L2 instead of
// HBM.  A prefetch only moves data into the cache; it changes no value.
__device__ __forceinline__ void prefetch_l2(const void *p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ void prefetch_level(const Group &g, const IPtrs &P, int lev, const double *__restrict__ Lv) {
  const int a = P.levptr[lev], b = P.levptr[lev + 1];
  for (int s = a + g.gw; s < b; s += g.nw) {
    const ISn sn = P.sns[s];
    const int nr = sn.ns + sn.rs;
    const char *lo = reinterpret_cast<const char *>(Lv + sn.lval);
    const char *hi = reinterpret_cast<const char *>(Lv + sn.lval + col_off(sn.ns, nr));
    const char *first = reinterpret_cast<const char *>(reinterpret_cast<uintptr_t>(lo) & ~uintptr_t(127));
    for (const char *q = first + 128 * g.lane; q < hi; q += 128 * 32) prefetch_l2(q);
    if (g.lane == 0 && sn.rs > 0) prefetch_l2(P.rows + sn.rows_off);
  }
  // the descriptors (32 bytes each; four to a line), inside the level's range
  for (int k = a + 4 * (32 * g.gw + g.lane); k < b; k += 4 * 32 * g.nw) prefetch_l2(P.sns + k);
}

// The levels [lev_lo, lev_lo + n_lev) of a subdomain by one group (CL: x
// read past L1).  Per etree level, by its supernode count c: c >= half the
// group's warps -- one warp per supernode; else c >= the group's CTAs -- one
// CTA per supernode (the CTA's warps share its panel rows); else (the top
// separators) one supernode at a time on the whole group.  One group barrier
// per level, two per 32-column block in the last case.
// ctr (one CTA's group only; nullptr for a cluster): a shared counter from
// which the warps of a level with one warp per supernode take their next
// supernode (largest first, as the planner orders them), so that they finish
// the level together; never reset within a call -- `base` counts the takes so
// far (a level of c supernodes takes c + (warps) times: each warp's last take
// finds the level empty).
__device__ __forceinline__ int take(int *ctr, int base, int lane, int n = 1) {
  int idx = 0;
  if (lane == 0) idx = atomicAdd(ctr, n) - base;
  return __shfl_sync(kFull, idx, 0);
}

// A level whose largest supernode (the first: the planner orders a level by
// work) has at most 16 columns is taken two supernodes at a time, one per
// half-warp (forward_half / backward_half); a pair with a wider member runs
// on the whole warp one after the other.  The level then takes
// 2 (ceil(c / 2) + warps) numbers.
template <bool CL, bool FWD>
__device__ void tiny_level(const Group &g, const IPtrs &P, int a, int c, const double *__restrict__ Lv, double *x,
                           double *ys, int64_t rd, int *ctr, int &base) {
  for (int k = take(ctr, base, g.lane, 2); k < c; k = take(ctr, base, g.lane, 2)) {
    const ISn s0 = P.sns[a + k];
    const bool two = k + 1 < c;
    const ISn s1 = two ? P.sns[a + k + 1] : s0;
    if (s0.ns <= 16 && (!two || s1.ns <= 16)) {
      const bool hi = g.lane >= 16;
      if (FWD) forward_half<CL>(hi ? s1 : s0, !hi || two, Lv, P.rows, x, ys, rd, g.lane);
      else backward_half<CL>(hi ? s1 : s0, !hi || two, Lv, P.rows, x, rd, g.lane);
    } else {
      if (FWD) forward_warp<CL>(s0, Lv, P.rows, x, ys, rd, g.lane);
      else backward_warp<CL>(s0, Lv, P.rows, x, rd, g.lane);
      if (two) {
        if (FWD) forward_warp<CL>(s1, Lv, P.rows, x, ys, rd, g.lane);
        else backward_warp<CL>(s1, Lv, P.rows, x, rd, g.lane);
      }
    }
  }
  base += 2 * ((c + 1) / 2 + g.nw);
}

template <bool CL>
__device__ void forward_levels(const Group &g, const IPtrs &P, int lev_lo, int n_lev, const double *__restrict__ Lv,
                               double *x, double (*ys)[32], int *ctr, int &base) {
  const int64_t rd = P.rd_off;
  const Group cta = cta_group(g.warp, g.lane);
  if (n_lev > 0) prefetch_level(g, P, lev_lo, Lv);
  for (int l = 0; l < n_lev; ++l) {
    if (l + 1 < n_lev) prefetch_level(g, P, lev_lo + l + 1, Lv);
    const int a = P.levptr[lev_lo + l], b = P.levptr[lev_lo + l + 1];
    if (2 * (b - a) >= g.nw) {
      if (ctr && P.sns[a].ns <= 16) {
        tiny_level<CL, true>(g, P, a, b - a, Lv, x, ys[g.warp], rd, ctr, base);
      } else if (ctr) {
        for (int k = take(ctr, base, g.lane); k < b - a; k = take(ctr, base, g.lane))
          forward_warp<CL>(P.sns[a + k], Lv, P.rows, x, ys[g.warp], rd, g.lane);
        base += (b - a) + g.nw;
      } else {
        for (int s = a + g.gw; s < b; s += g.nw) forward_warp<CL>(P.sns[s], Lv, P.rows, x, ys[g.warp], rd, g.lane);
      }
      g.sync();
    } else if (!g.cluster && b - a >= 2) {
      // 2 .. 7 supernodes on one CTA: each on its own subgroup of the warps, side by side
      const int W = nwarps(), c = b - a, j = g.warp * c / W, w0 = (W * j + c - 1) / c;
      const Group sg = sub_group(g.warp, g.lane, w0, (W * (j + 1) + c - 1) / c - w0, j);
      forward_group<CL>(sg, P.sns[a + j], Lv, P.rows, x, ys[g.warp], rd);
      __syncthreads();
    } else if (b - a >= g.size) {
      for (int s = a + g.rank; s < b; s += g.size) forward_group<CL>(cta, P.sns[s], Lv, P.rows, x, ys[g.warp], rd);
      if (g.cluster) g.sync();
    } else {
      for (int s = a; s < b; ++s) forward_group<CL>(g, P.sns[s], Lv, P.rows, x, ys[g.warp], rd);
    }
  }
}

template <bool CL>
__device__ void backward_levels(const Group &g, const IPtrs &P, int lev_lo, int n_lev,
                                const double *__restrict__ Lv, double *x, double *red, double *red_cta, int *ctr,
                                int &base) {
  const int64_t rd = P.rd_off;
  const Group cta = cta_group(g.warp, g.lane);
  for (int l = n_lev - 1; l >= 0; --l) {
    if (l > 0) prefetch_level(g, P, lev_lo + l - 1, Lv);
    const int a = P.levptr[lev_lo + l], b = P.levptr[lev_lo + l + 1];
    if (2 * (b - a) >= g.nw) {
      if (ctr && P.sns[a].ns <= 16) {
        tiny_level<CL, false>(g, P, a, b - a, Lv, x, nullptr, rd, ctr, base);
      } else if (ctr) {
        for (int k = take(ctr, base, g.lane); k < b - a; k = take(ctr, base, g.lane))
          backward_warp<CL>(P.sns[a + k], Lv, P.rows, x, rd, g.lane);
        base += (b - a) + g.nw;
      } else {
        for (int s = a + g.gw; s < b; s += g.nw) backward_warp<CL>(P.sns[s], Lv, P.rows, x, rd, g.lane);
      }
      g.sync();
    } else if (!g.cluster && b - a >= 2) {
      const int W = nwarps(), c = b - a, j = g.warp * c / W, w0 = (W * j + c - 1) / c;
      const Group sg = sub_group(g.warp, g.lane, w0, (W * (j + 1) + c - 1) / c - w0, j);
      backward_group<CL>(sg, P.sns[a + j], Lv, P.rows, x, rd, red, red_cta);
      __syncthreads();
    } else if (b - a >= g.size) {
      for (int s = a + g.rank; s < b; s += g.size) backward_group<CL>(cta, P.sns[s], Lv, P.rows, x, rd, red, red_cta);
      if (g.cluster) g.sync();
    } else {
      for (int s = a; s < b; ++s) backward_group<CL>(g, P.sns[s], Lv, P.rows, x, rd, red, red_cta);
    }
  }
}

// 1 / d for a diagonal entry d; ok: d positive and finite (tested on the bit
// pattern).  In single precision's range by Newton's iteration for the
// reciprocal, r <- r + r (1 - d r), from the single-precision reciprocal of d:
// two steps take its 24 correct bits past FP64's 53 (four FMAs and two
// conversions against the longer sequence of an FP64 division); otherwise a
// division.
__device__ __forceinline__ double pos_recip(double d, bool &ok) {
  const long long b = __double_as_longlong(d);
  const int ex = (int)((b >> 52) & 0x7FF);
  ok = b > 0 && ex < 0x7FF;
  if (ex > 1023 - 120 && ex < 1023 + 120) {
    double r = (double)__frcp_rn(__double2float_rn(d));
    double e = fma(-d, r, 1.0);
    r = fma(r, e, r);
    e = fma(-d, r, 1.0);
    return fma(r, e, r);
  }
  return 1.0 / d;
}

// x = B^T lambda for one subdomain (threads gt of nt), and the reciprocal
// diagonal 1 / L(c, c) of every column of its visited supernodes (once per
// call, all lanes busy, instead of a division per block in the solves); a
// diagonal entry that is not positive and finite sets status bit 0.
__device__ void gather_x(const IPtrs &P, const ISub &sd, const double *__restrict__ Lv,
                         const double *__restrict__ lam, double *x, int gt, int nt, const Group &g,
                         uint32_t *status) {
  for (int c = gt; c < sd.n; c += nt) x[c] = 0.0;
  double *rd = x + P.rd_off;
  // one supernode per thread up to 32 columns (independent loads side by side), a warp per larger one
  for (int s = sd.sn_lo + gt; s < sd.sn_hi; s += nt) {
    const ISn sn = P.sns[s];
    if (sn.ns > 32) continue;
    const int nr = sn.ns + sn.rs;
    int o = 0;
    for (int t = 0; t < sn.ns; ++t) {
      bool ok;
      const double r = pos_recip(Lv[sn.lval + o], ok);
      if (!ok) atomicOr(status, 1u);
      rd[sn.c0 + t] = ok ? r : 0.0;
      o += nr - t;
    }
  }
  for (int s = sd.sn_lo + gt / 32; s < sd.sn_hi; s += nt / 32) {
    const ISn sn = P.sns[s];
    if (sn.ns <= 32) continue;
    const int nr = sn.ns + sn.rs;
    for (int t = gt & 31; t < sn.ns; t += 32) {
      bool ok;
      const double r = pos_recip(Lv[sn.lval + col_off(t, nr)], ok);
      if (!ok) atomicOr(status, 1u);
      rd[sn.c0 + t] = ok ? r : 0.0;
    }
  }
  g.sync();
  for (int r = sd.g_lo + gt; r < sd.g_hi; r += nt) {
    const IRow row = P.grow[r];
    double v = 0.0;
    for (int e = row.e_lo; e < row.e_hi; ++e) v += P.gent[e].sign * lam[P.gent[e].gj];
    x[row.r] = v;
  }
}

template <bool CL>
__device__ void scatter_q(const IPtrs &P, int e_lo, int e_hi, const double *x, double *q, int gt, int nt) {
  for (int e = e_lo + gt; e < e_hi; e += nt) {
    const ISEnt t = P.sent[e];
    atomicAdd(q + t.gj, t.sign * ldx<CL>(x + t.r));
  }
}

// The whole implicit application for one subdomain by one group (the
// cluster, or one CTA).
template <bool CL>
__device__ void solve_subdomain(const Group &g, const IPtrs &P, const ISub &sd, const double *__restrict__ Lv,
                                const double *__restrict__ lam, double *q, double *X, uint32_t *status,
                                double (*ys)[32], double *red, double *red_cta, int *ctr) {
  const int tid = g.warp * 32 + g.lane;
  const int gt = g.rank * (int)blockDim.x + tid, nt = g.size * (int)blockDim.x;
  double *x = X + sd.x_off;
  gather_x(P, sd, Lv, lam, x, gt, nt, g, status);
  g.sync();
  int base = 0;
  forward_levels<CL>(g, P, sd.lev_lo, sd.n_lev, Lv, x, ys, ctr, base);
  backward_levels<CL>(g, P, sd.lev_lo, sd.n_lev, Lv, x, red, red_cta, ctr, base);
  scatter_q<CL>(P, sd.s_lo, sd.s_hi, x, q, gt, nt);
}

// Item kind 2: subdomain sub[j] on the CTA pair (2j, 2j + 1) of a cluster;
// CTA 2j + part solves subtree part (0: A, 1: B), the first CTA of the pair
// also the top chain.  Every CTA of the cluster passes the same three
// cluster barriers:
//   S1 after the first CTA's gather of x = B^T lambda (the second CTA reads
//      its rows afterwards, first touch of those lines on its SM);
//   S2 after both subtrees' forward solves (their updates of the top rows
//      are atomic in L2) -- then the first CTA solves the top forward and
//      backward, reading x past L1;
//   S3 after the top -- then each CTA solves its subtree backward (ancestor
//      rows of the top read past L1) and scatters its own rows.
// The subtrees share no rows, so between the barriers each CTA only reads
// rows that it or its own warps wrote, or that were complete at a barrier.
__device__ void solve_pair_item(const IItem &it, const IPtrs &P, const double *__restrict__ Lv,
                                const double *__restrict__ lam, double *q, double *X, uint32_t *status,
                                double (*ys)[32], double *red, double *red_cta, int *ctr, int warp, int lane) {
  cg::cluster_group cl = cg::this_cluster();
  const int r = (int)cl.block_rank(), j = r >> 1, part = r & 1;
  const bool act = j < it.n;
  const Group cta = cta_group(warp, lane);
  const int tid = warp * 32 + lane;
  ISub sd{};
  if (act) sd = P.subs[it.sub[j]];
  double *x = X + sd.x_off;
  const int lev_part = part == 0 ? sd.lev_lo : sd.lev_lo + sd.n_lev_a;
  const int n_part = part == 0 ? sd.n_lev_a : sd.n_lev_b;
  const int lev_top = sd.lev_lo + sd.n_lev_a + sd.n_lev_b, n_top = sd.n_lev - sd.n_lev_a - sd.n_lev_b;
  if (act && part == 0) gather_x(P, sd, Lv, lam, x, tid, (int)blockDim.x, cta, status);
  cl.sync();                                                             // S1
  int base = 0;
  if (act) forward_levels<false>(cta, P, lev_part, n_part, Lv, x, ys, ctr, base);
  cl.sync();                                                             // S2
  if (act && part == 0) {
    forward_levels<true>(cta, P, lev_top, n_top, Lv, x, ys, ctr, base);
    backward_levels<true>(cta, P, lev_top, n_top, Lv, x, red, red_cta, ctr, base);
    scatter_q<true>(P, sd.s_mid2, sd.s_hi, x, q, tid, (int)blockDim.x);
  }
  cl.sync();                                                             // S3
  if (act) {
    backward_levels<true>(cta, P, lev_part, n_part, Lv, x, red, red_cta, ctr, base);
    if (part == 0) scatter_q<true>(P, sd.s_lo, sd.s_mid1, x, q, tid, (int)blockDim.x);
    else scatter_q<true>(P, sd.s_mid1, sd.s_mid2, x, q, tid, (int)blockDim.x);
  }
}

// Launched in clusters of kCluster CTAs.  An item is one large subdomain
// solved by the whole cluster, up to kCluster small subdomains (one per
// CTA), or up to kCluster / 2 subdomains on CTA pairs.
__global__ void __launch_bounds__(kThreadsI, 1) implicit_kernel(const IPtrs P, const double *__restrict__ Lv,
                                                                const double *__restrict__ lam, double *q,
                                                                double *X, uint32_t *status) {
  __shared__ double ys[kWarps][32];
  __shared__ double red[kWarps * 32];
  __shared__ double red_cta[kWarps * 32];          // one 32-double row per (sub)group
  __shared__ int take_ctr;                          // supernodes taken (see take); zero before the first barrier
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) take_ctr = 0;
  const IItem it = P.items[blockIdx.x / kCluster];
  if (it.kind == 0) {
    const Group g = cluster_group(warp, lane);
    solve_subdomain<true>(g, P, P.subs[it.sub[0]], Lv, lam, q, X, status, ys, red, red_cta, nullptr);
    cg::this_cluster().sync();   // no CTA leaves while the first one may read its shared memory
  } else if (it.kind == 2) {
    solve_pair_item(it, P, Lv, lam, q, X, status, ys, red, red_cta, &take_ctr, warp, lane);
  } else {
    const int r = (int)(blockIdx.x % kCluster);   // also without a cluster launch
    if (r < it.n) {
      const Group g = cta_group(warp, lane);
      solve_subdomain<false>(g, P, P.subs[it.sub[r]], Lv, lam, q, X, status, ys, red, red_cta, &take_ctr);
    }
  }
}

}  // namespace

struct sci_ctx {
  std::string err;
  int32_t nsub = 0;
  int64_t n_dual = 0;
  std::vector<uint8_t> blob;
  IHeader hdr{};
  sci_sizes sizes{};
  void *plan_dev = nullptr;
  size_t plan_dev_bytes = 0;
  int64_t n_items = 0;
  int64_t n_pair_subdomains = 0;    // subdomains on CTA pairs (the launch then needs clusters)
  int64_t x_total = 0;              // doubles of all subdomains' x (the reciprocal diagonals follow)
  int32_t warps = kWarps;           // warps per CTA of the launch

  IPtrs ptrs() const {
    const uint8_t *b = static_cast<const uint8_t *>(plan_dev);
    IPtrs p;
    p.subs = reinterpret_cast<const ISub *>(b + hdr.sec_off[0]);
    p.sns = reinterpret_cast<const ISn *>(b + hdr.sec_off[1]);
    p.levptr = reinterpret_cast<const int32_t *>(b + hdr.sec_off[2]);
    p.rows = reinterpret_cast<const int32_t *>(b + hdr.sec_off[3]);
    p.grow = reinterpret_cast<const IRow *>(b + hdr.sec_off[4]);
    p.gent = reinterpret_cast<const IEnt *>(b + hdr.sec_off[5]);
    p.sent = reinterpret_cast<const ISEnt *>(b + hdr.sec_off[6]);
    p.items = reinterpret_cast<const IItem *>(b + hdr.sec_off[7]);
    p.rd_off = x_total;
    return p;
  }
};

namespace {

template <class V>
size_t put_section(std::vector<uint8_t> &blob, const std::vector<V> &v) {
  const size_t off = (blob.size() + 255) & ~size_t(255);
  blob.resize(off + v.size() * sizeof(V));
  if (!v.empty()) std::memcpy(blob.data() + off, v.data(), v.size() * sizeof(V));
  return off;
}

sc_status ifail(sci_ctx *c, sc_status st, const std::string &m) {
  if (c) c->err = m;
  return st;
}

// The two parts of a subdomain's visited etree forest for a CTA pair.  From
// the roots down: the current set of subtrees is dealt, largest first, to the
// lighter of two parts; if the lighter one gets at least a fifth of the set's
// work, those are the parts.  Otherwise the largest subtree's root and the
// other (small) subtrees go to the top -- a regularised fixed dof, for one,
// is a one-column tree of its own -- and the search goes on in the largest
// subtree's children.  part[s] = 0 / 1 / 2 (top); false if no split is found.
bool split_tree(const sc::SubPlan &S, const std::vector<int32_t> &vis, std::vector<int8_t> &part) {
  const int32_t nsn = (int32_t)S.sn_c0.size();
  std::vector<std::vector<int32_t>> ch(nsn);
  std::vector<int32_t> roots;
  std::vector<int64_t> w(nsn, 0);
  for (int32_t s : vis) {                       // vis: children before parents
    w[s] += (int64_t)S.sn_ns[s] * (S.sn_ns[s] + 1) / 2 + (int64_t)S.sn_ns[s] * S.sn_rs[s];
    if (S.sparent[s] >= 0) {
      ch[S.sparent[s]].push_back(s);
      w[S.sparent[s]] += w[s];
    } else {
      roots.push_back(s);
    }
  }
  part.assign(nsn, 2);
  std::vector<int32_t> cur = roots;
  while (!cur.empty()) {
    std::stable_sort(cur.begin(), cur.end(), [&](int32_t a, int32_t b) { return w[a] > w[b]; });
    int64_t load[2] = {0, 0};
    std::vector<int8_t> side(cur.size());
    for (size_t k = 0; k < cur.size(); ++k) {
      side[k] = load[0] <= load[1] ? 0 : 1;
      load[side[k]] += w[cur[k]];
    }
    if (cur.size() >= 2 && 5 * std::min(load[0], load[1]) >= load[0] + load[1]) {
      std::vector<int32_t> stack;
      for (size_t k = 0; k < cur.size(); ++k) {
        stack.assign(1, cur[k]);
        while (!stack.empty()) {
          const int32_t v = stack.back();
          stack.pop_back();
          part[v] = side[k];
          for (int32_t u : ch[v]) stack.push_back(u);
        }
      }
      return true;
    }
    cur = ch[cur[0]];                             // the rest of this set stays in the top
  }
  return false;
}

sc_status build(sci_ctx *ctx, int32_t nsub, const sc_subdomain_desc *d, int64_t cluster_min_work,
                int32_t pairs) {
  for (int32_t i = 0; i < nsub; ++i)
    if (d[i].Bt_val)
      return ifail(ctx, SC_ERR_INVALID_ARG, "subdomain " + std::to_string(i) + ": sci_plan takes signed-Boolean B^T (Bt_val must be NULL)");
  std::vector<ISub> subs;
  std::vector<ISn> sns;
  std::vector<int32_t> levptr, rows;
  std::vector<IRow> grow;
  std::vector<IEnt> gent;
  std::vector<ISEnt> sent;
  // subdomains largest first (CTA order), by visited entries of L
  std::vector<sc::SubPlan> P(nsub);
  std::vector<int64_t> work(nsub, 0), L_off(nsub + 1, 0), x_off(nsub + 1, 0);
  int64_t max_lev = 0, nnz_all = 0, m_all = 0;
  for (int32_t i = 0; i < nsub; ++i) {
    const std::string e = sc::analyze(i, d[i], P[i]);
    if (!e.empty()) return ifail(ctx, SC_ERR_INVALID_ARG, e);
    if (d[i].m > 0 && !d[i].lambda_map)
      return ifail(ctx, SC_ERR_INVALID_ARG, "subdomain " + std::to_string(i) + ": lambda_map is NULL");
    for (int32_t j = 0; j < d[i].m; ++j)
      if (d[i].lambda_map[j] < 0 || d[i].lambda_map[j] >= ctx->n_dual)
        return ifail(ctx, SC_ERR_INVALID_ARG, "subdomain " + std::to_string(i) + ": lambda_map out of range");
    L_off[i + 1] = L_off[i] + (d[i].n > 0 ? d[i].L_colptr[d[i].n] : 0);
    x_off[i + 1] = x_off[i] + d[i].n;
    const sc::SubPlan &S = P[i];
    for (size_t s = 0; s < S.sn_c0.size(); ++s)
      if (S.sn_jhi[s] > S.sn_jlo[s])
        work[i] += (int64_t)S.sn_ns[s] * (S.sn_ns[s] + 1) / 2 + (int64_t)S.sn_ns[s] * S.sn_rs[s];
    nnz_all += work[i];
    m_all += d[i].m;
  }
  std::vector<int32_t> order(nsub);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return work[a] > work[b]; });
  if (cluster_min_work < 0)
    cluster_min_work = std::max<int64_t>(1, 2 * nnz_all / std::max<int64_t>(1, std::min<int64_t>(kCtaSlots, nsub)) + 1);
  // CTA pairs only on request: measured on GB300 (config 2, 64 subdomains on
  // 152 SMs) a pair took 2.51 ms against 2.20 ms for one CTA per subdomain --
  // the subtrees are not the critical path, the per-level chains are
  const bool want_pairs = pairs == 1;
  std::vector<int8_t> is_pair(nsub, 0);
  for (int32_t i : order) {
    const sc::SubPlan &S = P[i];
    const sc_subdomain_desc &D = d[i];
    const int32_t nsn = (int32_t)S.sn_c0.size();
    std::vector<int32_t> h(nsn, 0), vis;
    for (int32_t s = 0; s < nsn; ++s) {
      if (S.sn_jhi[s] <= S.sn_jlo[s]) continue;
      vis.push_back(s);
      if (S.sparent[s] >= 0) h[S.sparent[s]] = std::max(h[S.sparent[s]], h[s] + 1);
    }
    std::vector<int8_t> part;
    const bool pair = want_pairs && work[i] < cluster_min_work && split_tree(S, vis, part);
    if (!pair) part.assign(nsn, 2);
    is_pair[i] = pair;
    // (part, level, work descending): parts A, B, then the top, one level
    // sequence each; within a level the largest supernodes first, so that the
    // warps taking them in turn finish the level together
    auto snw = [&](int32_t s) { return (int64_t)S.sn_ns[s] * (S.sn_ns[s] + 1) / 2 + (int64_t)S.sn_ns[s] * S.sn_rs[s]; };
    std::stable_sort(vis.begin(), vis.end(), [&](int32_t a, int32_t b) {
      if (part[a] != part[b]) return part[a] < part[b];
      if (h[a] != h[b]) return h[a] < h[b];
      return snw(a) > snw(b);
    });
    ISub sd{};
    sd.x_off = x_off[i];
    sd.n = D.n;
    sd.sn_lo = (int32_t)sns.size();
    sd.lev_lo = (int32_t)levptr.size();
    int32_t cur_part = -1, cur_h = -1, nlev = 0, nlev_part[3] = {0, 0, 0};
    for (int32_t s : vis) {
      if (part[s] != cur_part || h[s] != cur_h) {   // a new level (heights are increasing within a part)
        levptr.push_back((int32_t)sns.size());
        cur_part = part[s];
        cur_h = h[s];
        ++nlev;
        ++nlev_part[cur_part];
      }
      ISn sn{};
      const int32_t c0 = S.sn_c0[s], ns = S.sn_ns[s], rs = S.sn_rs[s];
      // the kernel addresses a panel with 32-bit offsets
      if ((int64_t)ns * (ns + rs) - (int64_t)ns * (ns - 1) / 2 >= (int64_t(1) << 31))
        return ifail(ctx, SC_ERR_INVALID_ARG, "subdomain " + std::to_string(i) +
                                                  ": a supernode panel of 2^31 or more entries (sci_plan addresses panels in 32 bits)");
      sn.lval = L_off[i] + D.L_colptr[c0];
      sn.rows_off = (int64_t)rows.size();
      sn.c0 = c0;
      sn.ns = ns;
      sn.rs = rs;
      sn.sub = i;
      const int64_t last = D.L_colptr[c0 + ns - 1];
      for (int32_t k = 0; k < rs; ++k) rows.push_back(D.L_rowind[last + 1 + k]);
      sns.push_back(sn);
    }
    sd.sn_hi = (int32_t)sns.size();
    sd.n_lev = nlev;
    sd.n_lev_a = nlev_part[0];
    sd.n_lev_b = nlev_part[1];
    levptr.push_back(sd.sn_hi);
    max_lev = std::max<int64_t>(max_lev, sd.n_lev);
    // B^T by row (gather) and by entry (scatter)
    std::vector<std::pair<int32_t, int32_t>> ent;   // (row, entry index)
    std::vector<ISEnt> by_part[3];                    // scatter entries by the part of their row
    for (int32_t j = 0; j < D.m; ++j)
      for (int32_t e = D.Bt_colptr[j]; e < D.Bt_colptr[j + 1]; ++e) {
        ent.emplace_back(D.Bt_rowind[e], e);
        const int32_t r = D.Bt_rowind[e];
        by_part[part[S.snode_of[r]]].push_back(ISEnt{r, D.lambda_map[j], (int32_t)D.Bt_sign[e], 0});
      }
    sd.s_lo = (int32_t)sent.size();
    sent.insert(sent.end(), by_part[0].begin(), by_part[0].end());
    sd.s_mid1 = (int32_t)sent.size();
    sent.insert(sent.end(), by_part[1].begin(), by_part[1].end());
    sd.s_mid2 = (int32_t)sent.size();
    sent.insert(sent.end(), by_part[2].begin(), by_part[2].end());
    std::vector<int32_t> col_of(ent.size());
    for (int32_t j = 0; j < D.m; ++j)
      for (int32_t e = D.Bt_colptr[j]; e < D.Bt_colptr[j + 1]; ++e) col_of[e] = j;
    std::stable_sort(ent.begin(), ent.end());
    sd.g_lo = (int32_t)grow.size();
    for (size_t a = 0; a < ent.size();) {
      size_t b = a;
      IRow r{ent[a].first, (int32_t)gent.size(), 0, 0};
      while (b < ent.size() && ent[b].first == ent[a].first) {
        const int32_t e = ent[b].second;
        gent.push_back(IEnt{D.lambda_map[col_of[e]], (int32_t)D.Bt_sign[e]});
        ++b;
      }
      r.e_hi = (int32_t)gent.size();
      grow.push_back(r);
      a = b;
    }
    sd.g_hi = (int32_t)grow.size();
    sd.s_hi = (int32_t)sent.size();
    subs.push_back(sd);
  }
  // items: subdomains with at least cluster_min_work visited entries get a
  // cluster each; the rest are packed kCluster to a cluster, one per CTA
  // (subs is largest first, so packed neighbours have similar work)
  // automatic: a cluster for a subdomain with more than twice an even share
  // of the CTAs the batch can occupy (measured on GB300: clusters shorten a
  // heavy tail of a few large subdomains, but cost more than they give on a
  // batch of similar ones)
  // pairs: kCluster / 2 subdomains to a cluster, one per CTA pair
  std::vector<IItem> items;
  for (int32_t k = 0; k < nsub;) {
    IItem it{};
    if (work[order[k]] >= cluster_min_work) {
      it.kind = 0;
      it.n = 1;
      it.sub[0] = k++;
    } else if (is_pair[order[k]]) {
      it.kind = 2;
      while (it.n < kCluster / 2 && k < nsub && is_pair[order[k]] && work[order[k]] < cluster_min_work)
        it.sub[it.n++] = k++;
    } else {
      it.kind = 1;
      while (it.n < kCluster && k < nsub && !is_pair[order[k]] && work[order[k]] < cluster_min_work)
        it.sub[it.n++] = k++;
    }
    items.push_back(it);
  }
  ctx->n_items = (int64_t)items.size();
  // 16 warps and one CTA per SM while the batch has at most one subdomain per
  // SM (a subdomain alone on its SM gets twice the warps for its wide lower
  // levels); 8 warps and two CTAs per SM beyond, so that twice as many
  // subdomains run at once
  ctx->warps = nsub <= kCtaSlots ? kWarps : kWarps / 2;
  int64_t n_big = 0;
  ctx->n_pair_subdomains = 0;
  for (const IItem &it : items) {
    n_big += it.kind == 0;
    if (it.kind == 2) ctx->n_pair_subdomains += it.n;
  }
  IHeader &H = ctx->hdr;
  H = IHeader{};
  H.magic = 0x50494353u;   // "SCIP"
  H.version = 2;
  H.nsub = nsub;
  H.n_sn = (int64_t)sns.size();
  H.n_levptr = (int64_t)levptr.size();
  H.n_rows = (int64_t)rows.size();
  H.n_grow = (int64_t)grow.size();
  H.n_gent = (int64_t)gent.size();
  H.n_sent = (int64_t)sent.size();
  H.n_items = (int64_t)items.size();
  std::vector<uint8_t> &blob = ctx->blob;
  blob.assign(kIHeaderBytes, 0);
  H.sec_off[0] = put_section(blob, subs);
  H.sec_off[1] = put_section(blob, sns);
  H.sec_off[2] = put_section(blob, levptr);
  H.sec_off[3] = put_section(blob, rows);
  H.sec_off[4] = put_section(blob, grow);
  H.sec_off[5] = put_section(blob, gent);
  H.sec_off[6] = put_section(blob, sent);
  H.sec_off[7] = put_section(blob, items);
  blob.resize((blob.size() + 255) & ~size_t(255));
  std::memcpy(blob.data(), &H, sizeof(H));
  sci_sizes &z = ctx->sizes;
  z.plan_bytes = blob.size();
  // status word, every subdomain's x, then its reciprocal diagonals at the same offsets
  ctx->x_total = x_off[nsub];
  z.ws_bytes = 256 + 2 * sizeof(double) * (size_t)x_off[nsub];
  z.L_values = L_off[nsub];
  z.n_supernodes = (int64_t)sns.size();
  z.nnz_visited = nnz_all;
  z.max_levels = max_lev;
  z.flops = 4.0 * (double)nnz_all;
  z.n_cluster_subdomains = n_big;
  z.bytes = 16.0 * (double)nnz_all + 16.0 * (double)m_all;
  return SC_OK;
}

}  // namespace

extern "C" {

sc_status sci_plan(sci_ctx **out, int32_t nsub, const sc_subdomain_desc *subdomains, int64_t n_dual,
                   const sci_options *opt) {
  if (!out) return SC_ERR_INVALID_ARG;
  *out = nullptr;
  sci_ctx *ctx = new (std::nothrow) sci_ctx();
  if (!ctx) return SC_ERR_OOM;
  *out = ctx;
  if (nsub < 0 || (nsub > 0 && !subdomains) || n_dual < 0)
    return ifail(ctx, SC_ERR_INVALID_ARG, "nsub < 0, n_dual < 0 or subdomains NULL");
  ctx->nsub = nsub;
  ctx->n_dual = n_dual;
  try {
    if (opt && (opt->pairs < -1 || opt->pairs > 1)) return ifail(ctx, SC_ERR_INVALID_ARG, "pairs must be -1, 0 or 1");
    return build(ctx, nsub, subdomains, opt ? opt->cluster_min_work : -1, opt ? opt->pairs : 0);
  } catch (const std::bad_alloc &) {
    return ifail(ctx, SC_ERR_OOM, "host allocation failed while planning");
  } catch (...) {
    return ifail(ctx, SC_ERR_INTERNAL, "unexpected exception while planning");
  }
}

sc_status sci_get_sizes(const sci_ctx *ctx, sci_sizes *s) {
  if (!ctx || !s) return SC_ERR_INVALID_ARG;
  *s = ctx->sizes;
  return SC_OK;
}

sc_status sci_upload_plan(sci_ctx *ctx, void *plan_dev, size_t bytes, void *stream) {
  if (!ctx) return SC_ERR_INVALID_ARG;
  if (!plan_dev || bytes < ctx->blob.size()) return ifail(ctx, SC_ERR_INVALID_ARG, "plan buffer NULL or too small");
  if (reinterpret_cast<uintptr_t>(plan_dev) % 256) return ifail(ctx, SC_ERR_INVALID_ARG, "plan buffer not 256-byte aligned");
  cudaError_t e = cudaMemcpyAsync(plan_dev, ctx->blob.data(), ctx->blob.size(), cudaMemcpyHostToDevice,
                      static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return ifail(ctx, SC_ERR_CUDA, std::string("plan upload: ") + cudaGetErrorString(e));
  // the host blob must stay alive until the asynchronous copy has read it
  const cudaError_t e2 = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e2 != cudaSuccess) return ifail(ctx, SC_ERR_CUDA, std::string("plan upload: ") + cudaGetErrorString(e2));
  ctx->plan_dev = plan_dev;
  ctx->plan_dev_bytes = bytes;
  return SC_OK;
}

sc_status sci_apply(sci_ctx *ctx, const double *L_values_dev, const double *lambda_dev, double *q_dev, void *ws_dev,
                    size_t ws_bytes, void *stream) {
  if (!ctx) return SC_ERR_INVALID_ARG;
  if (!ctx->plan_dev) return ifail(ctx, SC_ERR_STATE, "sci_upload_plan was not called");
  if (ctx->n_dual > 0 && (!lambda_dev || !q_dev)) return ifail(ctx, SC_ERR_INVALID_ARG, "lambda or q is NULL");
  if (ctx->sizes.L_values > 0 && !L_values_dev) return ifail(ctx, SC_ERR_INVALID_ARG, "L_values_dev is NULL");
  if (!ws_dev || ws_bytes < ctx->sizes.ws_bytes) return ifail(ctx, SC_ERR_OOM, "workspace NULL or too small");
  if (reinterpret_cast<uintptr_t>(ws_dev) % 256) return ifail(ctx, SC_ERR_INVALID_ARG, "workspace not 256-byte aligned");
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint32_t *status = static_cast<uint32_t *>(ws_dev);
  double *X = reinterpret_cast<double *>(static_cast<uint8_t *>(ws_dev) + 256);
  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(uint32_t), st);
  if (e == cudaSuccess && ctx->n_dual > 0) e = cudaMemsetAsync(q_dev, 0, sizeof(double) * (size_t)ctx->n_dual, st);
  if (e == cudaSuccess && ctx->n_items > 0) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(ctx->n_items * kCluster));
    cfg.blockDim = dim3(32 * ctx->warps);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kCluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    // no cluster when no item needs one (pair items synchronise their cluster)
    cfg.numAttrs = ctx->sizes.n_cluster_subdomains > 0 || ctx->n_pair_subdomains > 0 ? 1 : 0;
    e = cudaLaunchKernelEx(&cfg, implicit_kernel, ctx->ptrs(), L_values_dev, lambda_dev, q_dev, X, status);
  }
  if (e != cudaSuccess) return ifail(ctx, SC_ERR_CUDA, std::string("sci_apply: ") + cudaGetErrorString(e));
  return SC_OK;
}

sc_status sci_device_status(sci_ctx *ctx, const void *ws_dev, void *stream) {
  if (!ctx || !ws_dev) return SC_ERR_INVALID_ARG;
  uint32_t h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, ws_dev, sizeof(h), cudaMemcpyDeviceToHost, static_cast<cudaStream_t>(stream));
  if (e == cudaSuccess) e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return ifail(ctx, SC_ERR_CUDA, std::string("status read: ") + cudaGetErrorString(e));
  if (h & 1u) return ifail(ctx, SC_ERR_NOT_SPD, "a diagonal entry of L is not positive and finite");
  return h ? ifail(ctx, SC_ERR_INTERNAL, "unknown device status bits") : SC_OK;
}

sc_status sci_export_plan(const sci_ctx *ctx, void *dst, size_t bytes) {
  if (!ctx || !dst || bytes < ctx->blob.size()) return SC_ERR_INVALID_ARG;
  std::memcpy(dst, ctx->blob.data(), ctx->blob.size());
  return SC_OK;
}

const char *sci_last_error(const sci_ctx *ctx) { return ctx ? ctx->err.c_str() : "NULL context"; }

void sci_destroy(sci_ctx *ctx) { delete ctx; }

}  // extern "C"
