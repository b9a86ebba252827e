/* sc_implicit.h -- implicit application of the FETI dual operator on the GPU.
 *
 * Paper Sec. 2.2, Eq. "dualop_apply_impl": instead of multiplying by the
 * assembled F_i, each application runs, per subdomain,
 *
 *     x = P B_i^T lambda_i        (sparse gather of the dual vector)
 *     y = L_i^{-1} x              (sparse forward triangular solve)
 *     z = L_i^{-T} y              (sparse backward triangular solve)
 *     q += B_i P^T z              (sparse scatter into the dual vector)
 *
 * so that q = sum_i F_i lambda_i with F_i = B_i K_i^+ B_i^T, the same result as
 * sc_apply on the assembled F (Eq. "dualop_apply_expl").  The paper states the
 * trade-off this measures: the explicit product is faster per iteration, the
 * assembly pays off only after enough iterations (the amortisation point,
 * Sec. 2.2).  This is the GPU form of the implicit side of that comparison.
 *
 * Work: only the supernodes of L on the elimination-tree paths from B_i^T's
 * rows to the root are visited (the forward solve's right-hand side is zero
 * elsewhere, and the backward solve is read only at B_i^T's rows, which depend
 * on their ancestors alone).  A subdomain is solved by one CTA or, when large,
 * by a cluster of 8 CTAs; the supernodes of one etree level are solved
 * concurrently by the group's warps, 32-column blocks at a time (warp-level
 * diagonal-block solve, coalesced panel updates), and the few large
 * separators at the top of the tree by the whole group.
 *
 * Inputs: the same subdomain descriptors as sc_plan (include/sc.h: CSC L
 * pattern of P K_reg P^T with the diagonal first in each column, B^T's
 * pattern and signs in L's ordering, lambda_map) and, per call, the
 * concatenated CSC values of every L_i in subdomain order (the array
 * sc_assemble_batch takes).  lambda_map is required (non-NULL when m > 0).
 *
 * Memory: the caller owns every device buffer (plan tables, workspace,
 * L values, lambda, q).  The workspace holds a status word and one n_i-vector
 * per subdomain; it is temporary.  Streams as in sc.h (cudaStream_t as void*,
 * NULL = legacy default stream); device calls are asynchronous.
 *
 * Precision: FP64 throughout.  q is accumulated with FP64 atomic additions
 * (several subdomains share a multiplier), and so is the forward solve's
 * update of ancestor rows, so the last bits of q may differ from run to run.
 *
 * Errors: sc_status codes of sc.h.  A diagonal entry of L that is not
 * positive and finite sets bit 0 of the workspace's status word (read by
 * sci_device_status); q is then undefined. */
#ifndef SC_IMPLICIT_H
#define SC_IMPLICIT_H

#include <stddef.h>
#include <stdint.h>

#include "sc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sci_ctx sci_ctx;

typedef struct {
  size_t plan_bytes;        /* device plan tables (sci_upload_plan) */
  size_t ws_bytes;          /* device workspace of sci_apply */
  int64_t L_values;         /* doubles of the concatenated L values */
  int64_t n_supernodes;     /* supernodes visited (on the paths from B^T's rows to the root) */
  int64_t nnz_visited;      /* entries of L in those supernodes */
  int64_t max_levels;       /* deepest etree (in visited supernodes) of any subdomain */
  double flops;             /* 4 nnz_visited: one multiply-add per entry in each solve */
  double bytes;             /* algorithmic bytes: L entries read twice (16 nnz_visited) + 16 m */
  int64_t n_cluster_subdomains; /* subdomains solved by a whole 8-CTA cluster */
} sci_sizes;

/* cluster_min_work: subdomains with at least this many visited entries of L
 * are solved by a thread-block cluster of 8 CTAs (8 SMs' FP64 pipes; cluster
 * barriers between levels, distributed shared memory for the reductions),
 * the others by one CTA each (packed 8 to a cluster).  -1 (or a NULL options
 * pointer) selects more than 2 x (visited entries of the batch) /
 * min(304, nsub): twice an even share of the CTAs the batch can occupy (a
 * GB300 keeps 304 resident).  Clusters shorten a heavy tail of a few large
 * subdomains; on a batch of similar subdomains they cost more (cluster
 * barriers, L1-bypassing reads of x) than they give.  0 puts every subdomain
 * on a cluster. */
/* pairs: 1 solves each subdomain below cluster_min_work whose visited etree
 * splits on a pair of CTAs: the subtrees below the first node with two or
 * more substantial visited subtrees are dealt to the two CTAs (about half the
 * work each), which solve them at the same time; the chain above runs on the
 * first CTA; three cluster barriers per call.  0 (automatic) and -1: one CTA
 * per subdomain (on GB300 the pair form measured slower on the 64-subdomain
 * heat batch: the per-level chains, not the subtrees, bound the solve).
 * reserved: 0. */
typedef struct {
  int64_t cluster_min_work;
  int32_t pairs;
  int32_t reserved;
} sci_options;

/* Symbolic stage (host only): validates the patterns (the rules of sc_plan)
 * and builds the level schedule.  n_dual bounds lambda_map's values; options
 * may be NULL.  On failure *out may hold a context whose sci_last_error
 * explains; destroy it. */
sc_status sci_plan(sci_ctx **out, int32_t nsub, const sc_subdomain_desc *subdomains, int64_t n_dual,
                   const sci_options *options);

sc_status sci_get_sizes(const sci_ctx *ctx, sci_sizes *sizes);

/* Copies the plan tables into plan_dev (bytes >= plan_bytes, 256-byte
 * aligned device memory owned by the caller, kept until the last sci_apply). */
sc_status sci_upload_plan(sci_ctx *ctx, void *plan_dev, size_t bytes, void *stream);

/* q (n_dual doubles, overwritten) = sum_i B_i K_i^+ B_i^T lambda_i.
 * L_values_dev: concatenated CSC values; ws_dev: ws_bytes of workspace. */
sc_status sci_apply(sci_ctx *ctx, const double *L_values_dev, const double *lambda_dev, double *q_dev,
                    void *ws_dev, size_t ws_bytes, void *stream);

/* Synchronises `stream` and reads the status word of ws_dev: SC_OK or SC_ERR_NOT_SPD. */
sc_status sci_device_status(sci_ctx *ctx, const void *ws_dev, void *stream);

/* Host copy of the plan tables (bytes >= plan_bytes), for inspection.  Layout:
 * a 256-byte header {uint32 magic 'SCIP', uint32 version 1, int32 nsub, pad,
 * int64 n_sn, n_levptr, n_rows, n_grow, n_gent, n_sent, n_items,
 * uint64 sec_off[8]} and eight 256-byte aligned sections: subdomains (48 B each, largest first:
 * int64 x_off; int32 n, sn_lo, sn_hi, lev_lo, n_lev, g_lo, g_hi, s_lo, s_hi,
 * pad), supernodes (32 B: int64 lval, rows_off; int32 c0, ns, rs, sub),
 * level boundaries (int32), pruned rows (int32), gather rows (int32 r, e_lo,
 * e_hi, pad), gather entries (int32 gj, sign), scatter entries (int32 r, gj,
 * sign, pad), cluster items (int32 kind, n, sub[8]; kind 0: sub[0] on the
 * whole cluster, kind 1: sub[r] on CTA r for r < n). */
sc_status sci_export_plan(const sci_ctx *ctx, void *dst, size_t bytes);

const char *sci_last_error(const sci_ctx *ctx);
void sci_destroy(sci_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* SC_IMPLICIT_H */
