/* sc.h -- GPU assembly and application of FETI local dual operators
 *         (dense Schur complements) on GB300 (sm_103a), C ABI.
 *
 * What is computed (paper Sec. 2.1-2.2, Eq. "localdualoperator",
 * Eq. "localdualoperatorwithU"; Sec. 3.1, the Y^T Y form):
 *
 *     F_i = B_i K_i^+ B_i^T = B_i L_i^{-T} L_i^{-1} B_i^T = Y_i^T Y_i,
 *     Y_i = L_i^{-1} B_i^T,
 *
 * for every subdomain i of a batch, from the sparse Cholesky factor L_i of the
 * regularised subdomain matrix (already permuted by the fill-reducing
 * ordering P, so B_i^T's rows are given in L_i's ordering; paper Sec. 3), and
 * the explicit application q = sum_i B_i^T-scatter(F_i lambda_i)
 * (Eq. "dualop_apply_expl").
 *
 * Method (paper Sec. 3.2-3.3): the columns of B_i^T are sorted by their column
 * pivot (first nonzero in L's ordering; with an etree-postordered L this is
 * the paper's "stepped" shape), the forward substitution skips the zero rows
 * above the pivots and the structurally zero blocks of L ("factor splitting"
 * with "pruning" of empty rows), and the SYRK Y^T Y forms only the blocks of
 * the lower triangle whose inputs are structurally nonzero ("input splitting").
 * Here the blocks are the supernodes of L and the column range of Y that is
 * nonzero on each supernode.  Finally F is permuted back to B_i^T's original
 * column order (paper Sec. 3, end of the preamble).
 *
 * Stages (paper Sec. 2.2, the three solver stages):
 *   initialization -- sc_plan (host, symbolic only: patterns, never values),
 *                     sc_get_sizes, sc_upload_plan (plan tables to the GPU);
 *   preprocessing  -- sc_assemble_batch (numeric: new L values, same patterns);
 *   solution       -- sc_apply once per iteration of the dual solver.
 *
 * Memory: the caller owns every device buffer (plan tables, workspace, L
 * values, F, lambda, q).  F is persistent; the workspace is temporary and may
 * be reused by anything else between calls (paper Sec. 3.1, persistent vs
 * temporary memory).  The library itself allocates host memory only.
 *
 * Streams: every device call takes a cudaStream_t passed as void*; NULL is the
 * legacy default stream.  Calls are asynchronous unless stated otherwise.
 *
 * Errors: every call returns an sc_status; nothing is thrown across the ABI.
 * The message of the last failing call on a context is sc_last_error(ctx).
 * Device-side failures (non-positive or non-finite diagonal of L) are recorded
 * in the workspace's status word and reported by sc_device_status; F is then
 * undefined.
 *
 * Precision: FP64 throughout (IEEE binary64 multiply-add, round to nearest).
 */
#ifndef SC_H
#define SC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sc_ctx sc_ctx; /* opaque plan + state, owned by the library */

typedef enum {
  SC_OK = 0,
  SC_ERR_INVALID_ARG = 1, /* bad size, pointer, pattern or option */
  SC_ERR_NOT_SPD = 2,     /* a diagonal entry of L is not positive and finite */
  SC_ERR_CUDA = 3,        /* a CUDA runtime call failed (message has details) */
  SC_ERR_OOM = 4,         /* a buffer passed is smaller than sc_get_sizes asks */
  SC_ERR_TIMEOUT = 5,     /* a bounded device wait gave up (sc_options.poll_limit) */
  SC_ERR_INTERNAL = 6,
  SC_ERR_STATE = 7        /* call out of order (e.g. assemble before upload) */
} sc_status;

/* One subdomain, host arrays.  They are read during sc_plan only (patterns are
 * copied into the plan); values never pass through sc_plan.
 *   n, m        -- dofs of the subdomain, multipliers touching it (columns of B^T)
 *   L_colptr    -- [n+1] int64, CSC column pointers of L (lower, P K_reg P^T)
 *   L_rowind    -- [L_colptr[n]] int32, rows ascending, diagonal first per column
 *   Bt_colptr   -- [m+1] int32, CSC of B_i^T (n x m)
 *   Bt_rowind   -- [Bt_colptr[m]] int32, rows in L's ordering, ascending per column
 *   Bt_sign     -- [Bt_colptr[m]] int8, the entries of B_i^T (+1 or -1)
 *   lambda_map  -- [m] int32, local column -> global multiplier index
 *                  (used by sc_apply; may be NULL if sc_apply is never called)
 *   Bt_val      -- optional [Bt_colptr[m]] double, finite: the entries of the
 *                  right-hand side in place of Bt_sign (then NULL is allowed
 *                  for Bt_sign); the same F = C^T (L L^T)^{-1} C is assembled
 *                  for any sparse C, e.g. C = K_ib for the Schur complement
 *                  K_bi K_ii^{-1} K_ib of a Dirichlet preconditioner
 *                  (sc_plan only; sci_plan takes signed-Boolean columns)
 * Any number of nonzeros per column of B^T is accepted (general gluing); the
 * FETI case has exactly one. */
typedef struct {
  int32_t n, m;
  const int64_t *L_colptr;
  const int32_t *L_rowind;
  const int32_t *Bt_colptr;
  const int32_t *Bt_rowind;
  const int8_t *Bt_sign;
  const int32_t *lambda_map;
  const double *Bt_val;
} sc_subdomain_desc;

enum { SC_FP64 = 0, SC_SPLIT_BF16 = 1 };

/* precision: SC_FP64 -- every flop in IEEE binary64 (the default);
 *            SC_SPLIT_BF16 -- the off-diagonal GEMM work (the SYRK Y^T Y
 *            blocks and the TRSM updates below the diagonal triangles) runs
 *            on the tensor cores as exact products of 8-bit digit planes of
 *            the FP64 operands (BF16 in, FP32 accumulate, integer and FP64
 *            combination), n_slices digits per operand; the diagonal-triangle
 *            solves and the accumulation into Y and F stay FP64.  The error
 *            is below about 2^(-8 n_slices) relative to the product of the
 *            operands' column bounds; n_slices = 7 keeps 56 bits.
 * n_slices: 3..7 for SC_SPLIT_BF16 (0 selects 7); ignored for SC_FP64.
 * sub_slices: optional per-subdomain variant, nsub entries (host, read during
 *            sc_plan): 0 = FP64, 3..7 = split precision with that many
 *            digits; when given it overrides precision/n_slices.  Subdomains
 *            of each variant run as their own launch group; when a batch has
 *            several, sc_assemble_batch runs the groups concurrently on
 *            library-owned streams forked from and joined back into the
 *            caller's stream with events (the call stays asynchronous and
 *            ordered on the caller's stream). */
/* ws_limit: 0, or an upper bound in bytes for the workspace.  The subdomains
 *            (in their order) are then packed into waves whose temporary data
 *            (Y and, for split precision, the digit planes) fit the bound;
 *            waves run one after the other and reuse the same workspace (the
 *            paper's temporary memory pool, Sec. 3.1).  SC_ERR_OOM if one
 *            subdomain alone does not fit. */
/* persistent: 0 (default) launches one CTA per FP64 TRSM / SYRK task and
 *            lets the hardware block scheduler hand them out; 1 launches as
 *            many CTAs as the GPU keeps resident, which pull task indices
 *            (largest first) from an atomic counter in the workspace status
 *            area until the list is exhausted (a persistent work queue; no
 *            CTA waits on another). */
/* tile:     SYRK output tile of the split-precision subdomains: SC_TILE_32
 *            (default) -- 32x32 blocks of F on the warp-level tensor-core
 *            instruction (mma.sync); SC_TILE_TC128 -- 128x32 tiles (four row
 *            chunks by one column chunk, summed over the union of the four
 *            chunk pairs' supernode blocks) on the fifth-generation tensor
 *            cores (tcgen05.mma, accumulators in tensor memory).  Ignored for
 *            FP64 subdomains.  Same digits, same error bound.
 * sub_tile:  optional per-subdomain tile (nsub entries, host, read during
 *            sc_plan, 0 or 1); overrides `tile`.  Together with sub_slices it
 *            is the per-subdomain variant the autotuner and the learned
 *            selector choose (sc_select).
 * poll_limit: number of polls of every bounded device-side wait (the tcgen05
 *            kernels wait on mbarriers for their tensor-core work) before the
 *            kernel gives up, sets the timeout bit of the status word and
 *            returns (sc_device_status: SC_ERR_TIMEOUT); 0 selects 2^26. */
typedef struct {
  int32_t precision;
  int32_t n_slices;
  const int8_t *sub_slices;
  int64_t ws_limit;
  int32_t persistent;
  int32_t tile;
  const int8_t *sub_tile;
  int64_t poll_limit;
} sc_options;

enum { SC_TILE_32 = 0, SC_TILE_TC128 = 1 };

typedef struct {
  size_t plan_bytes;       /* device plan tables (sc_upload_plan) */
  size_t ws_bytes;         /* device workspace for sc_assemble_batch */
  int64_t F_doubles;       /* total doubles of all F_i (layout below) */
  int64_t L_values;        /* total entries of all L_i = sum_i L_colptr_i[n_i] */
  int32_t nsub;
  int32_t max_m;
} sc_sizes;

/* Per-batch counters of the plan (host, exact integers). */
typedef struct {
  double flops_trsm;        /* useful flops of the sparse forward substitution */
  double flops_syrk;        /* useful flops of the pruned SYRK (lower triangle) */
  double flops_trsm_exec;   /* flops the kernels issue (incl. 32-lane padding) */
  double flops_syrk_exec;
  double flops_dense;       /* sum_i n_i^2 m_i + n_i m_i (m_i + 1): the dense TRSM+SYRK yardstick */
  double bytes_assembly;    /* algorithmic bytes: 12 nnz(L) + 8 m(m+1)/2 per subdomain */
  double bytes_apply;       /* algorithmic bytes of sc_apply: 8 m(m+1)/2 + 16 m per subdomain */
  int64_t n_supernodes;     /* active supernodes (touched by some column) */
  int64_t n_trsm_tasks, n_syrk_tasks, n_apply_tasks;
  int64_t y_doubles;        /* workspace doubles of the sparse Y (all waves) */
  int64_t max_supernode;    /* columns of the largest active supernode */
  int64_t n_waves;          /* workspace waves (1 without ws_limit) */
} sc_stats;

/* ---- initialization -------------------------------------------------------- */

/* Validate the patterns and build the plan (host only; no CUDA call).
 * n_dual: length of the global dual vectors lambda and q (>= 1 + max lambda_map).
 * opt may be NULL (FP64 defaults).  *out is set whenever a context could be
 * allocated -- also on failure, so that sc_last_error(*out) explains it -- and
 * must be released with sc_destroy. */
sc_status sc_plan(sc_ctx **out, int32_t nsub, const sc_subdomain_desc *subdomains,
                  int64_t n_dual, const sc_options *opt);

sc_status sc_get_sizes(const sc_ctx *ctx, sc_sizes *out);
sc_status sc_get_stats(const sc_ctx *ctx, sc_stats *out);

/* F layout.  F_i (m_i x m_i, symmetric, rows/columns in B_i^T's column order)
 * is stored as its lower 32x32 tiles: tile (I, J), I >= J, is the block
 * rows [32I, 32I+32) x columns [32J, 32J+32); tiles are ordered I(I+1)/2 + J;
 * each tile is 1024 doubles, column-major; diagonal tiles hold both triangles;
 * entries beyond m_i are zero.  F_i starts at F_offsets[i] (doubles);
 * F_offsets has nsub+1 entries.  L values of subdomain i start at
 * L_offsets[i] in the concatenated L value array (nsub+1 entries). */
sc_status sc_get_offsets(const sc_ctx *ctx, int64_t *F_offsets, int64_t *L_offsets);

/* Copy the plan tables into caller-owned device memory of at least plan_bytes
 * (16-byte aligned); the context remembers the pointer for later calls.  The
 * copy is ordered on `stream`; the host tables stay owned by the context. */
sc_status sc_upload_plan(sc_ctx *ctx, void *plan_dev, size_t plan_bytes, void *stream);

/* ---- preprocessing ----------------------------------------------------------- */

/* Assemble every F_i from new L values (same patterns as planned).
 *   L_values_dev -- device, concatenated CSC values of all L_i (sizes.L_values)
 *   F_dev        -- device, sizes.F_doubles, written completely (padding zeroed)
 *   ws_dev       -- device workspace, >= sizes.ws_bytes, 256-byte aligned;
 *                   its contents on entry do not matter
 * Asynchronous on `stream`; check sc_device_status after completion. */
sc_status sc_assemble_batch(sc_ctx *ctx, const double *L_values_dev, double *F_dev,
                            void *ws_dev, size_t ws_bytes, void *stream);

/* Size of the library-owned scratch used by sc_assemble_batch_static. */
#define SC_STATIC_SCRATCH_BYTES ((size_t)64 << 20)

/* Batched assembly that allocates nothing: like sc_assemble_batch, but the
 * workspace is a 64 MiB array inside the library (SC_STATIC_SCRATCH_BYTES)
 * instead of caller memory.  The paper has no counterpart; this entry point
 * exists for callers that cannot call cudaMalloc -- a solver whose memory
 * manager reserved the free device memory up front, or a latency-sensitive
 * loop that cannot afford cudaMalloc's implicit device-wide synchronisation.
 * The caller still passes the inputs and outputs: the uploaded plan
 * (sc_upload_plan), L_values_dev and F_dev, as for sc_assemble_batch.
 *   - Plans whose sizes.ws_bytes exceeds SC_STATIC_SCRATCH_BYTES are rejected
 *     with SC_ERR_OOM before anything is launched.
 *   - The array is allocated in every CUDA context that loads the library's
 *     module (one copy per context, each at its own address) and stays
 *     allocated until that context is destroyed; for a device's primary
 *     context that is the end of the process.
 *   - Every call looks up the array's address in the calling thread's current
 *     context, so calls under different contexts use their own copies.
 *   - Every call in one context shares that context's array, which keeps the
 *     previous call's contents: calls that overlap on the GPU (other streams,
 *     other threads) race and must be serialised by the caller.
 *   - The call synchronises `stream` (it reads the device status word back
 *     into host memory) and returns this call's device status (SC_OK or
 *     SC_ERR_NOT_SPD), so no sc_device_status call is needed.
 *   - F_dev must be 8-byte aligned, as for sc_assemble_batch.
 * No cudaMalloc, cudaFree or allocating library routine is called. */
sc_status sc_assemble_batch_static(sc_ctx *ctx, const double *L_values_dev, double *F_dev, void *stream);

/* Synchronises `stream` and reads the device status word in ws_dev:
 * SC_OK, SC_ERR_NOT_SPD when a diagonal of L was not positive and finite, or
 * SC_ERR_TIMEOUT when a bounded device wait gave up (F is then undefined). */
sc_status sc_device_status(sc_ctx *ctx, const void *ws_dev, void *stream);

/* ---- solution ------------------------------------------------------------------ */

/* q = sum_i scatter_i(F_i * gather_i(lambda))  (Eq. "dualop_apply_expl" summed
 * over subdomains).  lambda_dev, q_dev: device, n_dual doubles each; q is
 * overwritten (the library zeroes it first).  Asynchronous on `stream`. */
sc_status sc_apply(sc_ctx *ctx, const double *F_dev, const double *lambda_dev, double *q_dev,
                   void *stream);

/* The same product with the multiply-adds on the integer pipes (GB300's FP64
 * pipe bounds sc_apply): every stored 32x32 tile of F and every 32-entry block
 * of lambda is cut to 53-bit fixed point against its own largest exponent,
 * the fixed-point values are split into two 27-bit limbs, the tile-vector
 * products are formed exactly with 32x32 -> 64-bit integer multiply-adds
 * and rounded to FP64 once per row and tile.  Error: about 2^-52 of
 * 32 max|tile| max|block| per row and tile (an FP64 GEMV's rounding is of
 * the same size).  Same arguments, layout and asynchrony as sc_apply; q is
 * overwritten.  The paper's Eq. "dualop_apply_expl"; the fixed-point form is
 * this library's. */
sc_status sc_apply_fixed(sc_ctx *ctx, const double *F_dev, const double *lambda_dev, double *q_dev,
                         void *stream);

/* The same product with the stored tiles split between GB300's two
 * arithmetic paths so that both work at once: of every four tiles a warp
 * visits, fp64_quarters (0..4) are multiplied in FP64 on the FP64 pipe (as
 * sc_apply) and the rest in fixed point on the integer pipes (as
 * sc_apply_fixed); each row and tile is rounded once either way, so the
 * error bound is that of the two forms.  fp64_quarters = 0 is sc_apply_fixed.
 * Same arguments, layout and asynchrony as sc_apply; q is overwritten. */
sc_status sc_apply_mixed(sc_ctx *ctx, const double *F_dev, const double *lambda_dev, double *q_dev,
                         int32_t fp64_quarters, void *stream);

/* ---- the product from a digit form of F, on the tensor cores ----------------
 * (paper Eq. "dualop_apply_expl"; the digit form and its tensor-core product
 * are this library's.)  sc_apply_digits_prepare writes, once per assembly, a
 * digit form of the tile-packed F: every stored 32x32 tile in 55-bit fixed
 * point against its largest exponent, as seven balanced base-256 digits of
 * one byte each (7184 bytes per tile against 8192 in FP64).  sc_apply_digits
 * then forms q = F lambda from it with exact integer digit products on the
 * FP16 tensor cores (mma.sync) and one FP64 scaling per row and tile: the
 * error is that of holding each tile and 32-entry block of lambda in 55 bits
 * against their largest entries (below 2^-49 of 32 max|tile| max|block| per
 * row and tile), the size of an FP64 product's rounding. */

/* Bytes of the digit-form buffer Fd: the digit tiles, per-call scratch for
 * the digits of lambda (944 bytes per 32-row block of every F_i) and a
 * 16-byte status word. */
sc_status sc_apply_digits_size(const sc_ctx *ctx, int64_t *bytes);

/* Fd_dev (device, sc_apply_digits_size bytes, 16-byte aligned, caller-owned)
 * := the digit form of F_dev (tile-packed, as written by sc_assemble_batch or
 * any operator of the same layout, every entry finite).  Asynchronous on
 * `stream`; F_dev is only read. */
sc_status sc_apply_digits_prepare(sc_ctx *ctx, const double *F_dev, void *Fd_dev, void *stream);

/* q_dev (n_dual doubles, overwritten) := sum_i scatter_i(F_i gather_i(lambda))
 * from the digit form Fd_dev (sc_apply_digits_prepare).  The call writes the
 * scratch part of Fd_dev: calls on one Fd_dev must not overlap.  Asynchronous
 * on `stream`; SC_ERR_STATE if the plan has no lambda_map.  The kernel's
 * waits for its bulk copies are bounded by sc_options.poll_limit polls; one
 * that gives up sets the timeout bit of Fd_dev's status word (q is then
 * incomplete). */
sc_status sc_apply_digits(sc_ctx *ctx, void *Fd_dev, const double *lambda_dev, double *q_dev, void *stream);

/* Reads and clears Fd_dev's status word (synchronises `stream`): SC_OK, or
 * SC_ERR_TIMEOUT if a call since the last check gave up a bounded wait. */
sc_status sc_apply_digits_status(sc_ctx *ctx, void *Fd_dev, void *stream);

/* Expand F_i into a dense full m_i x m_i column-major device matrix dst_dev
 * with leading dimension ld >= m_i.  Asynchronous on `stream`. */
sc_status sc_export_F(sc_ctx *ctx, const double *F_dev, int32_t i, double *dst_dev, int32_t ld,
                      void *stream);

/* ---- learned variant choice (row a9 of the hot path; no counterpart in the paper) -- */

/* Features of every subdomain, from the plan (host, exact counters): log2 of
 * n, m, nnz(L), active supernodes, the largest active supernode, the useful
 * TRSM flops, the useful SYRK flops, the dense-equivalent flops and the
 * doubles of the sparse Y, and log2(max / min diagonal entry of L) when
 * L_values_host (the concatenated values, host) is given, else 0.
 * out: nsub x SC_NUM_FEATURES floats, row-major. */
#define SC_NUM_FEATURES 10
sc_status sc_subdomain_features(const sc_ctx *ctx, const double *L_values_host, float *out);

/* A trained variant predictor: the MLP of include/sc_mlp.h with
 * n_in = SC_NUM_FEATURES, n_out = n_variants + (number of split variants),
 * whose outputs (after y = y' * y_scale + y_shift) are the log10 time of every
 * variant and then the log10 relative error of every split variant, in
 * variant order; inputs are normalised as x' = (x - x_shift) / x_scale.
 * A variant is (slices[v], tiles[v]): 0 = FP64 (tile SC_TILE_32), or 3..7
 * digits with SC_TILE_32 or SC_TILE_TC128 (sc_options).  The FP64 variant must
 * be one of them.  params_dev is device memory; the other arrays are host. */
typedef struct {
  int32_t n_variants;
  const int8_t *slices;
  const int8_t *tiles;
  int32_t n_hidden;
  const float *params_dev;
  const float *x_shift, *x_scale;
  const float *y_shift, *y_scale;
} sc_selector;

/* Device workspace of sc_select, in floats. */
sc_status sc_select_workspace(const sc_ctx *ctx, const sc_selector *sel, size_t *ws_floats);

/* Per subdomain of the planned batch, the fastest variant whose predicted
 * error times `margin` (>= 1) meets `tol`, the FP64 variant qualifying always:
 * the features of sc_subdomain_features, one MLP forward pass over the batch
 * on the GPU (sc_mlp_forward, ws_dev caller-owned), the choice on the host.
 * Writes sub_slices and sub_tile (nsub entries each, host) for the
 * sc_options of the plan that then runs the batch.  Synchronises `stream`. */
sc_status sc_select(sc_ctx *ctx, const sc_selector *sel, const double *L_values_host, double tol, double margin,
                    float *ws_dev, size_t ws_floats, int8_t *sub_slices, int8_t *sub_tile, void *stream);

/* ---- misc ---------------------------------------------------------------------- */

/* Stage timing.  With timing on, sc_assemble_batch records a CUDA event on its
 * stream before the first kernel and after each stage: [0] prep (reciprocal
 * diagonal, F padding), [1] sparse TRSM, [2] pruned SYRK (for a batch with
 * several variant groups, [1] covers the TRSM and the SYRK of all groups and
 * [2] is zero).  sc_stage_times
 * synchronises on the last recorded event and writes up to n elapsed times
 * (milliseconds) of the last timed call.  Events are created by
 * sc_enable_stage_timing(ctx, 1) on the current device and destroyed by
 * sc_enable_stage_timing(ctx, 0) or sc_destroy. */
sc_status sc_enable_stage_timing(sc_ctx *ctx, int32_t on);
sc_status sc_stage_times(sc_ctx *ctx, float *ms, int32_t n);

/* Copy the plan tables (exactly sizes.plan_bytes) into host memory `dst`.  The
 * blob starts with a 512-byte self-describing header (magic "SCPL", version,
 * counts, section offsets and sizes); it is what sc_upload_plan copies to the
 * device, so it can be stored and inspected.  SC_ERR_OOM if bytes is too small. */
sc_status sc_export_plan(const sc_ctx *ctx, void *dst, size_t bytes);

/* Byte offsets inside the workspace: the 4-byte device status word, the
 * reciprocal diagonal of L (one double per column of every subdomain) and
 * the sparse Y blocks (sizes/stats.y_doubles doubles). */
sc_status sc_workspace_layout(const sc_ctx *ctx, size_t *status_off, size_t *invdiag_off, size_t *y_off);

const char *sc_last_error(const sc_ctx *ctx);
void sc_destroy(sc_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* SC_H */
