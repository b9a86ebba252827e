/* Host sparse Cholesky producing the factor L consumed by the Schur-complement
 * library (input producer, FP64, CPU only; not part of the GPU hot path).
 *
 * Paper Sec. 2.2 (two-stage factorisation, symbolic then numeric, of the
 * regularised subdomain matrix K_reg = L L^T; K^+ = K_reg^{-1}).
 *
 * Conventions
 *   - K is passed in full symmetric CSC (both triangles), original dof order,
 *     int64 column pointers, int32 row indices, FP64 values.  Host memory,
 *     owned by the caller, only read during the call.
 *   - fixed[] lists the dofs fixed to regularise a floating subdomain: their
 *     rows and columns are replaced by the identity (fixing-node reading of
 *     the paper's regularisation).
 *   - perm_in[new] = old is the fill-reducing ordering (NULL = identity).  With
 *     do_postorder != 0 the etree postorder is composed into it; the final
 *     ordering is returned by scf_export.
 *   - The factor is CSC lower triangular of P K_reg P^T, rows ascending,
 *     diagonal first in each column.  The handle owns it until scf_free.
 * Errors: SCF_ERR_INVALID_ARG (bad sizes, indices or permutation),
 *         SCF_ERR_NOT_SPD (non-positive or non-finite pivot), SCF_ERR_OOM.
 *         No partial result is returned on error (*out stays NULL).
 */
#ifndef SC_FACTOR_H
#define SC_FACTOR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { SCF_OK = 0, SCF_ERR_INVALID_ARG = 1, SCF_ERR_NOT_SPD = 2, SCF_ERR_OOM = 3 };

typedef struct scf_factor scf_factor;

/* Symbolic and numeric stage in one call: scf_analyze, then scf_numeric into
 * the handle's own values. */
int scf_factorize(int32_t n, const int64_t *K_colptr, const int32_t *K_rowind, const double *K_val,
                  int32_t nfixed, const int32_t *fixed, const int32_t *perm_in, int32_t do_postorder,
                  scf_factor **out);

/* Symbolic stage alone (paper Sec. 2.2): ordering (perm_in, optional
 * postorder), the pattern of L, and the map from K's stored entries to the
 * regularised, permuted matrix.  Only K's pattern is read.  The handle's
 * values are zero until scf_numeric writes them elsewhere; scf_export of
 * colptr, rowind and perm is valid at once.  K_colptr must start at 0 and
 * be non-decreasing, every row index in [0, n): SCF_ERR_INVALID_ARG
 * otherwise. */
int scf_analyze(int32_t n, const int64_t *K_colptr, const int32_t *K_rowind, int32_t nfixed, const int32_t *fixed,
                const int32_t *perm_in, int32_t do_postorder, scf_factor **out);

/* Numeric stage for an analysed pattern: L's values (scf_nnz doubles, the
 * CSC layout scf_export gives) from K_val, the stored values of a K with
 * exactly the pattern given to scf_analyze (same K_colptr, K_rowind; the
 * values may differ from call to call).  The handle is only read, so
 * several threads may run scf_numeric on one handle into different outputs.
 * L_val is caller memory (host, e.g. a pinned staging buffer) and is fully
 * overwritten on success; on SCF_ERR_NOT_SPD its contents are unspecified.
 * Gives bit for bit the values scf_factorize gives for the same input. */
int scf_numeric(const scf_factor *f, const double *K_val, double *L_val);

/* number of stored entries of L (lower triangle incl. diagonal); -1 on NULL */
int64_t scf_nnz(const scf_factor *f);

/* copy L out: colptr[n+1], rowind[nnz], val[nnz], perm[n] (new -> old); any
 * pointer may be NULL to skip that array */
int scf_export(const scf_factor *f, int64_t *colptr, int32_t *rowind, double *val, int32_t *perm);

void scf_free(scf_factor *f);

/* Implicit application of the dual operator on the host (paper Sec. 2.2,
 * Eq. "dualop_apply_impl"): q = sum_i B_i L_i^{-T} L_i^{-1} B_i^T lambda_i,
 * i.e. a sparse scatter, two sparse triangular solves and a sparse gather per
 * subdomain.  Arrays as in sc_subdomain_desc plus L's values; all host memory,
 * read only; q (n_dual doubles) is overwritten.  nthreads <= 0 uses every
 * hardware thread; threads split the subdomains and sum private dual vectors
 * in a fixed order.  Returns SCF_ERR_INVALID_ARG on bad sizes or maps, or
 * on a pattern that is not CSC lower with the diagonal first and rows
 * strictly ascending (checked on every call; scf_implicit_plan checks once). */
typedef struct {
  int32_t n, m;
  const int64_t *L_colptr;
  const int32_t *L_rowind;
  const double *L_val;
  const int32_t *Bt_colptr;
  const int32_t *Bt_rowind;
  const int8_t *Bt_sign;
  const int32_t *lambda_map;
} scf_apply_subdomain;

int scf_implicit_apply(int32_t nsub, const scf_apply_subdomain *subs, int64_t n_dual, const double *lambda,
                       double *q, int32_t nthreads);

/* x = L^-T L^-1 b for one factor in CSC (the arrays of scf_export, L's
 * ordering): a forward and a backward sparse triangular solve on the host.
 * b and x are n doubles, host memory; x may equal b.  SCF_ERR_INVALID_ARG on
 * NULL arrays or a pattern that is not CSC lower with the diagonal first and
 * rows strictly ascending. */
int scf_solve(int32_t n, const int64_t *L_colptr, const int32_t *L_rowind, const double *L_val, const double *b,
              double *x);

/* The same product with its symbolic work done once (the implicit approach's
 * own preprocessing, paper Sec. 2.2).  scf_implicit_plan reads the patterns:
 * per subdomain the supernodes of L (runs of columns with one shared
 * pattern, checked entry by entry) and the supernodes on the etree paths from
 * B^T's rows, the only ones the two solves touch.  It copies the
 * scf_apply_subdomain records but not the arrays they point to: those must
 * stay valid, and their patterns unchanged, while the plan is used; L's
 * values may change between runs (new factor, same pattern).
 * scf_implicit_run then solves supernode by supernode: dense triangles on
 * contiguous rows, the rows below updated from contiguous L values through
 * one scatter (forward) or one gather (backward) per supernode.  Same
 * threading and fixed summation order as scf_implicit_apply; the results of
 * the two agree to rounding.  SCF_ERR_INVALID_ARG on bad sizes, maps or row
 * indices; SCF_ERR_OOM if the plan cannot be allocated (*out stays NULL). */
typedef struct scf_implicit scf_implicit;
int scf_implicit_plan(int32_t nsub, const scf_apply_subdomain *subs, int64_t n_dual, scf_implicit **out);
int scf_implicit_run(const scf_implicit *plan, const double *lambda, double *q, int32_t nthreads);
void scf_implicit_free(scf_implicit *plan);

#ifdef __cplusplus
}
#endif

#endif /* SC_FACTOR_H */
