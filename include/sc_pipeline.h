/* sc_pipeline.h -- the numeric stage of the whole assembly as a CPU/GPU
 * pipeline.
 *
 * Paper Sec. 2.2 (stages) and Sec. 5 (the configuration in which the CPU
 * factorises while the GPU assembles): the subdomains' numeric Cholesky
 * factorisations run on host threads, the Schur-complement assembly on the
 * GPU.  Here the batch is cut into chunks, each with its own plan
 * (include/sc.h), and the chunks go through three overlapped steps:
 *
 *     host threads   factorise chunk c+1 into a pinned staging buffer
 *     copy stream    host->device copy of chunk c's L values
 *     compute stream sc_assemble_batch of chunk c
 *
 * so that the host factorisation hides the GPU work (or the other way round)
 * instead of adding to it.  The symbolic work (ordering, sc_plan, plan
 * upload, and the symbolic stage of every host factorisation, scf_analyze of
 * sc_factor.h, which scp_create runs) is the initialisation stage and
 * happens before, once; scp_run runs only the numeric stage (scf_numeric),
 * writing each L straight into the staging buffer.
 *
 * Inputs per subdomain (host memory owned by the caller): K in full
 * symmetric CSC (original dof order), the fixed dofs of the regularisation,
 * and the final fill-reducing ordering perm[new] = old with which the
 * chunk's plan was made (the factor is computed as L L^T = P K_reg P^T with
 * exactly this P, no further reordering).  K's pattern, the fixed dofs and
 * perm are read in scp_create; K's values (K_val) are read during every
 * scp_run, so new values on the same pattern give new factors and F.
 * Per chunk: its plan (sc_plan of exactly the subdomains [lo, hi), uploaded)
 * and device buffers for its L values (plan's L_values doubles), F and
 * workspace.  Chunks may share a workspace (they run in order on one
 * stream); the copy into a chunk's L buffer waits for the assembly two
 * chunks earlier, so two L buffers used alternately are enough.
 *
 * The library allocates two pinned host staging buffers (the largest
 * chunk's L values each), CUDA events and one copy stream per context.
 *
 * Errors: sc_status codes of sc.h.  SC_ERR_NOT_SPD when a host factorisation
 * meets a non-positive pivot (scp_run); SC_ERR_INVALID_ARG when a factor's
 * pattern does not match its plan (different nnz per subdomain) or arguments
 * are invalid (scp_create); SC_ERR_INTERNAL when a host allocation fails;
 * SC_ERR_CUDA on a CUDA error. */
#ifndef SC_PIPELINE_H
#define SC_PIPELINE_H

#include <stddef.h>
#include <stdint.h>

#include "sc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct scp_ctx scp_ctx;

typedef struct {
  int32_t n;
  const int64_t *K_colptr;
  const int32_t *K_rowind;
  const double *K_val;
  int32_t nfixed;
  const int32_t *fixed;
  const int32_t *perm;
} scp_subdomain;

typedef struct {
  int32_t lo, hi;         /* subdomains [lo, hi) of the scp_subdomain array */
  sc_ctx *plan;           /* plan of exactly these subdomains, uploaded */
  double *L_dev;          /* device, >= the plan's L_values doubles */
  double *F_dev;          /* device, >= the plan's F_doubles */
  void *ws_dev;           /* device workspace of sc_assemble_batch */
  size_t ws_bytes;
} scp_chunk;

typedef struct {
  double wall_ms;         /* scp_run: first factorisation to the last assembly's completion */
  double factor_ms;       /* sum over chunks of the host factorisation wall time */
  double h2d_ms;          /* sum over chunks of the copy time (CUDA events) */
  double assembly_ms;     /* sum over chunks of the assembly time (CUDA events) */
  double serial_ms;       /* factor_ms + h2d_ms + assembly_ms: the same work one step after another */
  int64_t h2d_bytes;
} scp_times;

/* nthreads <= 0: every hardware thread (used for the symbolic stage here and
 * the numeric stage in scp_run).  The arrays are copied (the pointers inside
 * scp_subdomain are not: K_val must outlive every scp_run). */
sc_status scp_create(scp_ctx **out, int32_t nsub, const scp_subdomain *subs, int32_t nchunks,
                     const scp_chunk *chunks, int32_t nthreads);

/* Runs the pipeline on `stream` (the compute stream) and returns when every
 * chunk's F is assembled.  times may be NULL. */
sc_status scp_run(scp_ctx *ctx, void *stream, scp_times *times);

const char *scp_last_error(const scp_ctx *ctx);
void scp_destroy(scp_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* SC_PIPELINE_H */
