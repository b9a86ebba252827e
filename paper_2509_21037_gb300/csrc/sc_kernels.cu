// sm_103a kernels of the Schur-complement assembly and application (FP64).
//
//   prep_kernel   -- reciprocal of L's diagonal for every column of an active
//                    supernode; a non-positive / non-finite pivot sets the
//                    NOT_SPD bit of the workspace status word (paper Sec. 3.1:
//                    the factor is copied in; here its CSC columns are read
//                    in place, because a fundamental supernode's CSC column is
//                    already a dense trapezoidal panel column).
//   trsm_kernel   -- Y = L^{-1} P B^T on one 32-column chunk of the pivot-sorted
//                    columns (paper Sec. 3.2): zero + seed the chunk's nonzero
//                    part of Y, then for each supernode the chunk touches
//                    (children first) a blocked forward substitution: 32x32
//                    diagonal triangle solved by one warp (lane = column),
//                    then the GEMM update of every panel row below it -- the
//                    rest of the diagonal block and the pruned rows, whose
//                    results land in the ancestors' Y blocks.
//   syrk_kernel   -- one 32x32 block of F = Y^T Y in pivot-sorted order
//                    (paper Sec. 3.3), summed over the supernodes active on
//                    both chunks; the epilogue writes it straight into the
//                    user's column order (the final back-permutation).
//   apply_kernel  -- q += scatter(F_i gather(lambda)) reading each stored
//                    lower tile once and using it for both triangles.
//   export_kernel -- tile-packed F_i -> dense full column-major matrix.
//
// FP64 on GB300 is a narrow pipe (about 1.2 TFLOP/s for the whole GPU), so
// these kernels are bound by FP64 issue; the work they do is what the plan's
// sparsity pattern leaves, and the launch sizes keep every SM busy with
// several CTAs so that one CTA's serial triangle solve overlaps other CTAs'
// updates.
#include <cuda_runtime.h>

#include <algorithm>

#include <cstdint>

#include "sc_internal.h"

namespace sc {

__global__ void prep_kernel(const int64_t *__restrict__ lcp, const int32_t *__restrict__ active,
                            int64_t nact, const double *__restrict__ Lv, double *__restrict__ invd,
                            uint32_t *__restrict__ status) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nact;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t g = active[k];
    const double d = Lv[lcp[g]];
    if (!(d > 0.0) || !isfinite(d)) {
      atomicOr(status, kStatusNotSpd);
      invd[g] = 0.0;
    } else {
      invd[g] = 1.0 / d;
    }
  }
}

// Zero the entries of F beyond m: rows >= m of the last tile row and columns
// >= m of the last diagonal tile.  One CTA per subdomain.
__global__ void fpad_kernel(const SubDev *__restrict__ subs, double *__restrict__ F) {
  const SubDev sd = subs[blockIdx.x];
  if (sd.nt == 0) return;
  const int rem = sd.m - (sd.nt - 1) * kTile;
  if (rem == kTile) return;
  const int I = sd.nt - 1;
  for (int J = 0; J <= I; ++J) {
    double *T = F + sd.F_off + ((int64_t)I * (I + 1) / 2 + J) * (kTile * kTile);
    for (int e = threadIdx.x; e < kTile * kTile; e += blockDim.x) {
      const int r = e & (kTile - 1), c = e / kTile;
      if (r >= rem || (J == I && c >= rem)) T[e] = 0.0;
    }
  }
}

// One TRSM task (a 32-column chunk of one subdomain).  Xs: the current 32-row
// block of the solved chunk, [row][column]; cps[q] = index of L(p, c0+kb+q) minus p.
// The diagonal triangles are solved by warp `tri` of the CTA (see tri_warp).
__device__ __forceinline__ void trsm_task(const PlanPtrs &P, const TrsmTask t, const double *__restrict__ Lv,
                                          const double *__restrict__ invd, double *__restrict__ Y,
                                          double (*Xs)[33], int64_t *cps, int tri) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int c_hi = t.c_lo + t.w;

  // zero the chunk's part of every touched Y block, then seed B^T's entries
  for (int li = 0; li < t.list_len; ++li) {
    const SnDev s = P.sns[P.trsm_list[t.list_off + li]];
    const int a = max(s.jlo, t.c_lo), b = min(s.jhi, c_hi), w = b - a, ws = s.jhi - s.jlo;
    double *Ys = Y + s.y_off + (a - s.jlo);
    const int total = s.ns * w;
    for (int idx = tid; idx < total; idx += kThreads) {
      const int r = idx / w, c = idx - r * w;
      Ys[(int64_t)r * ws + c] = 0.0;
    }
  }
  __syncthreads();
  for (int e = t.seed_lo + tid; e < t.seed_hi; e += kThreads) {
    const Seed sd = P.seeds[e];
    Y[sd.y_off] = sd.value;
  }
  __syncthreads();

  for (int li = 0; li < t.list_len; ++li) {
    const SnDev s = P.sns[P.trsm_list[t.list_off + li]];
    const int a = max(s.jlo, t.c_lo), b = min(s.jhi, c_hi), w = b - a, ws = s.jhi - s.jlo;
    double *Ys = Y + s.y_off + (a - s.jlo);
    const int64_t *cp = P.lcp + s.lcp_off;
    const double *id = invd + s.lcp_off;
    const int64_t *rm = P.rmap + s.rmap_off;
    const int colsh = a - s.jlo;
    const int nrow = s.ns + s.rs;
    for (int kb = 0; kb < s.ns; kb += 32) {
      const int kw = min(32, s.ns - kb);
      // columns at or after the block's cut are still zero in these rows
      const int wk = min(b, P.cuts[s.cut_off + (kb >> 5)]) - a;
      if (wk <= 0) continue;
      // The triangle, 8 columns at a time: warp `tri` solves the 8x8 diagonal
      // piece, then all warps update the block's rows below it (every entry
      // gets its updates in the same column order as a column-by-column solve)
      if (tid < kw) cps[tid] = cp[kb + tid] - (kb + tid);
      for (int e = tid; e < kw * 32; e += kThreads) {
        const int q = e >> 5, c = e & 31;
        if (c < wk) Xs[q][c] = Ys[(int64_t)(kb + q) * ws + c];
      }
      __syncthreads();
      for (int p0 = 0; p0 < kw; p0 += 8) {
        const int pe = min(p0 + 8, kw);
        if (warp == tri && lane < wk) {
          for (int q = p0; q < pe; ++q) {
            const double xq = Xs[q][lane] * id[kb + q];
            Xs[q][lane] = xq;
            const double *Lc = Lv + cps[q];
            for (int r = q + 1; r < pe; ++r) Xs[r][lane] = fma(-Lc[kb + r], xq, Xs[r][lane]);
          }
        }
        __syncthreads();
        if (pe < kw) {
          if (lane < wk) {
            for (int r = pe + ((warp - tri) & 3); r < kw; r += kThreads / 32) {
              double xr = Xs[r][lane];
              for (int q = p0; q < pe; ++q) xr = fma(-Lv[cps[q] + kb + r], Xs[q][lane], xr);
              Xs[r][lane] = xr;
            }
          }
          __syncthreads();
        }
      }
      if (warp == tri && lane < wk)
        for (int q = 0; q < kw; ++q) Ys[(int64_t)(kb + q) * ws + lane] = Xs[q][lane];
      __syncthreads();
      // Update of the rows below.  The FP64 pipe charges a warp instruction in
      // full whatever the number of active lanes, so the (row, column) pairs
      // of the update are numbered row-major over the wk live columns and
      // dealt to the CTA's threads in turn: every lane of a warp step works
      // (but the last), whatever wk is.
      {
        const int dp = kThreads / wk, dc = kThreads - dp * wk;   // one step of kThreads pairs
        int p = kb + kw + tid / wk, cl = tid - (tid / wk) * wk;
        while (p < nrow) {                                       // pair (p, cl) exists iff p < nrow
          // the target row is the accumulator: no separate subtraction on the FP64 pipe
          double *tg = (p < s.ns) ? (Ys + (int64_t)p * ws) : (Y + rm[p - s.ns] + colsh);
          double acc = tg[cl];
#pragma unroll 16
          for (int q = 0; q < kw; ++q) acc = fma(-Lv[cps[q] + p], Xs[q][cl], acc);
          tg[cl] = acc;
          p += dp;
          cl += dc;
          if (cl >= wk) {
            cl -= wk;
            ++p;
          }
        }
      }
      __syncthreads();
    }
  }
}

// The warp of a CTA that solves the serial 32x32 triangles.  The FP64 pipe
// belongs to the SM's four sub-partitions and a CTA's warps are spread over
// them, so a fixed choice (warp 0) would put the triangle work of every
// co-resident CTA on one sub-partition; a hash of the task index spreads it.
__device__ __forceinline__ int tri_warp(unsigned k) { return (int)((k * 2654435761u) >> 30); }

// Work-queue form (queue != nullptr): a grid sized to the resident CTAs pulls
// task indices from an atomic counter until the list is exhausted; otherwise
// one CTA per task.  Tasks are ordered largest first by the planner.
__global__ void __launch_bounds__(kThreads, 16) trsm_kernel(const PlanPtrs P, const double *__restrict__ Lv,
                                                        const double *__restrict__ invd, double *__restrict__ Y,
                                                        unsigned *queue, int ntask) {
  __shared__ double Xs[32][33];
  __shared__ int64_t cps[32];
  __shared__ int next;
  if (!queue) {
    trsm_task(P, P.trsm_tasks[blockIdx.x], Lv, invd, Y, Xs, cps, tri_warp(blockIdx.x));
    return;
  }
  for (;;) {
    if (threadIdx.x == 0) next = (int)atomicAdd(queue, 1u);
    __syncthreads();
    const int k = next;
    __syncthreads();
    if (k >= ntask) break;
    trsm_task(P, P.trsm_tasks[k], Lv, invd, Y, Xs, cps, tri_warp((unsigned)k));
    __syncthreads();
  }
}

// Diagonal output block (q1 == q2) of F = Y^T Y: only its lower triangle is
// needed, and the FP64 pipe charges masked lanes in full, so the 528 lower
// elements are dealt to the threads directly (slot u of thread t is element
// t + 128 u, u < 5) and the chunk's tile is loaded once.
__device__ __forceinline__ void syrk_diag_block(const PlanPtrs &P, const SyrkTask &t, const SubDev &sd,
                                                const double *__restrict__ Y, double *__restrict__ F,
                                                double (*As)[33]) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int jlo = t.q1 * kChunk;
  constexpr int kLower = 32 * 33 / 2;   // 528
  int rr[5], cc[5];
#pragma unroll
  for (int u = 0; u < 5; ++u) {
    const int e = tid + kThreads * u;
    int r = (int)((sqrtf(8.f * e + 1.f) - 1.f) * 0.5f);
    while ((r + 1) * (r + 2) / 2 <= e) ++r;     // exact integer correction
    while (r * (r + 1) / 2 > e) --r;
    rr[u] = e < kLower ? r : 0;
    cc[u] = e < kLower ? e - r * (r + 1) / 2 : 0;
  }
  const bool fifth = tid + kThreads * 4 < kLower;  // only the first 16 threads (warp 0) own slot 4
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int li = 0; li < t.list_len; ++li) {
    const SnDev s = P.sns[P.syrk_list[t.list_off + li]];
    const int ws = s.jhi - s.jlo;
    const double *Ys = Y + s.y_off;
    const int ja = jlo + lane - s.jlo;
    const bool oka = ja >= 0 && ja < ws;
    for (int k0 = 0; k0 < s.ns; k0 += 32) {
      if (jlo >= P.cuts[s.cut_off + (k0 >> 5)]) continue;
      const int kk = min(32, s.ns - k0);
      for (int k = warp; k < kk; k += kThreads / 32) As[k][lane] = oka ? Ys[(int64_t)(k0 + k) * ws + ja] : 0.0;
      __syncthreads();
      if (warp == 0) {
        for (int k = 0; k < kk; ++k) {
#pragma unroll
          for (int u = 0; u < 4; ++u) acc[u] = fma(As[k][rr[u]], As[k][cc[u]], acc[u]);
          if (fifth) acc[4] = fma(As[k][rr[4]], As[k][cc[4]], acc[4]);
        }
      } else {
        for (int k = 0; k < kk; ++k) {
#pragma unroll
          for (int u = 0; u < 4; ++u) acc[u] = fma(As[k][rr[u]], As[k][cc[u]], acc[u]);
        }
      }
      __syncthreads();
    }
  }
  const int32_t *perm = P.perm_cols + sd.col_off;
#pragma unroll
  for (int u = 0; u < 5; ++u) {
    if (tid + kThreads * u >= kLower) continue;
    const int j1 = jlo + rr[u], j2 = jlo + cc[u];
    if (j1 < sd.m && j2 < sd.m) {
      const int a = perm[j1], b = perm[j2];
      const int hi = max(a, b), lo = min(a, b);
      const int I = hi / kTile, J = lo / kTile;
      double *T = F + sd.F_off + ((int64_t)I * (I + 1) / 2 + J) * (kTile * kTile);
      T[(hi % kTile) + kTile * (lo % kTile)] = acc[u];
      if (I == J) T[(lo % kTile) + kTile * (hi % kTile)] = acc[u];
    }
  }
}

// One SYRK task (a 32x32 block of F); As, Bs: [k][column of the chunk]
__device__ __forceinline__ void syrk_task(const PlanPtrs &P, const SyrkTask t, const double *__restrict__ Y,
                                          double *__restrict__ F, double (*As)[33], double (*Bs)[33]) {
  const SubDev sd = P.subs[t.sub];
  if (t.q1 == t.q2) {
    syrk_diag_block(P, t, sd, Y, F, As);
    return;
  }
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int j1lo = t.q1 * kChunk, j2lo = t.q2 * kChunk;
  double acc[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) acc[u] = 0.0;
  for (int li = 0; li < t.list_len; ++li) {
    const SnDev s = P.sns[P.syrk_list[t.list_off + li]];
    const int ws = s.jhi - s.jlo;
    const double *Ys = Y + s.y_off;
    const int ja = j1lo + lane - s.jlo, jb = j2lo + lane - s.jlo;
    const bool oka = ja >= 0 && ja < ws, okb = jb >= 0 && jb < ws;
    for (int k0 = 0; k0 < s.ns; k0 += 32) {
      // rows of this block are zero for sorted columns >= cut; j1lo >= j2lo
      if (j1lo >= P.cuts[s.cut_off + (k0 >> 5)]) continue;
      const int kk = min(32, s.ns - k0);
      for (int k = warp; k < kk; k += kThreads / 32) {
        const double *row = Ys + (int64_t)(k0 + k) * ws;
        As[k][lane] = oka ? row[ja] : 0.0;
        Bs[k][lane] = okb ? row[jb] : 0.0;
      }
      __syncthreads();
      for (int k = 0; k < kk; ++k) {
        const double bv = Bs[k][lane];
#pragma unroll
        for (int u = 0; u < 8; ++u) acc[u] = fma(As[k][warp * 8 + u], bv, acc[u]);
      }
      __syncthreads();
    }
  }
  const int32_t *perm = P.perm_cols + sd.col_off;
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int j1 = j1lo + warp * 8 + u, j2 = j2lo + lane;
    if (j1 < sd.m && j2 < sd.m) {
      const int a = perm[j1], b = perm[j2];
      const int hi = max(a, b), lo = min(a, b);
      const int I = hi / kTile, J = lo / kTile;
      double *T = F + sd.F_off + ((int64_t)I * (I + 1) / 2 + J) * (kTile * kTile);
      T[(hi % kTile) + kTile * (lo % kTile)] = acc[u];
      if (I == J) T[(lo % kTile) + kTile * (hi % kTile)] = acc[u];
    }
  }
}

__global__ void __launch_bounds__(kThreads) syrk_kernel(const PlanPtrs P, const double *__restrict__ Y,
                                                        double *__restrict__ F, unsigned *queue, int ntask) {
  __shared__ double As[32][33], Bs[32][33];
  __shared__ int next;
  if (!queue) {
    syrk_task(P, P.syrk_tasks[blockIdx.x], Y, F, As, Bs);
    return;
  }
  for (;;) {
    if (threadIdx.x == 0) next = (int)atomicAdd(queue, 1u);
    __syncthreads();
    const int k = next;
    __syncthreads();
    if (k >= ntask) break;
    syrk_task(P, P.syrk_tasks[k], Y, F, As, Bs);
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kThreads) apply_kernel(const PlanPtrs P, const double *__restrict__ F,
                                                         const double *__restrict__ lam,
                                                         double *__restrict__ q) {
  __shared__ double Ts[kThreads / 32][32][33];
  __shared__ double red[kThreads / 32][32];
  const ApplyTask t = P.apply_tasks[blockIdx.x];
  const SubDev sd = P.subs[t.sub];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int32_t *map = P.lambda + sd.col_off;
  const int I = t.I;
  const int rowI = I * kTile + lane;
  const double pI = rowI < sd.m ? lam[map[rowI]] : 0.0;
  double y = 0.0;
  for (int J = warp; J <= I; J += kThreads / 32) {
    const double *Tg = F + sd.F_off + ((int64_t)I * (I + 1) / 2 + J) * (kTile * kTile);
#pragma unroll 8
    for (int c = 0; c < 32; ++c) Ts[warp][c][lane] = Tg[c * 32 + lane];
    __syncwarp();
    const int colJ = J * kTile + lane;
    const double pJ = colJ < sd.m ? lam[map[colJ]] : 0.0;
#pragma unroll 8
    for (int c = 0; c < 32; ++c) y = fma(Ts[warp][c][lane], __shfl_sync(0xffffffffu, pJ, c), y);
    if (J < I) {
      double z = 0.0;
#pragma unroll 8
      for (int r = 0; r < 32; ++r) z = fma(Ts[warp][lane][r], __shfl_sync(0xffffffffu, pI, r), z);
      if (colJ < sd.m) atomicAdd(q + map[colJ], z);
    }
    __syncwarp();
  }
  red[warp][lane] = y;
  __syncthreads();
  if (warp == 0) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) s += red[w][lane];
    if (rowI < sd.m) atomicAdd(q + map[rowI], s);
  }
}

__global__ void export_kernel(const SubDev *__restrict__ subs, int32_t i, const double *__restrict__ F,
                              double *__restrict__ dst, int32_t ld) {
  const SubDev sd = subs[i];
  const int64_t total = (int64_t)sd.m * sd.m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(e % sd.m), b = (int)(e / sd.m);
    const int hi = max(a, b), lo = min(a, b);
    const int I = hi / kTile, J = lo / kTile;
    const double *T = F + sd.F_off + ((int64_t)I * (I + 1) / 2 + J) * (kTile * kTile);
    dst[a + (int64_t)b * ld] = T[(hi % kTile) + kTile * (lo % kTile)];
  }
}

// ---------------------------------------------------------------------------
// launchers

static inline cudaStream_t S(void *s) { return static_cast<cudaStream_t>(s); }

// CTAs of `kernel` (kThreads threads, static shared memory) the GPU keeps resident at once
template <class K>
int resident_ctas(K kernel) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, kThreads, 0);
  return std::max(1, sms * std::max(1, per));
}

int launch_prep(const sc_ctx &c, const double *Lv, double *invd, uint32_t *status, double *F, void *ws,
                void *stream) {
  const PlanPtrs p = c.ptrs();
  if (c.n_active_cols > 0) {
    int64_t blocks = (c.n_active_cols + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    prep_kernel<<<(unsigned)blocks, 256, 0, S(stream)>>>(p.lcp, p.active_cols, c.n_active_cols, Lv, invd,
                                                         status);
  }
  if (c.nsub > 0) fpad_kernel<<<c.nsub, 128, 0, S(stream)>>>(p.subs, F);
  int e = (int)cudaGetLastError();
  if (!e && c.n_slices > 0) e = launch_colexp_reset(c, ws, stream);
  return e;
}

// First half of one variant group's pipeline: (digit planes of L,) sparse TRSM.
int launch_group_trsm(const sc_ctx &c, int w, int v, const double *Lv, const double *invd, void *ws, double *Y,
                      void *stream) {
  const auto &G = c.waves[w];
  if (v == 0) {
    if (G.trsm[0][1] > 0) {
      PlanPtrs p = c.ptrs();
      p.trsm_tasks += G.trsm[0][0];
      const int n = (int)G.trsm[0][1];
      if (c.persistent) {
        unsigned *q = reinterpret_cast<unsigned *>(static_cast<uint8_t *>(ws) + c.ws.status_off + 64);
        cudaError_t e = cudaMemsetAsync(q, 0, sizeof(unsigned), S(stream));
        if (e != cudaSuccess) return (int)e;
        const int grid = std::min(n, resident_ctas(trsm_kernel));
        trsm_kernel<<<(unsigned)grid, kThreads, 0, S(stream)>>>(p, Lv, invd, Y, q, n);
      } else {
        trsm_kernel<<<(unsigned)n, kThreads, 0, S(stream)>>>(p, Lv, invd, Y, nullptr, n);
      }
    }
    return (int)cudaGetLastError();
  }
  const int S = var_digits(v);
  int e = launch_lpack_split(c, S, G.sblk[v][0], G.sblk[v][1], Lv, ws, stream);
  if (!e) e = launch_trsm_split(c, S, G.trsm[v][0], G.trsm[v][1], Lv, invd, ws, Y, stream);
  return e;
}

// Second half: (digit planes of Y,) pruned SYRK with the back permutation.
int launch_group_syrk(const sc_ctx &c, int w, int v, const double *Y, void *ws, double *F, void *stream) {
  const auto &G = c.waves[w];
  if (v == 0) {
    if (G.syrk[0][1] > 0) {
      PlanPtrs p = c.ptrs();
      p.syrk_tasks += G.syrk[0][0];
      const int n = (int)G.syrk[0][1];
      if (c.persistent) {
        unsigned *q = reinterpret_cast<unsigned *>(static_cast<uint8_t *>(ws) + c.ws.status_off + 128);
        cudaError_t e = cudaMemsetAsync(q, 0, sizeof(unsigned), S(stream));
        if (e != cudaSuccess) return (int)e;
        const int grid = std::min(n, resident_ctas(syrk_kernel));
        syrk_kernel<<<(unsigned)grid, kThreads, 0, S(stream)>>>(p, Y, F, q, n);
      } else {
        syrk_kernel<<<(unsigned)n, kThreads, 0, S(stream)>>>(p, Y, F, nullptr, n);
      }
    }
    return (int)cudaGetLastError();
  }
  const int S = var_digits(v);
  int e = launch_yslice_group(c, S, G.sblk[v][0], G.sblk[v][1], Y, ws, stream, (v & kVarTile) != 0);
  if (e) return e;
  if (v & kVarTile) return launch_syrk_tc(c, S, G.syrk[v][0], G.syrk[v][1], ws, F, stream);
  return launch_syrk_split(c, S, G.syrk[v][0], G.syrk[v][1], ws, F, stream);
}

int launch_apply(const sc_ctx &c, const double *F, const double *lam, double *q, void *stream) {
  if (c.n_apply > 0) apply_kernel<<<(unsigned)c.n_apply, kThreads, 0, S(stream)>>>(c.ptrs(), F, lam, q);
  return (int)cudaGetLastError();
}

int launch_export(const sc_ctx &c, const double *F, int32_t i, double *dst, int32_t ld, void *stream) {
  const int64_t total = (int64_t)c.m[i] * c.m[i];
  if (total > 0) {
    int64_t blocks = (total + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    export_kernel<<<(unsigned)blocks, 256, 0, S(stream)>>>(c.ptrs().subs, i, F, dst, ld);
  }
  return (int)cudaGetLastError();
}

}  // namespace sc
