// sc_apply_fixed (include/sc.h): q = sum_i scatter_i(F_i gather_i(lambda))
// with the multiply-adds on the integer pipes instead of GB300's narrow FP64
// pipe (paper Eq. "dualop_apply_expl", the per-iteration product).
//
// Per 32x32 stored tile T of F_i and 32-entry block l of lambda:
//   * T is cut to 53-bit fixed point against its largest exponent
//     (M = round(T 2^(52-E)), |T| < 2^E, from the FP64 bit pattern with
//     integer operations), l likewise against its own;
//   * each fixed-point value is split into two 27-bit limbs, M = mh 2^27 + ml;
//   * sum_j M_ij L_j = d2 2^54 + d1 2^27 + d0 with d2 = sum mh lh,
//     d1 = sum (mh ll + ml lh), d0 = sum ml ll: 32x32 -> 64-bit multiply-adds,
//     exact (each term < 2^54, 32 terms < 2^60);
//   * d2, d1, d0 are combined in FP64 and scaled by 2^(E_T + E_l - 2094):
//     one rounding per row and tile.
// Every stored tile is read once from HBM and used for both triangles, as in
// the FP64 apply (rows: lane = row over the tile's columns; columns: lane =
// column over its rows, through the shared-memory copy of the tile).  The
// error is that of representing each tile and lambda block in 53 bits
// relative to their largest entry, about 2^-52 of 32 max|T| max|l| per row
// and tile, the size of an FP64 GEMV's rounding.
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "sc_internal.h"

using namespace sc;

namespace {

constexpr uint32_t kFull = 0xffffffffu;

__device__ __forceinline__ uint32_t exp_field(double x) {
  return (uint32_t)(__double_as_longlong(x) >> 52) & 0x7FFu;
}

// round(x 2^(52 - E)) for |x| < 2^E = 2^(exmax - 1022), split into limbs (hi, lo)
__device__ __forceinline__ int2 fixed_limbs(double x, uint32_t exmax) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const uint32_t ex = (uint32_t)(b >> 52) & 0x7FFu;
  int64_t M = 0;
  if (ex != 0) {
    const uint64_t mant = (b & ((1ull << 52) - 1)) | (1ull << 52);
    const uint32_t s = exmax - ex + 1;            // >= 1
    const uint64_t r = s > 63 ? 0ull : (mant + (1ull << (s - 1))) >> s;
    M = (b >> 63) ? -(int64_t)r : (int64_t)r;
  }
  return make_int2((int)(M & ((1ll << 27) - 1)), (int)(M >> 27));   // (ml, mh)
}

// d2 + d1 2^-27 + d0 2^-54, scaled by 2^e
__device__ __forceinline__ double combine(long long d0, long long d1, long long d2, int e) {
  const double v = fma((double)d0, 0x1p-54, fma((double)d1, 0x1p-27, (double)d2));
  if (e >= -1022 && e <= 1023) return v * __longlong_as_double((long long)(e + 1023) << 52);
  return ldexp(v, e);
}

__device__ __forceinline__ void mac(long long &d0, long long &d1, long long &d2, int2 m, int2 l) {
  // all limbs are exact int32 (|mh|, |lh| <= 2^26, ml, ll < 2^27)
  d0 += (long long)m.x * l.x;
  d1 += (long long)m.y * l.x + (long long)m.x * l.y;
  d2 += (long long)m.y * l.y;
}

// fp64_quarters (0..4): of every four tiles a warp visits, this many are
// multiplied in FP64 (FP64 pipe) and the rest in fixed point (integer pipes),
// so that both pipes work at once; 0 is the pure fixed-point product.
__global__ void __launch_bounds__(kThreads, 6) apply_fixed_kernel(const PlanPtrs P, const double *__restrict__ F,
                                                               const double *__restrict__ lam,
                                                               double *__restrict__ q, int fp64_quarters) {
  __shared__ double Ts[kThreads / 32][32][33];     // the tile, then its limbs in place
  __shared__ int2 LJ[kThreads / 32][32];           // limbs of the lambda block J
  __shared__ int2 LI[kThreads / 32][32];           // limbs of the lambda block I
  __shared__ double red[kThreads / 32][32];
  const ApplyTask t = P.apply_tasks[blockIdx.x];
  const SubDev sd = P.subs[t.sub];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int32_t *map = P.lambda + sd.col_off;
  const int I = t.I;
  const int rowI = I * kTile + lane;
  const double pI = rowI < sd.m ? lam[map[rowI]] : 0.0;
  const uint32_t exI = __reduce_max_sync(kFull, exp_field(pI));
  LI[warp][lane] = fixed_limbs(pI, exI);
  int2 *Tl = reinterpret_cast<int2 *>(&Ts[warp][0][0]);
  double y = 0.0;
  for (int J = warp; J <= I; J += kThreads / 32) {
    const double *Tg = F + sd.F_off + ((int64_t)I * (I + 1) / 2 + J) * (kTile * kTile);
    // stage the tile in shared memory (column c, row lane), eight loads in flight
    // at a time, so that no lane keeps the whole tile in registers
    uint32_t em = 0;
#pragma unroll 8
    for (int c = 0; c < 32; ++c) {
      const double v = Tg[c * 32 + lane];
      Ts[warp][c][lane] = v;
      em = max(em, exp_field(v));
    }
    const uint32_t exT = __reduce_max_sync(kFull, em);
    const int colJ = J * kTile + lane;
    const double pJ = colJ < sd.m ? lam[map[colJ]] : 0.0;
    if (((J >> 2) + J) % 4 < fp64_quarters) {     // this tile on the FP64 pipe (uniform across the warp)
      __syncwarp();
#pragma unroll 8
      for (int c = 0; c < 32; ++c) y = fma(Ts[warp][c][lane], __shfl_sync(kFull, pJ, c), y);
      if (J < I) {
        double z = 0.0;
#pragma unroll 8
        for (int r = 0; r < 32; ++r) z = fma(Ts[warp][lane][r], __shfl_sync(kFull, pI, r), z);
        if (colJ < sd.m) atomicAdd(q + map[colJ], z);
      }
      __syncwarp();
      continue;
    }
    const uint32_t exJ = __reduce_max_sync(kFull, exp_field(pJ));
    if (exT == 0) continue;                        // an all-zero tile adds nothing (uniform)
    // each lane converts the entries it staged, in place
#pragma unroll 8
    for (int c = 0; c < 32; ++c) Tl[c * 33 + lane] = fixed_limbs(Ts[warp][c][lane], exT);
    LJ[warp][lane] = fixed_limbs(pJ, exJ);
    __syncwarp();
    // rows: lane = row i of the tile, sum over its columns c
    if (exJ != 0) {
      long long d0 = 0, d1 = 0, d2 = 0;
#pragma unroll 8
      for (int c = 0; c < 32; ++c) mac(d0, d1, d2, Tl[c * 33 + lane], LJ[warp][c]);
      y += combine(d0, d1, d2, (int)exT + (int)exJ - 2094);
    }
    // columns (off-diagonal tiles): lane = column j, sum over the tile's rows r
    if (J < I && exI != 0) {
      long long d0 = 0, d1 = 0, d2 = 0;
#pragma unroll 8
      for (int r = 0; r < 32; ++r) mac(d0, d1, d2, Tl[lane * 33 + r], LI[warp][r]);
      if (colJ < sd.m) atomicAdd(q + map[colJ], combine(d0, d1, d2, (int)exT + (int)exI - 2094));
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

}  // namespace

namespace {

sc_status apply_split(sc_ctx *ctx, const double *F_dev, const double *lambda_dev, double *q_dev, int fp64_quarters,
                      void *stream, const char *who) {
  if (!ctx) return SC_ERR_INVALID_ARG;
  if (!ctx->plan_dev && !ctx->blob.empty()) return fail(ctx, SC_ERR_STATE, "sc_upload_plan was not called");
  if (!ctx->has_lambda) return fail(ctx, SC_ERR_STATE, "planned without lambda_map");
  if (ctx->n_dual > 0 && (!lambda_dev || !q_dev)) return fail(ctx, SC_ERR_INVALID_ARG, "lambda_dev or q_dev is NULL");
  if (ctx->sizes.F_doubles > 0 && !F_dev) return fail(ctx, SC_ERR_INVALID_ARG, "F_dev is NULL");
  if (fp64_quarters < 0 || fp64_quarters > 4) return fail(ctx, SC_ERR_INVALID_ARG, "fp64_quarters must be 0..4");
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSuccess;
  if (ctx->n_dual > 0) e = cudaMemsetAsync(q_dev, 0, sizeof(double) * (size_t)ctx->n_dual, st);
  // the largest shared-memory carve-out, so that six CTAs (37 KB each) fit an SM
  if (e == cudaSuccess && ctx->n_apply > 0)
    e = cudaFuncSetAttribute(apply_fixed_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
  if (e == cudaSuccess && ctx->n_apply > 0) {
    apply_fixed_kernel<<<(unsigned)ctx->n_apply, kThreads, 0, st>>>(ctx->ptrs(), F_dev, lambda_dev, q_dev,
                                                                     fp64_quarters);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return fail(ctx, SC_ERR_CUDA, std::string(who) + ": " + cudaGetErrorString(e));
  return SC_OK;
}

}  // namespace

extern "C" sc_status sc_apply_fixed(sc_ctx *ctx, const double *F_dev, const double *lambda_dev, double *q_dev,
                                    void *stream) {
  return apply_split(ctx, F_dev, lambda_dev, q_dev, 0, stream, "sc_apply_fixed");
}

extern "C" sc_status sc_apply_mixed(sc_ctx *ctx, const double *F_dev, const double *lambda_dev, double *q_dev,
                                    int32_t fp64_quarters, void *stream) {
  return apply_split(ctx, F_dev, lambda_dev, q_dev, fp64_quarters, stream, "sc_apply_mixed");
}
