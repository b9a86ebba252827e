// Split-precision variants of the off-diagonal GEMM work (sm_103a tensor cores).
//
// The paper runs its TRSM/SYRK blocks as FP64 library calls; on GB300 the FP64
// pipe is ~1.2 TFLOP/s while the BF16 tensor path runs at hundreds of TFLOP/s.
// Here the pruned SYRK (paper Sec. 3.3) is computed with an error-free slicing
// of its FP64 operands (the scheme of Ozaki, Ogita, Oishi and Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59, 2012), adapted
// to 8-bit digits:
//
//   * every column j of the task's Y operand gets one exponent bound 2^Ej over
//     all rows the task reads (|y| < 2^Ej);
//   * |y| 2^-Ej in [0, 1) is cut into S unsigned 8-bit digits u_0..u_{S-1}
//     (y = sign * 2^Ej * sum_t u_t 2^(-8(t+1)) + truncation below 2^(Ej-8S)),
//     taken from the FP64 bit pattern with integer operations only; each
//     signed digit is exactly a BF16 value;
//   * products of digit planes t and t' run on the tensor cores (mma.sync
//     m16n8k16, BF16 in, FP32 accumulate); for one 32-row block the sum over
//     all pairs with t + t' = d is an integer below 7 * 32 * 255^2 < 2^24, so
//     the FP32 accumulator holds it exactly;
//   * the exact block sums are added as int32 (flushed to FP64 every 128
//     blocks), and the output is sum_d I_d 2^(-8(d+2)) * 2^(Ej1 + Ej2) in FP64.
//
// Only pairs with t + t' <= S - 1 are formed (S(S+1)/2 products); the terms
// dropped and the digit truncation are below 2^(-8S) relative to the
// product of the column bounds.  S = 7 keeps 56 bits of every operand.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "sc_internal.h"

namespace sc {

namespace {

constexpr int kPad = 40;   // bf16 row stride of a digit plane (conflict-free fragment loads)

// 2^e exactly, for e in the normal range (built from the bit pattern)
__device__ __forceinline__ double pow2i(int e) { return __longlong_as_double((long long)(e + 1023) << 52); }

__device__ __forceinline__ int biased_exponent(double y) {
  return (int)((__double_as_longlong(y) >> 52) & 0x7FF);
}

// 64-bit fixed point of |y| * 2^-(emax - 1022) * 2^63 (truncated), emax the
// column's largest biased exponent.  Returns 0 for y == 0.
__device__ __forceinline__ uint64_t fixed_point(double y, int emax) {
  const uint64_t bits = (uint64_t)__double_as_longlong(y);
  int e = (int)((bits >> 52) & 0x7FF);
  uint64_t mant = bits & ((1ull << 52) - 1);
  if (e) mant |= (1ull << 52);
  else e = 1;                                   // subnormal: same scale as e = 1
  const int sh = e - emax + 10;                 // <= 10 because e <= emax
  if (sh >= 0) return mant << sh;
  if (sh > -64) return mant >> (-sh);
  return 0;
}

__device__ __forceinline__ __nv_bfloat16 digit_bf16(uint64_t X, int t, bool neg) {
  const int u = (int)((X >> (55 - 8 * t)) & 0xFF);
  return __float2bfloat16_rn(neg ? -(float)u : (float)u);   // |u| <= 255: exact
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t ld_pair(const __nv_bfloat16 *p) {
  return *reinterpret_cast<const uint32_t *>(p);
}

// One 32x32 block of F = Y^T Y (sorted chunks q1 >= q2), split precision.
// Warp w computes rows 16*(w>>1) .. +16 and columns 16*(w&1) .. +16 of the
// block as two m16n8 tiles.
template <int S>
__global__ void __launch_bounds__(kThreads) syrk_split_kernel(const PlanPtrs P, const double *__restrict__ Y,
                                                              double *__restrict__ F) {
  __shared__ __align__(16) __nv_bfloat16 PA[S][32][kPad];   // digit planes of the J1 columns, [t][j][k]
  __shared__ __align__(16) __nv_bfloat16 PB[S][32][kPad];   // digit planes of the J2 columns
  __shared__ int emaxA[32], emaxB[32];
  const SyrkTask t = P.syrk_tasks[blockIdx.x];
  const SubDev sd = P.subs[t.sub];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int j1lo = t.q1 * kChunk, j2lo = t.q2 * kChunk;

  // pass 1: per-column exponent bounds over every row this task reads
  if (tid < 32) { emaxA[tid] = 0; emaxB[tid] = 0; }
  __syncthreads();
  {
    int ma = 0, mb = 0;
    for (int li = 0; li < t.list_len; ++li) {
      const SnDev s = P.sns[P.syrk_list[t.list_off + li]];
      const int ws = s.jhi - s.jlo;
      const double *Ys = Y + s.y_off;
      const int ja = j1lo + lane - s.jlo, jb = j2lo + lane - s.jlo;
      const bool oka = ja >= 0 && ja < ws, okb = jb >= 0 && jb < ws;
      for (int k0 = 0; k0 < s.ns; k0 += 32) {
        if (j1lo >= P.cuts[s.cut_off + (k0 >> 5)]) continue;
        const int kk = min(32, s.ns - k0);
        for (int k = warp; k < kk; k += kThreads / 32) {
          const double *row = Ys + (int64_t)(k0 + k) * ws;
          if (oka) ma = max(ma, biased_exponent(row[ja]));
          if (okb) mb = max(mb, biased_exponent(row[jb]));
        }
      }
    }
    atomicMax(&emaxA[lane], ma);
    atomicMax(&emaxB[lane], mb);
  }
  __syncthreads();

  const int g = lane >> 2, tg = lane & 3;
  const int mrow = 16 * (warp >> 1);            // this warp's rows (J1) in the block
  const int ncol = 16 * (warp & 1);             // this warp's columns (J2): two n8 tiles
  int iacc[S][8];
  double dacc[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    dacc[i] = 0.0;
#pragma unroll
    for (int d = 0; d < S; ++d) iacc[d][i] = 0;
  }
  int blocks = 0;
  for (int li = 0; li < t.list_len; ++li) {
    const SnDev s = P.sns[P.syrk_list[t.list_off + li]];
    const int ws = s.jhi - s.jlo;
    const double *Ys = Y + s.y_off;
    for (int k0 = 0; k0 < s.ns; k0 += 32) {
      if (j1lo >= P.cuts[s.cut_off + (k0 >> 5)]) continue;
      const int kk = min(32, s.ns - k0);
      // slice the 32x32 operands into digit planes (rows k >= kk are zero)
      for (int k = warp; k < 32; k += kThreads / 32) {
        const int ja = j1lo + lane - s.jlo, jb = j2lo + lane - s.jlo;
        double va = 0.0, vb = 0.0;
        if (k < kk) {
          const double *row = Ys + (int64_t)(k0 + k) * ws;
          if (ja >= 0 && ja < ws) va = row[ja];
          if (jb >= 0 && jb < ws) vb = row[jb];
        }
        const uint64_t Xa = fixed_point(va, emaxA[lane]), Xb = fixed_point(vb, emaxB[lane]);
        const bool na = va < 0.0, nb = vb < 0.0;
#pragma unroll
        for (int d = 0; d < S; ++d) {
          PA[d][lane][k] = digit_bf16(Xa, d, na);
          PB[d][lane][k] = digit_bf16(Xb, d, nb);
        }
      }
      __syncthreads();
#pragma unroll
      for (int d = 0; d < S; ++d) {
        float c[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
        for (int ta = 0; ta <= d; ++ta) {
          const int tb = d - ta;
#pragma unroll
          for (int ks = 0; ks < 32; ks += 16) {
            uint32_t a[4];
            a[0] = ld_pair(&PA[ta][mrow + g][ks + 2 * tg]);
            a[1] = ld_pair(&PA[ta][mrow + g + 8][ks + 2 * tg]);
            a[2] = ld_pair(&PA[ta][mrow + g][ks + 2 * tg + 8]);
            a[3] = ld_pair(&PA[ta][mrow + g + 8][ks + 2 * tg + 8]);
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
              const uint32_t b0 = ld_pair(&PB[tb][ncol + 8 * nt + g][ks + 2 * tg]);
              const uint32_t b1 = ld_pair(&PB[tb][ncol + 8 * nt + g][ks + 2 * tg + 8]);
              mma_bf16(c[nt], a, b0, b1);
            }
          }
        }
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
          for (int r = 0; r < 4; ++r) iacc[d][nt * 4 + r] += __float2int_rn(c[nt][r]);
      }
      __syncthreads();
      if (++blocks == 128) {          // int32 headroom: 128 blocks * 1.46e7 < 2^31
        blocks = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          double v = 0.0;
#pragma unroll
          for (int d = 0; d < S; ++d) v += (double)iacc[d][i] * pow2i(-8 * (d + 2));
          dacc[i] += v;
#pragma unroll
          for (int d = 0; d < S; ++d) iacc[d][i] = 0;
        }
      }
    }
  }
  const int32_t *perm = P.perm_cols + sd.col_off;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int nt = i >> 2, r = i & 3;
    const int rl = mrow + g + ((r & 2) ? 8 : 0);              // row in the block (J1)
    const int cl = ncol + 8 * nt + 2 * tg + (r & 1);          // column in the block (J2)
    double v = dacc[i];
#pragma unroll
    for (int d = 0; d < S; ++d) v += (double)iacc[d][i] * pow2i(-8 * (d + 2));
    const int j1 = j1lo + rl, j2 = j2lo + cl;
    if (j1 < sd.m && j2 < sd.m && (t.q1 != t.q2 || j1 >= j2)) {
      const int e = (emaxA[rl] - 1022) + (emaxB[cl] - 1022);
      v = ldexp(v, e);
      const int a = perm[j1], b = perm[j2];
      const int hi = max(a, b), lo = min(a, b);
      const int I = hi / kTile, J = lo / kTile;
      double *T = F + sd.F_off + ((int64_t)I * (I + 1) / 2 + J) * (kTile * kTile);
      T[(hi % kTile) + kTile * (lo % kTile)] = v;
      if (I == J) T[(lo % kTile) + kTile * (hi % kTile)] = v;
    }
  }
}

}  // namespace

int launch_syrk_split(const sc_ctx &c, const double *Y, double *F, void *stream) {
  if (c.n_syrk <= 0) return (int)cudaGetLastError();
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const unsigned grid = (unsigned)c.n_syrk;
  const PlanPtrs p = c.ptrs();
  switch (c.n_slices) {
    case 3: syrk_split_kernel<3><<<grid, kThreads, 0, st>>>(p, Y, F); break;
    case 4: syrk_split_kernel<4><<<grid, kThreads, 0, st>>>(p, Y, F); break;
    case 5: syrk_split_kernel<5><<<grid, kThreads, 0, st>>>(p, Y, F); break;
    case 6: syrk_split_kernel<6><<<grid, kThreads, 0, st>>>(p, Y, F); break;
    default: syrk_split_kernel<7><<<grid, kThreads, 0, st>>>(p, Y, F); break;
  }
  return (int)cudaGetLastError();
}

}  // namespace sc
