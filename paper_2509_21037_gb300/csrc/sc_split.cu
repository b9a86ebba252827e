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
//   * every column j of a subdomain's Y gets one exponent bound 2^Ej over all
//     its rows (|y| < 2^Ej), every row of an L panel block one bound over the
//     block's 32 columns;
//   * |y| 2^-Ej in [0, 1) is cut into S unsigned 8-bit digits u_0..u_{S-1}
//     (y = sign * 2^Ej * sum_t u_t 2^(-8(t+1)) + truncation below 2^(Ej-8S)),
//     taken from the FP64 bit pattern with integer operations only; each
//     signed digit is exactly a BF16 value;
//   * products of digit planes t and t' run on the tensor cores (mma.sync
//     m16n8k16, BF16 in, FP32 accumulate); for one 32-row block the sum over
//     all pairs with t + t' = d is an integer below 7 * 32 * 255^2 < 2^24, so
//     the FP32 accumulator holds it exactly;
//   * the exact block sums are added as int32 (flushed every 128 blocks), the
//     digit groups are combined exactly in 64-bit integers, and the output
//     sum_d I_d 2^(-8(d+2)) * 2^(Ej1 + Ej2) is formed with one conversion to
//     FP64 and one scaling (the FP64 pipe is the scarce resource on GB300).
//
// L and Y are cut into digit planes once per assembly (lpack_kernel after
// the reciprocal diagonal; ycolexp/yslice after the TRSM), so the TRSM and
// SYRK tasks only load BF16 planes.
//
// Only pairs with t + t' <= S - 1 are formed (S(S+1)/2 products); the terms
// dropped and the digit truncation are below 2^(-8S) relative to the
// product of the column bounds.  S = 7 keeps 56 bits of every operand.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "sc_digits.cuh"
#include "sc_internal.h"

namespace sc {

namespace {

using namespace digits;

constexpr int kPad = 40;   // bf16 row stride of a digit plane (conflict-free fragment loads)

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


// Digit planes of L's panel rows below one 32x32 diagonal block (one CTA per
// (supernode, block) item; one thread per panel row, so every CSC column is
// read contiguously).
template <int S>
__global__ void __launch_bounds__(kThreads) lpack_kernel(const PlanPtrs P, const double *__restrict__ Lv,
                                                         __nv_bfloat16 *__restrict__ Ld,
                                                         int16_t *__restrict__ lexp, int64_t ld_rows) {
  const int si = P.sblk[2 * blockIdx.x], b = P.sblk[2 * blockIdx.x + 1];
  const SnDev s = P.sns[si];
  const int64_t *cp = P.lcp + s.lcp_off;
  const int nrow = s.ns + s.rs;
  const int kb = 32 * b, kw = min(32, s.ns - kb);
  const int nb = nrow - kb - kw;
  const int64_t base = s.ld_off + (int64_t)b * nrow - 16LL * b * (b + 1);
  for (int r = threadIdx.x; r < nb; r += kThreads) {
    const int p = kb + kw + r;
    double v[32];
    int e = 0;
#pragma unroll
    for (int q = 0; q < 32; ++q) {
      v[q] = q < kw ? Lv[cp[kb + q] - (kb + q) + p] : 0.0;
      e = max(e, biased_exponent(v[q]));
    }
    lexp[base + r] = (int16_t)e;
    uint64_t X[32];
    uint32_t neg = 0;
#pragma unroll
    for (int q = 0; q < 32; ++q) {
      X[q] = fixed_point(v[q], e);                  // once per entry, not once per digit plane
      neg |= (v[q] < 0.0 ? 1u : 0u) << q;
    }
#pragma unroll
    for (int d = 0; d < S; ++d) {
      // the row's 64 bytes of this plane as four 16-byte stores
      uint4 *row = reinterpret_cast<uint4 *>(Ld + (int64_t)d * ld_rows * 32 + (base + r) * 32);
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        uint32_t w[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          const int q = 8 * g + 2 * h;
          const __nv_bfloat16 lo = digit_bf16(X[q], d, (neg >> q) & 1u);
          const __nv_bfloat16 hi = digit_bf16(X[q + 1], d, (neg >> (q + 1)) & 1u);
          w[h] = (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
        }
        row[g] = make_uint4(w[0], w[1], w[2], w[3]);
      }
    }
  }
}

// Column exponent bounds of Y over one (supernode, 32-row block) item.
__global__ void __launch_bounds__(kThreads) ycolexp_kernel(const PlanPtrs P, const double *__restrict__ Y,
                                                           int *__restrict__ colexp) {
  const int si = P.sblk[2 * blockIdx.x], b = P.sblk[2 * blockIdx.x + 1];
  const SnDev s = P.sns[si];
  const SubDev sd = P.subs[s.sub];
  const int ws = s.jhi - s.jlo;
  const int r0 = 32 * b, r1 = min(s.ns, r0 + 32);
  for (int c = threadIdx.x; c < ws; c += kThreads) {
    int e = 0;
    for (int r = r0; r < r1; ++r) e = max(e, biased_exponent(Y[s.y_off + (int64_t)r * ws + c]));
    if (e) atomicMax(&colexp[sd.col_off + s.jlo + c], e);
  }
}

// Digit planes of Y for one (supernode, 32-row block) item: 32x32 tiles are
// read row-wise (coalesced), transposed in shared memory and written
// column-major (coalesced), rows padded to 32.
// kBalanced (the tcgen05 SYRK's planes): the magnitude is cut against twice the
// column bound (|y| 2^-(Ej + 1) < 1/2, so the top digit is at most 127) and
// recoded into balanced digits in [-128, 128] (least significant first: a
// digit above 127 becomes digit - 256 and carries one into the next), so
// every digit product is at most 2^14 in magnitude.
template <int S, bool kBalanced>
__global__ void __launch_bounds__(kThreads) yslice_kernel(const PlanPtrs P, const double *__restrict__ Y,
                                                          const int *__restrict__ colexp,
                                                          __nv_bfloat16 *__restrict__ Yd, int64_t yd_plane) {
  __shared__ double Ts[32][33];
  const int si = P.sblk[2 * blockIdx.x], b = P.sblk[2 * blockIdx.x + 1];
  const SnDev s = P.sns[si];
  const SubDev sd = P.subs[s.sub];
  const int ws = s.jhi - s.jlo;
  const int npad = (s.ns + 31) / 32 * 32;
  const int r0 = 32 * b;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c0 = 0; c0 < ws; c0 += 32) {
    for (int i = warp; i < 32; i += kThreads / 32) {
      const int r = r0 + i, c = c0 + lane;
      Ts[i][lane] = (r < s.ns && c < ws) ? Y[s.y_off + (int64_t)r * ws + c] : 0.0;
    }
    __syncthreads();
    for (int j = warp; j < 32; j += kThreads / 32) {
      const int c = c0 + j;
      if (c < ws) {
        const double v = Ts[lane][j];
        const int64_t e = s.yd_off + (int64_t)c * npad + r0 + lane;
        if (kBalanced) {
          const uint64_t X = fixed_point(v, colexp[sd.col_off + s.jlo + c] + 1);
          int dig[S];
          int carry = 0;
#pragma unroll
          for (int d = S - 1; d >= 0; --d) {
            int u = (int)((X >> (55 - 8 * d)) & 0xFF) + carry;
            carry = (d > 0 && u >= 128) ? 1 : 0;
            dig[d] = u - 256 * carry;
          }
#pragma unroll
          for (int d = 0; d < S; ++d)
            Yd[(int64_t)d * yd_plane + e] = __float2bfloat16_rn(v < 0.0 ? -(float)dig[d] : (float)dig[d]);
        } else {
          const uint64_t X = fixed_point(v, colexp[sd.col_off + s.jlo + c]);
#pragma unroll
          for (int d = 0; d < S; ++d) Yd[(int64_t)d * yd_plane + e] = digit_bf16(X, d, v < 0.0);
        }
      }
    }
    __syncthreads();
  }
}

// One 32x32 block of F = Y^T Y (sorted chunks q1 >= q2) from Y's digit
// planes.  Warp w computes rows 16*(w>>1).. and columns 16*(w&1).. of the
// block as two m16n8 tiles.
template <int S>
// 4 resident CTAs for up to 5 digits, 3 for 6 and 7 (register-bound fragments)
__global__ void __launch_bounds__(kThreads, (S <= 5 ? 4 : 3)) syrk_split_kernel(const PlanPtrs P, const __nv_bfloat16 *__restrict__ Yd,
                                                              int64_t yd_plane, const int *__restrict__ colexp,
                                                              double *__restrict__ F) {
  // two stages of the digit tiles: [stage][operand][t][column][k]; the next
  // active 32-row block is fetched with asynchronous copies while this one
  // is multiplied
  extern __shared__ __align__(16) unsigned char syrk_smem[];
  typedef __nv_bfloat16 Tile[S][32][kPad];
  Tile *stages = reinterpret_cast<Tile *>(syrk_smem);          // stages[2 * buf + op]
  const SyrkTask t = P.syrk_tasks[blockIdx.x];
  const SubDev sd = P.subs[t.sub];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, tg = lane & 3;
  const int j1lo = t.q1 * kChunk, j2lo = t.q2 * kChunk;
  const int mrow = 16 * (warp >> 1), ncol = 16 * (warp & 1);
  // per output: the Horner words of the digit-group sums, accumulated over
  // blocks (linear, exact: < 128 blocks * 2^24 * 256^(h-1) < 2^63)
  Groups<S> acc[8];
  double dacc[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) dacc[i] = 0.0;
  int blocks = 0;
  // the active (supernode, 32-row block) pairs in order: rows of a supernode
  // at or after its pivot cut for this chunk are zero and skipped
  auto advance = [&](int &li, int &k0) -> bool {
    for (;;) {
      k0 += 32;
      while (li < t.list_len && k0 >= P.sns[P.syrk_list[t.list_off + li]].ns) {
        ++li;
        k0 = 0;
      }
      if (li >= t.list_len) return false;
      const SnDev &sn = P.sns[P.syrk_list[t.list_off + li]];
      if (j1lo < P.cuts[sn.cut_off + (k0 >> 5)]) return true;
    }
  };
  // 2 operands x S planes x 32 columns x 4 vectors of 8 digits, 16 bytes each
  auto fetch = [&](int li, int k0, int buf) {
    const SnDev sn = P.sns[P.syrk_list[t.list_off + li]];
    const int npad = (sn.ns + 31) / 32 * 32;
    for (int v = tid; v < 2 * S * 32 * 4; v += kThreads) {
      const int part = v & 3, col = (v >> 2) & 31, d = (v >> 7) % S, op = (v >> 7) / S;
      const int j = (op == 0 ? j1lo : j2lo) + col - sn.jlo;
      const bool in = j >= 0 && j < sn.jhi - sn.jlo;
      const __nv_bfloat16 *src =
          in ? Yd + (int64_t)d * yd_plane + sn.yd_off + (int64_t)j * npad + k0 + 8 * part : Yd;
      const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&stages[2 * buf + op][d][col][8 * part]);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(in ? 16 : 0)
                   : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  int li = 0, k0 = -32, buf = 0;
  bool have = advance(li, k0);
  if (have) fetch(li, k0, 0);
  while (have) {
    int nli = li, nk0 = k0;
    const bool nhave = advance(nli, nk0);
    if (nhave) {
      fetch(nli, nk0, buf ^ 1);
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");   // this block's copies are done
    } else {
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    }
    __syncthreads();
    const Tile &PA = stages[2 * buf], &PB = stages[2 * buf + 1];
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
          for (int r = 0; r < 4; ++r) acc[nt * 4 + r].accumulate(d, __float2int_rn(c[nt][r]));
      }
      __syncthreads();                // the next iteration's fetch overwrites this stage
      if (++blocks == 128) {          // int64 headroom, see acc
        blocks = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          dacc[i] += acc[i].value_wide();
          acc[i] = Groups<S>();
        }
      }
    li = nli;
    k0 = nk0;
    have = nhave;
    buf ^= 1;
  }
  const int32_t *perm = P.perm_cols + sd.col_off;
  const int *ce = colexp + sd.col_off;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int nt = i >> 2, r = i & 3;
    const int rl = mrow + g + ((r & 2) ? 8 : 0);
    const int cl = ncol + 8 * nt + 2 * tg + (r & 1);
    const int j1 = j1lo + rl, j2 = j2lo + cl;
    if (j1 < sd.m && j2 < sd.m && (t.q1 != t.q2 || j1 >= j2)) {
      double v = dacc[i] + acc[i].value_wide();
      const int e = (ce[j1] - 1022) + (ce[j2] - 1022);
      v = (e >= -1022 && e <= 1023) ? v * pow2i(e) : ldexp(v, e);
      const int a = perm[j1], b = perm[j2];
      const int hi = max(a, b), lo = min(a, b);
      const int I = hi / kTile, J = lo / kTile;
      double *T = F + sd.F_off + ((int64_t)I * (I + 1) / 2 + J) * (kTile * kTile);
      T[(hi % kTile) + kTile * (lo % kTile)] = v;
      if (I == J) T[(lo % kTile) + kTile * (hi % kTile)] = v;
    }
  }
}

// Sparse TRSM of one 32-column chunk with split-precision updates: the 32x32
// diagonal triangles are solved in FP64 by one warp exactly as in the FP64
// path; the update of the panel rows below (L[p, block] X, paper Sec. 3.2's
// pruned GEMM) runs on the tensor cores from digit planes of X (column
// bounds, shared memory) and of L's rows (pre-cut by lpack_kernel), combined
// exactly in integers and subtracted from Y in FP64.
template <int S>
// 6 resident CTAs for up to 4 digits (the TRSM is latency-bound: more warps
// hide the L digit and Y loads), 5 for 5 digits (at 6 its registers spill), 4 for
// 6 and 7 digits (their fragments would spill)
__global__ void __launch_bounds__(kThreads, (S <= 4 ? 6 : S == 5 ? 5 : 4)) trsm_split_kernel(const PlanPtrs P, const double *__restrict__ Lv,
                                                              const double *__restrict__ invd,
                                                              const __nv_bfloat16 *__restrict__ Ld,
                                                              const int16_t *__restrict__ lexp, int64_t ld_rows,
                                                              double *__restrict__ Y) {
  __shared__ double Xs[32][33];
  __shared__ int64_t cps[32];
  __shared__ __align__(16) __nv_bfloat16 PX[S][32][kPad];   // digit planes of X, [t][column][row]
  __shared__ int emaxX[32];
  const TrsmTask t = P.trsm_tasks[blockIdx.x];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, tg = lane & 3;
  const int c_hi = t.c_lo + t.w;
  // the warp that solves the FP64 triangles: spread over the SM's sub-partitions
  // across co-resident CTAs (a hash of the task index; see tri_warp in sc_kernels.cu)
  const int tri = (int)(((unsigned)blockIdx.x * 2654435761u) >> 30);

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
    const int a = max(s.jlo, t.c_lo), b = min(s.jhi, c_hi), ws = s.jhi - s.jlo;
    double *Ys = Y + s.y_off + (a - s.jlo);
    const int64_t *cp = P.lcp + s.lcp_off;
    const double *id = invd + s.lcp_off;
    const int64_t *rm = P.rmap + s.rmap_off;
    const int colsh = a - s.jlo;
    const int nrow = s.ns + s.rs;
    for (int kb = 0, blk = 0; kb < s.ns; kb += 32, ++blk) {
      const int kw = min(32, s.ns - kb);
      const int wk = min(b, P.cuts[s.cut_off + (kb >> 5)]) - a;
      if (wk <= 0) continue;
      const int nb = nrow - (kb + kw);
      const int64_t base = s.ld_off + (int64_t)blk * nrow - 16LL * blk * (blk + 1);
      // the L digit fragments of a warp's first m-tile depend on L only: the
      // warps that do not solve the triangle fetch them while it is solved
      uint32_t afr[S][2][4];
      auto load_afr = [&](int mt) {
        const int ra = mt * 16 + g, rb = ra + 8;
        const bool va = ra < nb, vb = rb < nb;
#pragma unroll
        for (int d = 0; d < S; ++d) {
          const uint32_t *pa = reinterpret_cast<const uint32_t *>(Ld + (int64_t)d * ld_rows * 32 + (base + ra) * 32);
          const uint32_t *pb = reinterpret_cast<const uint32_t *>(Ld + (int64_t)d * ld_rows * 32 + (base + rb) * 32);
#pragma unroll
          for (int ks = 0; ks < 2; ++ks) {
            afr[d][ks][0] = va ? pa[8 * ks + tg] : 0u;
            afr[d][ks][1] = vb ? pb[8 * ks + tg] : 0u;
            afr[d][ks][2] = va ? pa[8 * ks + tg + 4] : 0u;
            afr[d][ks][3] = vb ? pb[8 * ks + tg + 4] : 0u;
          }
        }
      };
      const bool pre = warp != tri && warp * 16 < nb;
      if (pre) load_afr(warp);
      // The FP64 triangle, 8 columns at a time: warp `tri` solves the 8x8
      // diagonal piece, then all four warps update the block's rows below it
      // (one warp alone would hold its sub-partition's FP64 unit for the whole
      // chain of ~kw^2 / 2 instructions while the others wait).  Every entry
      // gets its updates in the same column order as a column-by-column solve.
      if (tid < kw) cps[tid] = cp[kb + tid] - (kb + tid);
      for (int e = tid; e < kw * 32; e += kThreads) {
        const int q = e >> 5, c = e & 31;
        Xs[q][c] = c < wk ? Ys[(int64_t)(kb + q) * ws + c] : 0.0;
      }
      __syncthreads();
      for (int p0 = 0; p0 < kw; p0 += 8) {
        const int pe = min(p0 + 8, kw);
        if (warp == tri && lane < wk) {
          if (pe - p0 == 8) {                 // a full piece: its column of X in registers
            double x[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) x[i] = Xs[p0 + i][lane];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              x[i] *= id[kb + p0 + i];
              const double *Lc = Lv + cps[p0 + i] + kb + p0;
#pragma unroll
              for (int r = i + 1; r < 8; ++r) x[r] = fma(-Lc[r], x[i], x[r]);
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) Xs[p0 + i][lane] = x[i];
          } else {
            for (int q = p0; q < pe; ++q) {
              const double xq = Xs[q][lane] * id[kb + q];
              Xs[q][lane] = xq;
              const double *Lc = Lv + cps[q];
              for (int r = q + 1; r < pe; ++r) Xs[r][lane] = fma(-Lc[kb + r], xq, Xs[r][lane]);
            }
          }
        }
        __syncthreads();
        if (pe < kw) {                        // then pe == p0 + 8
          if (lane < wk) {
            double x[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) x[i] = Xs[p0 + i][lane];
            for (int r = pe + ((warp - tri) & 3); r < kw; r += kThreads / 32) {
              double xr = Xs[r][lane];
#pragma unroll
              for (int i = 0; i < 8; ++i) xr = fma(-Lv[cps[p0 + i] + kb + r], x[i], xr);
              Xs[r][lane] = xr;
            }
          }
          __syncthreads();
        }
      }
      if (warp == tri) {
        int em = 0;
        if (lane < wk) {
          for (int q = 0; q < kw; ++q) {
            Ys[(int64_t)(kb + q) * ws + lane] = Xs[q][lane];
            em = max(em, biased_exponent(Xs[q][lane]));
          }
        }
        emaxX[lane] = em;
      }
      __syncthreads();
      if (nb <= 0) continue;                  // nothing below this block (uniform)
      for (int e = tid; e < 32 * 32; e += kThreads) {
        const int q = e >> 5, c = e & 31;
        const double v = (q < kw && c < wk) ? Xs[q][c] : 0.0;
        const uint64_t X = fixed_point(v, emaxX[c]);
        const bool neg = v < 0.0;
#pragma unroll
        for (int d = 0; d < S; ++d) PX[d][c][q] = digit_bf16(X, d, neg);
      }
      __syncthreads();
      for (int mt = warp; mt * 16 < nb; mt += kThreads / 32) {
        const int r0 = mt * 16;               // first block row of this m-tile
        const int ra = r0 + g, rb = r0 + g + 8;
        const bool va = ra < nb, vb = rb < nb;
        const int ea = va ? lexp[base + ra] : 0, eb = vb ? lexp[base + rb] : 0;
        // this lane's two target rows (a pruned row through its map), looked up once per m-tile
        double *tga = nullptr, *tgb = nullptr;
        if (va) {
          const int p = kb + kw + ra;
          tga = (p < s.ns) ? (Ys + (int64_t)p * ws) : (Y + rm[p - s.ns] + colsh);
        }
        if (vb) {
          const int p = kb + kw + rb;
          tgb = (p < s.ns) ? (Ys + (int64_t)p * ws) : (Y + rm[p - s.ns] + colsh);
        }
        if (!(pre && mt == warp)) load_afr(mt);
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
          if (8 * nt >= wk) break;                   // uniform across the warp
          // the targets' current values, loaded before the products so that
          // their latency overlaps the MMAs
          double yv[4];
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const bool vr = (r & 2) ? vb : va;
            const int col = 8 * nt + 2 * tg + (r & 1);
            yv[r] = (vr && col < wk) ? ((r & 2) ? tgb : tga)[col] : 0.0;
          }
          Groups<S> gr[4];
#pragma unroll
          for (int d = 0; d < S; ++d) {
            float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int ta = 0; ta <= d; ++ta) {
              const int tb = d - ta;
#pragma unroll
              for (int ks = 0; ks < 2; ++ks) {
                const uint32_t b0 = ld_pair(&PX[tb][8 * nt + g][16 * ks + 2 * tg]);
                const uint32_t b1 = ld_pair(&PX[tb][8 * nt + g][16 * ks + 2 * tg + 8]);
                mma_bf16(c, afr[ta][ks], b0, b1);
              }
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) gr[r].add(d, __float2int_rn(c[r]));
          }
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const bool vr = (r & 2) ? vb : va;
            const int col = 8 * nt + 2 * tg + (r & 1);
            if (vr && col < wk) {
              const int e = (((r & 2) ? eb : ea) - 1022) + (emaxX[col] - 1022);
              // one conversion and one FMA on the FP64 pipe: both power-of-two
              // scalings folded into a single exponent
              const double v = (double)gr[r].block_int();
              const int eb = e + Groups<S>::kBlockShift;
              double *tgt = (r & 2) ? tgb : tga;
              if (eb >= -1022 && eb <= 1023) tgt[col] = fma(-v, pow2i(eb), yv[r]);
              else tgt[col] = yv[r] - ldexp(v, eb);
            }
          }
        }
      }
      __syncthreads();
    }
  }
}

}  // namespace

#define SC_SPLIT_SWITCH(S_, CALL) \
  switch (S_) {                   \
    case 3: CALL(3); break;       \
    case 4: CALL(4); break;       \
    case 5: CALL(5); break;       \
    case 6: CALL(6); break;       \
    default: CALL(7); break;      \
  }

int launch_lpack_split(const sc_ctx &c, int S_, int64_t base, int64_t count, const double *Lv, void *ws,
                       void *stream) {
  if (count <= 0) return (int)cudaGetLastError();
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint8_t *w = static_cast<uint8_t *>(ws);
  __nv_bfloat16 *Ld = reinterpret_cast<__nv_bfloat16 *>(w + c.ws.ld_off);
  int16_t *lexp = reinterpret_cast<int16_t *>(w + c.ws.lexp_off);
  PlanPtrs p = c.ptrs();
  p.sblk += 2 * base;
#define LP(S) lpack_kernel<S><<<(unsigned)count, kThreads, 0, st>>>(p, Lv, Ld, lexp, c.ws.ld_rows)
  SC_SPLIT_SWITCH(S_, LP)
#undef LP
  return (int)cudaGetLastError();
}

int launch_trsm_split(const sc_ctx &c, int S_, int64_t base, int64_t count, const double *Lv, const double *invd,
                      void *ws, double *Y, void *stream) {
  if (count <= 0) return (int)cudaGetLastError();
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint8_t *w = static_cast<uint8_t *>(ws);
  const __nv_bfloat16 *Ld = reinterpret_cast<const __nv_bfloat16 *>(w + c.ws.ld_off);
  const int16_t *lexp = reinterpret_cast<const int16_t *>(w + c.ws.lexp_off);
  PlanPtrs p = c.ptrs();
  p.trsm_tasks += base;
#define TS(S) trsm_split_kernel<S><<<(unsigned)count, kThreads, 0, st>>>(p, Lv, invd, Ld, lexp, c.ws.ld_rows, Y)
  SC_SPLIT_SWITCH(S_, TS)
#undef TS
  return (int)cudaGetLastError();
}

int launch_colexp_reset(const sc_ctx &c, void *ws, void *stream) {
  int64_t ncols = 0;
  for (int32_t m : c.m) ncols += m;
  if (ncols <= 0) return 0;
  uint8_t *w = static_cast<uint8_t *>(ws);
  return (int)cudaMemsetAsync(w + c.ws.colexp_off, 0, sizeof(int) * (size_t)ncols, static_cast<cudaStream_t>(stream));
}

int launch_yslice_group(const sc_ctx &c, int S_, int64_t base, int64_t count, const double *Y, void *ws,
                        void *stream, bool balanced) {
  if (count <= 0) return (int)cudaGetLastError();
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint8_t *w = static_cast<uint8_t *>(ws);
  int *colexp = reinterpret_cast<int *>(w + c.ws.colexp_off);
  __nv_bfloat16 *Yd = reinterpret_cast<__nv_bfloat16 *>(w + c.ws.yd_off);
  PlanPtrs p = c.ptrs();
  p.sblk += 2 * base;
  ycolexp_kernel<<<(unsigned)count, kThreads, 0, st>>>(p, Y, colexp);
#define YS(S) yslice_kernel<S, false><<<(unsigned)count, kThreads, 0, st>>>(p, Y, colexp, Yd, c.ws.yd_plane)
#define YB(S) yslice_kernel<S, true><<<(unsigned)count, kThreads, 0, st>>>(p, Y, colexp, Yd, c.ws.yd_plane)
  if (balanced) {
    SC_SPLIT_SWITCH(S_, YB)
  } else {
    SC_SPLIT_SWITCH(S_, YS)
  }
#undef YS
#undef YB
  return (int)cudaGetLastError();
}

int launch_syrk_split(const sc_ctx &c, int S_, int64_t base, int64_t count, void *ws, double *F, void *stream) {
  if (count <= 0) return (int)cudaGetLastError();
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint8_t *w = static_cast<uint8_t *>(ws);
  const int *colexp = reinterpret_cast<const int *>(w + c.ws.colexp_off);
  const __nv_bfloat16 *Yd = reinterpret_cast<const __nv_bfloat16 *>(w + c.ws.yd_off);
  PlanPtrs p = c.ptrs();
  p.syrk_tasks += base;
#define SY(S)                                                                                              \
  {                                                                                                        \
    const int smem = (int)(4 * sizeof(__nv_bfloat16) * S * 32 * kPad);                                     \
    cudaFuncSetAttribute(syrk_split_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);         \
    syrk_split_kernel<S><<<(unsigned)count, kThreads, smem, st>>>(p, Yd, c.ws.yd_plane, colexp, F);        \
  }
  SC_SPLIT_SWITCH(S_, SY)
#undef SY
  return (int)cudaGetLastError();
}

}  // namespace sc
