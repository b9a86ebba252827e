// sc_apply_digits (include/sc.h): q = sum_i scatter_i(F_i gather_i(lambda))
// on the tensor cores, from a digit form of F made once per assembly (paper
// Eq. "dualop_apply_expl", the product every solver iteration repeats).
//
// Digit form (sc_apply_digits_prepare).  Every stored 32x32 tile T of F is
// cut to fixed point against its largest exponent, M = round(T 2^(54 - E_T))
// with |T| < 2^E_T, so |M| <= 2^54, and M is written in seven balanced
// base-256 digits d_0 .. d_6 in [-128, 127] (M = sum_k d_k 256^(6-k)), one
// offset-binary byte (d + 128) each.  For one digit the four bytes of a 2x2
// block of entries (rows 2R, 2R+1; columns 2C, 2C+1) share a 32-bit word, so
// that one byte permute forms the pair of entries an MMA fragment holds for
// either direction of the symmetric product.  7184 bytes per tile against
// 8192 in FP64.
//
// Apply.  Per call every 32-entry block l of lambda_i is cut the same way
// (L = round(l 2^(54 - E_l)), digits w_0 .. w_6) and laid out as the B
// operands of the MMAs: for digit k of T, B_k[c][j] = w_(j-k)(c), so that the
// chain of m16n8k16 MMAs over k = 0..6 leaves in column j the integer
//   D_j = sum_(k+e=j) sum_c d_k(., c) w_e(c),  |D_j| <= 7 * 32 * 2^14 < 2^22,
// exactly, in FP32 (classes j <= 7; the classes j >= 8 lie below 2^-56 of
// the tile's scale and are dropped).  The T digits enter as FP16 subnormals
// (offset-binary byte b -> b 2^-24, a byte permute with a zero byte); the
// offset's contribution 128 sum_c w is removed in the conversion to integer,
// v + 1.5 * 2^23 in one FMA.  Rows: y_I += T l_J; columns (off-diagonal
// tiles): y_J += T^T l_I, from the same words.  The classes are combined
// exactly in 64-bit integers, V = sum_j D_j 256^(5-j) (the last two classes
// truncated to units of 2^-16), and converted once:
//   T l = 2^(E_T + E_l - 52) V.
// The error is that of holding each tile and lambda block in 55 bits against
// their largest entries, below 2^-49 of 32 max|T| max|l| per row and tile,
// the size of an FP64 GEMV's rounding.
//
// Tiles are streamed in storage order: each pair of warps takes a contiguous
// range of tiles and copies tile and lambda_J digits into its shared-memory
// ring with 16-byte asynchronous copies (kStages deep); one warp of the pair
// forms the rows (kept in registers over the current row block), the other
// the columns (added atomically per tile), both from the same stage.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <string>

#include "sc_internal.h"

using namespace sc;

namespace {

constexpr uint32_t kFull = 0xffffffffu;
constexpr int kDigitsF = 7;
constexpr int kPlaneWords = 256;                                // 16 x 16 words per digit plane
constexpr int kTileBytes = kDigitsF * kPlaneWords * 4 + 16;     // planes + header (biased e_max)
constexpr int kLamRows = 14;                                    // lambda digit rows e = -6 .. 7
constexpr int kLamCjOff = kLamRows * 32 * 2;                    // class constants after the digit rows
constexpr int kLamBytes = kLamCjOff + 8 * 4 + 16;               // + class constants + header (biased e_max)
constexpr int kStageBytes = kTileBytes + kLamBytes;
constexpr int kPairs = 8;                                       // warp pairs per CTA (one CTA per SM)
constexpr int kStages = 3;                                      // ring depth per pair
constexpr int kPrepWarps = 4;                                   // prepare: 7 KB of shared memory per warp
constexpr int kLamWarps = 8;
static_assert(kTileBytes % 16 == 0 && kLamBytes % 16 == 0, "16-byte copies");

// word of block (R, C) in a digit plane: rows of 16 words, the column index
// XOR-swizzled by bits 1 and 2 of R so that both access patterns of the
// apply (rows: R = g + 8mb, C = t + 4q; columns: R = t + 4q, C = g + 8mb;
// g = lane / 4, t = lane % 4) hit 32 distinct banks
__host__ __device__ __forceinline__ int widx(int R, int C) { return 16 * R + (C ^ (((R & 2) << 2) | (R & 4))); }

__device__ __forceinline__ int biased_exp(double x) { return (int)((__double_as_longlong(x) >> 52) & 0x7FF); }

// round(x 2^(1076 - emax)) for |x| < 2^(emax - 1022): |M| <= 2^54
__device__ __forceinline__ long long fixed55(double x, int emax) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  int e = (int)((b >> 52) & 0x7FF);
  unsigned long long mant = b & ((1ull << 52) - 1);
  if (e) mant |= 1ull << 52;
  else e = 1;
  const int sh = e + 1 - emax;                 // <= 1
  unsigned long long m;
  if (sh >= 0) m = mant << sh;
  else if (sh > -60) m = (mant + (1ull << (-sh - 1))) >> (-sh);
  else m = 0;
  return (b >> 63) ? -(long long)m : (long long)m;
}

// balanced base-256 digits of M (|M| <= 2^54), most significant first, in
// offset binary: ob[k] = d_k + 128
__device__ __forceinline__ void digits7(long long M, int (&d)[kDigitsF]) {
#pragma unroll
  for (int k = kDigitsF - 1; k >= 0; --k) {
    const int v = (int)((M + 128) & 255) - 128;
    d[k] = v;
    M = (M - v) >> 8;
  }
}

// 2^e as a double, also outside the normal range
__device__ __forceinline__ double pow2(int e) {
  if (e >= -1022 && e <= 1023) return __longlong_as_double((long long)(e + 1023) << 52);
  return ldexp(1.0, e);
}

__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
  uint32_t r;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(sel));
  return r;
}

__device__ __forceinline__ void mma_f16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                        uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// ---------------------------------------------------------------------------
// Digit form of F: one warp per tile; lane r holds row r.
__global__ void __launch_bounds__(kPrepWarps * 32) digits_prepare_kernel(const double *__restrict__ F,
                                                                        unsigned char *__restrict__ Fd,
                                                                        int64_t n_tiles) {
  __shared__ __align__(16) uint32_t wsm[kPrepWarps][kDigitsF * kPlaneWords];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t tile = (int64_t)blockIdx.x * kPrepWarps + warp;
  if (tile >= n_tiles) return;
  const double *T = F + tile * 1024;
  double x[32];
  int e = 0;
#pragma unroll
  for (int c = 0; c < 32; ++c) {
    x[c] = T[c * 32 + lane];
    e = max(e, biased_exp(x[c]));
  }
  const int emax = (int)__reduce_max_sync(kFull, (unsigned)e);
  const int R = lane >> 1, odd = lane & 1;
#pragma unroll
  for (int C = 0; C < 16; ++C) {
    int d0[kDigitsF], d1[kDigitsF];
    digits7(fixed55(x[2 * C], emax), d0);
    digits7(fixed55(x[2 * C + 1], emax), d1);
    // this row's bytes of columns 2C, 2C+1 for each digit, two digits per 32-bit word
    uint32_t h[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int k0 = 2 * p, k1 = 2 * p + 1;
      const uint32_t lo = (uint32_t)(d0[k0] + 128) | ((uint32_t)(d1[k0] + 128) << 8);
      const uint32_t hi = k1 < kDigitsF ? ((uint32_t)(d0[k1] + 128) | ((uint32_t)(d1[k1] + 128) << 8)) : 0u;
      h[p] = lo | (hi << 16);
    }
    uint32_t o[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) o[p] = __shfl_xor_sync(kFull, h[p], 1);
    if ((C & 1) == odd) {
      // even row's bytes (2R, 2C), (2R, 2C+1) and odd row's (2R+1, 2C), (2R+1, 2C+1)
#pragma unroll
      for (int k = 0; k < kDigitsF; ++k) {
        const int p = k >> 1, s = (k & 1) * 16;
        const uint32_t ev = ((odd ? o[p] : h[p]) >> s) & 0xFFFFu;
        const uint32_t ov = ((odd ? h[p] : o[p]) >> s) & 0xFFFFu;
        wsm[warp][k * kPlaneWords + widx(R, C)] = prmt(ev, ov, 0x5140);   // x00 x10 x01 x11
      }
    }
  }
  __syncwarp();
  uint4 *dst = reinterpret_cast<uint4 *>(Fd + tile * kTileBytes);
  const uint4 *src = reinterpret_cast<const uint4 *>(&wsm[warp][0]);
  for (int i = lane; i < kDigitsF * kPlaneWords / 4; i += 32) dst[i] = src[i];
  if (lane == 0) dst[kDigitsF * kPlaneWords / 4] = make_uint4((uint32_t)emax, 0u, 0u, 0u);
}

// ---------------------------------------------------------------------------
// Lambda blocks: one warp per apply task (sub, I), block I of lambda_i.
// Entry: 14 rows of 16 FP16 pairs, row r = digit e + 6 (rows of e outside
// 0..6 are zero, so that the digit g - k of class column g and F digit k is
// a plain row index); pair C = (entries 2C, 2C + 1) at position
// 4 (C mod 4) + C / 4 of its row, so that the four pairs C = t, 4 + t, 8 + t,
// 12 + t a lane needs per digit are one 16-byte load; then float cj[8]
// (class constants 1.5 * 2^23 - 128 S_j), int e_max (biased), padding.
// The same launch zeroes q (the product kernel adds into it).
__global__ void __launch_bounds__(kLamWarps * 32) digits_lambda_kernel(const PlanPtrs P, int64_t n_tasks,
                                                                      const double *__restrict__ lam,
                                                                      unsigned char *__restrict__ tab,
                                                                      double *__restrict__ q, int64_t n_dual) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_dual; i += (int64_t)gridDim.x * blockDim.x)
    q[i] = 0.0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t task = (int64_t)blockIdx.x * kLamWarps + warp;
  if (task >= n_tasks) return;
  const ApplyTask at = P.apply_tasks[task];
  const SubDev sd = P.subs[at.sub];
  const int row = at.I * 32 + lane;
  const double v = row < sd.m ? lam[P.lambda[sd.col_off + row]] : 0.0;
  const int emax = (int)__reduce_max_sync(kFull, (unsigned)biased_exp(v));
  int w[kDigitsF];
  digits7(fixed55(v, emax), w);
  unsigned char *ent = tab + task * kLamBytes;
  __half *wt = reinterpret_cast<__half *>(ent);
  const int C = lane >> 1, pos = 2 * (4 * (C & 3) + (C >> 2)) + (lane & 1);
#pragma unroll
  for (int r = 0; r < kLamRows; ++r) {
    const int e = r - 6;
    wt[r * 32 + pos] = __int2half_rn(e >= 0 && e < kDigitsF ? w[e] : 0);
  }
  // S_j = sum over the digits e with 0 <= j - e <= 6 of sum_c w_e(c)
  int colsum[kDigitsF];
#pragma unroll
  for (int e = 0; e < kDigitsF; ++e) colsum[e] = (int)__reduce_add_sync(kFull, (unsigned)w[e]);
  if (lane < 8) {
    int S = 0;
#pragma unroll
    for (int e = 0; e < kDigitsF; ++e)
      if (lane - e >= 0 && lane - e < kDigitsF) S += colsum[e];
    reinterpret_cast<float *>(ent + kLamCjOff)[lane] = 12582912.0f - 128.0f * (float)S;
  }
  if (lane == 0) reinterpret_cast<int *>(ent + kLamCjOff + 32)[0] = emax;
}

// the first tile of apply task k (storage order: subdomain, row block I, J = 0..I)
__device__ __forceinline__ int64_t task_tile0(const PlanPtrs &P, int64_t k) {
  const ApplyTask a = P.apply_tasks[k];
  return P.subs[a.sub].F_off / 1024 + (int64_t)a.I * (a.I + 1) / 2;
}

// exact integer of an FP32 accumulator (subnormal-offset form) for class constant c
__device__ __forceinline__ int acc_int(float d, float c) {
  return __float_as_int(__fmaf_rn(d, 16777216.0f, c)) - 0x4B400000;
}

// combine the classes of the outputs held as (class 2t, class 2t + 1) of
// four outputs rho = 2 mb + h, sum over the four lanes t of a quad, and leave
// in lane t the integer V = sum_j D_j 256^(5-j) of output rho = t
__device__ __forceinline__ long long class_sum(const float (&d)[2][4], float c0, float c1, int t) {
  long long v[4];
#pragma unroll
  for (int mb = 0; mb < 2; ++mb) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int p = acc_int(d[mb][2 * h], c0) * 256 + acc_int(d[mb][2 * h + 1], c1);
      v[2 * mb + h] = t < 3 ? ((long long)p << (16 * (2 - t))) : (long long)(p >> 16);
    }
  }
  const bool hi2 = (t & 2) != 0;
  long long k0 = hi2 ? v[2] : v[0], k1 = hi2 ? v[3] : v[1];
  const long long s0 = hi2 ? v[0] : v[2], s1 = hi2 ? v[1] : v[3];
  k0 += __shfl_xor_sync(kFull, s0, 2);
  k1 += __shfl_xor_sync(kFull, s1, 2);
  const bool hi1 = (t & 1) != 0;
  long long k = hi1 ? k1 : k0;
  const long long s = hi1 ? k0 : k1;
  k += __shfl_xor_sync(kFull, s, 1);
  return k;
}

struct TileCursor {
  int64_t task;
  int sub, I, J, m;
  __device__ __forceinline__ void load(const PlanPtrs &P) {
    const ApplyTask a = P.apply_tasks[task];
    sub = a.sub;
    I = a.I;
    m = P.subs[a.sub].m;
  }
  __device__ __forceinline__ void next(const PlanPtrs &P) {
    if (++J > I) {
      ++task;
      J = 0;
      load(P);
    }
  }
};

__device__ __forceinline__ void mbar_init(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar));
}

// bounded wait for the completion of phase `parity` of an mbarrier
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long limit) {
  uint32_t done = 0;
  for (long long it = 0; it < limit; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// tile `tile` and the lambda block of task `lam_entry` into a stage: two bulk
// copies completing on the stage's mbarrier (one thread)
__device__ __forceinline__ void fetch_stage(uint32_t stage, uint32_t bar, const unsigned char *Fd,
                                            const unsigned char *tab, int64_t tile, int64_t lam_entry) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(kStageBytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   stage),
               "l"(Fd + tile * kTileBytes), "r"(kTileBytes), "r"(bar)
               : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   stage + kTileBytes),
               "l"(tab + lam_entry * kLamBytes), "r"(kLamBytes), "r"(bar)
               : "memory");
}

// The product.  Warps come in pairs sharing a shared-memory ring of kStages
// tiles (each with its lambda_J block), filled by bulk copies that one
// thread of the pair issues: the even warp of a pair forms the row sums
// T l_J, the odd warp the column sums T^T l_I of the same tiles.  Both wait
// for a stage's mbarrier and meet at the pair's named barrier (tile n
// landed, both warps done with tile n - 1), after which the stage of tile
// n - 1 is refilled.  Every mbarrier wait is bounded by poll_limit polls;
// one that gives up sets the timeout bit of *status, the pair stops, waits
// (bounded) for its copies in flight and returns.
__global__ void __launch_bounds__(kPairs * 64, 1) apply_digits_kernel(const PlanPtrs P, int64_t n_tasks,
                                                                     int64_t n_tiles,
                                                                     const unsigned char *__restrict__ Fd,
                                                                     const unsigned char *__restrict__ tab,
                                                                     double *__restrict__ q,
                                                                     uint32_t *__restrict__ status,
                                                                     long long poll_limit) {
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ __align__(8) uint64_t mbar[kPairs][kStages];
  __shared__ int abort_flag[kPairs];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int pair = warp >> 1, half = warp & 1;    // half 0: rows, 1: columns
  const int g = lane >> 2, t = lane & 3;
  const bool issuer = half == 0 && lane == 0;
  const uint32_t ring = smem_u32(dsm + (size_t)pair * kStages * kStageBytes);
  const uint32_t bar0 = smem_u32(&mbar[pair][0]);
  const int64_t np = (int64_t)gridDim.x * kPairs, gp = (int64_t)blockIdx.x * kPairs + pair;
  const int64_t t0 = n_tiles * gp / np, t1 = n_tiles * (gp + 1) / np;
  if (t0 >= t1) return;                           // uniform over the pair
  if (issuer) {
    for (int s = 0; s < kStages; ++s) mbar_init(bar0 + 8 * s);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    abort_flag[pair] = 0;
  }
  asm volatile("bar.sync %0, 64;\n" ::"r"(1 + pair) : "memory");
  int64_t lo = 0, hi = n_tasks - 1;               // the task holding tile t0
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) / 2;
    if (task_tile0(P, mid) <= t0) lo = mid;
    else hi = mid - 1;
  }
  TileCursor cur{lo, 0, 0, 0, 0};
  cur.load(P);
  cur.J = (int)(t0 - task_tile0(P, lo));
  TileCursor pre = cur;                           // the next tile to fetch (issuing warp)
  const int64_t ntile = t1 - t0;
  if (half == 0) {
    for (int s = 0; s < kStages - 1 && s < ntile; ++s) {
      if (issuer) fetch_stage(ring + s * kStageBytes, bar0 + 8 * s, Fd, tab, t0 + s, pre.task - pre.I + pre.J);
      if (s + 1 < ntile) pre.next(P);             // only within the range: the next task exists
    }
  }
  // output of this lane after the class combination: row / column 16 (t >> 1) + 2 g + (t & 1) of the tile
  const int myrow = 16 * (t >> 1) + 2 * g + (t & 1);
  // word offsets (in words) of this lane's four blocks per digit plane:
  // rows: R = 8 mb + g, C = 8 kb + 4 h + t; columns: R = 8 kb + 4 h + t, C = 8 mb + g
  int woff[2][2];                                 // [kb][h] (rows) or [mb][h] (columns), before + 128 mb / kb
#pragma unroll
  for (int x = 0; x < 2; ++x)
#pragma unroll
    for (int h = 0; h < 2; ++h) woff[x][h] = half ? widx(4 * h + t, 8 * x + g) : widx(g, 8 * x + 4 * h + t);
  double yrow = 0.0;
  uint4 bI[kDigitsF];                             // columns: B fragments of lambda_I
  float cI0 = 0.f, cI1 = 0.f;
  int eI = 0;
  auto load_lamI = [&](int64_t task) {
    const unsigned char *ent = tab + task * kLamBytes;
#pragma unroll
    for (int k = 0; k < kDigitsF; ++k) bI[k] = reinterpret_cast<const uint4 *>(ent)[(g - k + 6) * 4 + t];
    const float *cj = reinterpret_cast<const float *>(ent + kLamCjOff);
    cI0 = cj[2 * t];
    cI1 = cj[2 * t + 1];
    eI = reinterpret_cast<const int *>(ent + kLamCjOff + 32)[0];
  };
  if (half) load_lamI(cur.task);
  int s = 0;
  uint32_t phase = 0;
  int64_t n = 0;
  bool aborted = false;
  for (; n < ntile; ++n) {
    if (!mbar_wait(bar0 + 8 * s, phase, poll_limit)) abort_flag[pair] = 1;
    // tile n landed; both warps are done with tile n - 1
    asm volatile("bar.sync %0, 64;\n" ::"r"(1 + pair) : "memory");
    if (*(volatile int *)&abort_flag[pair]) {
      aborted = true;
      break;
    }
    const int sp = s == 0 ? kStages - 1 : s - 1;  // the stage of tile n - 1: refill with tile n + kStages - 1
    if (half == 0 && n + kStages - 1 < ntile) {
      if (issuer) fetch_stage(ring + sp * kStageBytes, bar0 + 8 * sp, Fd, tab, t0 + n + kStages - 1,
                              pre.task - pre.I + pre.J);
      if (n + kStages < ntile) pre.next(P);
    }
    const unsigned char *stage = dsm + (size_t)pair * kStages * kStageBytes + (size_t)s * kStageBytes;
    const uint32_t *pw = reinterpret_cast<const uint32_t *>(stage);
    const int eT = reinterpret_cast<const int *>(stage + kDigitsF * kPlaneWords * 4)[0];
    const bool offdiag = cur.J < cur.I;
    float d[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
    if (half == 0) {
      // rows: A[m][kappa] = T digits, M rows (g, g+8) = tile rows (2R, 2R+1), R = 8 mb + g;
      // K pairs (2t, 2t+1) / (2t+8, 2t+9) = tile columns of C = 8 kb + t / 8 kb + 4 + t
      const unsigned char *lj = stage + kTileBytes;
      const uint4 *wj = reinterpret_cast<const uint4 *>(lj);
#pragma unroll
      for (int k = 0; k < kDigitsF; ++k) {
        const uint32_t *pk = pw + k * kPlaneWords;
        const uint4 b = wj[(g - k + 6) * 4 + t];   // pairs C = t, 4 + t, 8 + t, 12 + t
#pragma unroll
        for (int mb = 0; mb < 2; ++mb) {
#pragma unroll
          for (int kb = 0; kb < 2; ++kb) {
            const uint32_t w0 = pk[woff[kb][0] + 128 * mb], w1 = pk[woff[kb][1] + 128 * mb];
            mma_f16(d[mb], prmt(w0, 0u, 0x4240), prmt(w0, 0u, 0x4341), prmt(w1, 0u, 0x4240),
                    prmt(w1, 0u, 0x4341), kb ? b.z : b.x, kb ? b.w : b.y);
          }
        }
      }
      const float *cj = reinterpret_cast<const float *>(lj + kLamCjOff);
      const int eJ = reinterpret_cast<const int *>(lj + kLamCjOff + 32)[0];
      const long long V = class_sum(d, cj[2 * t], cj[2 * t + 1], t);
      yrow = fma((double)V, pow2(eT + eJ - 2096), yrow);
    } else if (offdiag) {
      // columns: A'[m][kappa] = T^T digits, M rows (g, g+8) = tile columns (2C, 2C+1), C = 8 mb + g;
      // K pairs = tile rows of R = 8 kb + t / 8 kb + 4 + t
#pragma unroll
      for (int k = 0; k < kDigitsF; ++k) {
        const uint32_t *pk = pw + k * kPlaneWords;
#pragma unroll
        for (int mb = 0; mb < 2; ++mb) {
#pragma unroll
          for (int kb = 0; kb < 2; ++kb) {
            const uint32_t w0 = pk[woff[mb][0] + 128 * kb], w1 = pk[woff[mb][1] + 128 * kb];
            mma_f16(d[mb], prmt(w0, 0u, 0x4140), prmt(w0, 0u, 0x4342), prmt(w1, 0u, 0x4140),
                    prmt(w1, 0u, 0x4342), kb ? bI[k].z : bI[k].x, kb ? bI[k].w : bI[k].y);
          }
        }
      }
      const long long V = class_sum(d, cI0, cI1, t);
      const int col = 32 * cur.J + myrow;
      if (col < cur.m) atomicAdd(q + P.lambda[P.subs[cur.sub].col_off + col], (double)V * pow2(eT + eI - 2096));
    }
    if (++s == kStages) {
      s = 0;
      phase ^= 1u;
    }
    const bool last = n + 1 == ntile;
    const int sub = cur.sub, I = cur.I, m = cur.m;
    if (!last) cur.next(P);
    if (last || cur.J == 0) {
      // the row block is complete (or this pair's range ends in it)
      if (half == 0) {
        const int row = 32 * I + myrow;
        if (row < m) atomicAdd(q + P.lambda[P.subs[sub].col_off + row], yrow);
        yrow = 0.0;
      } else if (!last) {
        load_lamI(cur.task);
      }
    }
  }
  if (aborted && issuer) {
    atomicOr(status, kStatusTimeout);
    // copies in flight: tiles n .. min(ntile, n + kStages - 1) - 1; their
    // waits keep at least the default bound whatever poll_limit is, so that
    // no copy still lands in this CTA's shared memory after it returns
    const long long drain = poll_limit > (1LL << 26) ? poll_limit : (1LL << 26);
    for (int64_t j = n; j < ntile && j < n + kStages - 1; ++j)
      mbar_wait(bar0 + 8 * (int)(j % kStages), (uint32_t)((j / kStages) & 1), drain);
  }
}

sc_status check_digits(sc_ctx *ctx, const void *Fd, const char *who) {
  if (!ctx) return SC_ERR_INVALID_ARG;
  if (!ctx->plan_dev && !ctx->blob.empty()) return fail(ctx, SC_ERR_STATE, "sc_upload_plan was not called");
  if (ctx->sizes.F_doubles > 0 && !Fd) return fail(ctx, SC_ERR_INVALID_ARG, std::string(who) + ": Fd_dev is NULL");
  if (Fd && (reinterpret_cast<uintptr_t>(Fd) & 15u))
    return fail(ctx, SC_ERR_INVALID_ARG, std::string(who) + ": Fd_dev is not 16-byte aligned");
  return SC_OK;
}

int64_t digit_tiles(const sc_ctx *ctx) { return ctx->sizes.F_doubles / 1024; }

// buffer: digit tiles | lambda scratch (one entry per apply task) | status word (16 bytes)
int64_t status_offset(const sc_ctx *ctx) { return digit_tiles(ctx) * kTileBytes + ctx->n_apply * kLamBytes; }

}  // namespace

extern "C" sc_status sc_apply_digits_size(const sc_ctx *ctx, int64_t *bytes) {
  if (!ctx || !bytes) return SC_ERR_INVALID_ARG;
  *bytes = status_offset(ctx) + 16;
  return SC_OK;
}

extern "C" sc_status sc_apply_digits_prepare(sc_ctx *ctx, const double *F_dev, void *Fd_dev, void *stream) {
  if (sc_status s = check_digits(ctx, Fd_dev, "sc_apply_digits_prepare")) return s;
  if (ctx->sizes.F_doubles > 0 && !F_dev) return fail(ctx, SC_ERR_INVALID_ARG, "F_dev is NULL");
  const int64_t nt = digit_tiles(ctx);
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(static_cast<unsigned char *>(Fd_dev) + status_offset(ctx), 0, 16, st);
  if (e == cudaSuccess && nt > 0) {
    digits_prepare_kernel<<<(unsigned)((nt + kPrepWarps - 1) / kPrepWarps), kPrepWarps * 32, 0, st>>>(
        F_dev, static_cast<unsigned char *>(Fd_dev), nt);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return fail(ctx, SC_ERR_CUDA, std::string("sc_apply_digits_prepare: ") + cudaGetErrorString(e));
  return SC_OK;
}

extern "C" sc_status sc_apply_digits(sc_ctx *ctx, void *Fd_dev, const double *lambda_dev, double *q_dev,
                                     void *stream) {
  if (sc_status s = check_digits(ctx, Fd_dev, "sc_apply_digits")) return s;
  if (!ctx->has_lambda) return fail(ctx, SC_ERR_STATE, "planned without lambda_map");
  if (ctx->n_dual > 0 && (!lambda_dev || !q_dev)) return fail(ctx, SC_ERR_INVALID_ARG, "lambda_dev or q_dev is NULL");
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t nt = digit_tiles(ctx);
  unsigned char *Fd = static_cast<unsigned char *>(Fd_dev);
  unsigned char *tab = Fd + nt * kTileBytes;
  cudaError_t e = cudaSuccess;
  if (nt == 0) {
    if (ctx->n_dual > 0) e = cudaMemsetAsync(q_dev, 0, sizeof(double) * (size_t)ctx->n_dual, st);
  } else {
    // lambda digits; the same launch zeroes q
    digits_lambda_kernel<<<(unsigned)((ctx->n_apply + kLamWarps - 1) / kLamWarps), kLamWarps * 32, 0, st>>>(
        ctx->ptrs(), ctx->n_apply, lambda_dev, tab, q_dev, ctx->n_dual);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && nt > 0) {
    const int smem = kPairs * kStages * kStageBytes;
    e = cudaFuncSetAttribute(apply_digits_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) {
      int dev = 0, sms = 0;
      e = cudaGetDevice(&dev);
      if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e == cudaSuccess) {
        const int64_t grid = std::min<int64_t>(sms, (nt + kPairs - 1) / kPairs);
        const long long limit = ctx->poll_limit > 0 ? (long long)ctx->poll_limit : (1LL << 26);
        apply_digits_kernel<<<(unsigned)grid, kPairs * 64, smem, st>>>(
            ctx->ptrs(), ctx->n_apply, nt, Fd, tab, q_dev, reinterpret_cast<uint32_t *>(Fd + status_offset(ctx)),
            limit);
        e = cudaGetLastError();
      }
    }
  }
  if (e != cudaSuccess) return fail(ctx, SC_ERR_CUDA, std::string("sc_apply_digits: ") + cudaGetErrorString(e));
  return SC_OK;
}

extern "C" sc_status sc_apply_digits_status(sc_ctx *ctx, void *Fd_dev, void *stream) {
  if (sc_status s = check_digits(ctx, Fd_dev, "sc_apply_digits_status")) return s;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned char *w = static_cast<unsigned char *>(Fd_dev) + status_offset(ctx);
  uint32_t h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, w, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && h) e = cudaMemsetAsync(w, 0, sizeof(h), st);
  if (e != cudaSuccess) return fail(ctx, SC_ERR_CUDA, std::string("sc_apply_digits_status: ") + cudaGetErrorString(e));
  if (h & kStatusTimeout)
    return fail(ctx, SC_ERR_TIMEOUT, "sc_apply_digits: a bounded device wait gave up (sc_options.poll_limit polls)");
  return SC_OK;
}
