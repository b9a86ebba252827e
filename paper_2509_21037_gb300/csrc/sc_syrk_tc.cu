// Split-precision pruned SYRK on the fifth-generation tensor cores (tcgen05,
// accumulators in tensor memory), the off-diagonal GEMM work of paper
// Sec. 3.3 with the exact digit slicing of sc_split.cu.
//
// One CTA computes a 128 x 32 tile of F_i in pivot-sorted order: rows are the
// sorted columns j1 of four consecutive 32-column chunks (q1 .. q1 + 3), its
// columns the 32 sorted columns j2 of chunk q2, summed over the supernodes
// active on chunk q2 and on any of the four row chunks, and over those
// supernodes' 32-row blocks that are not cut off for the tile (paper
// Sec. 3.3: only blocks whose inputs are structurally nonzero).
//
// Per 32-row block of Y (K = 32):
//   * the block's digit planes (S planes, 128 + 32 columns, BF16 digits of
//     the FP64 values of Y against per-column exponent bounds) are copied
//     into shared memory in the canonical K-major layout without swizzle
//     (8-row x 16-byte core matrices) by 16-byte asynchronous copies, three
//     stages deep, two blocks ahead of the tensor cores;
//   * one thread issues, for every digit group d = t + t' < S and every pair
//     (t, t'), two tcgen05.mma kind::f16 (M = 128, N = 32, K = 16; BF16 in,
//     FP32 accumulate) into the group's 32 accumulator columns in tensor
//     memory, then tcgen05.commit to an mbarrier;
//   * while the tensor cores run the next block into the other of two
//     accumulator buffers, the eight warps read the finished buffer back
//     (tcgen05.ld; warp w owns tensor-memory lanes 32 (w mod 4) .. and
//     columns 16 (w / 4) ..) and add the exact group sums into 32-bit
//     integers with one FP32 add and one integer add each: the planes hold
//     balanced digits (|digit| <= 128, yslice_kernel), so a group's block sum
//     is an integer below 7 * 32 * 2^14 < 2^22, where FP32 is exact and
//     v + 1.5 * 2^23 puts v in the low mantissa bits; every 256 blocks and at
//     the end the groups are combined exactly in 64-bit integers (Horner) and
//     added to one FP64 value per output.
// The epilogue forms each output with one conversion to FP64 and one scaling
// and writes it in the user's column order, as the mma.sync kernel does.
//
// Every wait on an mbarrier is bounded by `poll_limit` polls; a wait that
// runs out sets the timeout bit of the workspace status word, the CTA stops
// issuing work, waits for its own asynchronous copies, frees its tensor
// memory and returns (sc_device_status then reports SC_ERR_TIMEOUT).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "sc_digits.cuh"
#include "sc_internal.h"

namespace sc {

namespace {

using namespace digits;

constexpr int kTcThreads = 256;   // 8 warps; warps w and w + 4 share tensor-memory lane quarter w % 4
constexpr int kTileM = 128;       // tile rows (sorted columns j1): four chunks
constexpr int kTileN = 32;        // tile columns (sorted columns j2): one chunk
constexpr int kStages = 3;        // shared-memory stages of the digit planes
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kBufCols = 256;  // accumulator buffer stride in tensor-memory columns (S * 32 <= 224)

// Byte offset of element (r, k), r < R, k < 32, of one digit plane of one
// block in the canonical K-major layout without swizzle: two K-slabs of 16
// (one MMA each), each of R/8 row groups of two 8 x 16-byte core matrices.
// LBO (K direction, between the two core matrices of a row group) = 128 B,
// SBO (M/N direction, between row groups) = 256 B.
__host__ __device__ constexpr uint32_t tc_off(int r, int k, int R) {
  return (uint32_t)((k >> 4) * (R * 32) + (r >> 3) * 256 + ((k >> 3) & 1) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor (tcgen05): start, LBO, SBO in 16-byte units,
// descriptor version 1, base offset 0, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(256u >> 4) << 32) |
         ((uint64_t)1 << 46);
}

// instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N = 32 (idesc_n sets other N), M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTileN >> 3) << 17) |
                            ((uint32_t)(kTileM >> 4) << 24);

__device__ __forceinline__ void mma_tc(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

// the instruction descriptor for N columns (M = 128)
__device__ __forceinline__ uint32_t idesc_n(int n) {
  return (kIdesc & ~(0x3Fu << 17)) | ((uint32_t)(n >> 3) << 17);
}

// bounded wait for the completion of phase `parity` of an mbarrier
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long limit) {
  uint32_t done = 0;
  for (long long it = 0; it < limit; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity));
    if (done) return true;
  }
  return false;
}

template <int S>
__global__ void __launch_bounds__(kTcThreads, 1)
    syrk_tc_kernel(const PlanPtrs P, const __nv_bfloat16 *__restrict__ Yd, int64_t yd_plane,
                   const int *__restrict__ colexp, double *__restrict__ F, uint32_t *__restrict__ status,
                   long long poll_limit) {
  // [stage][A: S planes x 128 x 32 | B: S planes x 32 x 32] BF16, canonical layout
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  constexpr uint32_t kAPlane = kTileM * 32 * 2, kBPlane = kTileN * 32 * 2;
  constexpr uint32_t kStageBytes = S * (kAPlane + kBPlane);
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;

  const SyrkTask t = P.syrk_tasks[blockIdx.x];
  const SubDev sd = P.subs[t.sub];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int j1lo = t.q1 * kChunk, j2lo = t.q2 * kChunk;
  const int j1min = max(j1lo, j2lo);      // first row of the tile that is on or below the diagonal
  const uint32_t smem0 = smem_u32(tc_smem);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;\n");
    abort_flag = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  const uint32_t tmem = tmem_base;

  // the active (supernode, 32-row block) pairs in order
  auto advance = [&](int &li, int &k0) -> bool {
    for (;;) {
      k0 += 32;
      while (li < t.list_len && k0 >= P.sns[P.syrk_list[t.list_off + li]].ns) {
        ++li;
        k0 = 0;
      }
      if (li >= t.list_len) return false;
      const SnDev &sn = P.sns[P.syrk_list[t.list_off + li]];
      if (j1min < P.cuts[sn.cut_off + (k0 >> 5)]) return true;
    }
  };
  // 16-byte copies of one block's digit planes into stage `st`: per plane,
  // 128 + 32 columns x 4 chunks of 8 rows; columns outside [jlo, jhi) are zero.
  // Eight consecutive threads take eight consecutive columns of one chunk, so
  // the eight 16-byte stores of a shared-memory wavefront land in distinct
  // banks (their offsets differ in (column mod 8) * 16); the four chunks of a
  // column (64 contiguous bytes of Y's digits) come from the same warp.
  auto fetch = [&](int li, int k0, int st) {
    const SnDev sn = P.sns[P.syrk_list[t.list_off + li]];
    const int npad = (sn.ns + 31) / 32 * 32;
    const uint32_t base = smem0 + (uint32_t)st * kStageBytes;
    constexpr int kPer = (kTileM + kTileN) * 4;      // copies per plane
    for (int v = tid; v < S * kPer; v += kTcThreads) {
      const int d = v / kPer, w = v - d * kPer;
      const int kc = (w >> 3) & 3, col = (w & 7) | ((w >> 5) << 3);
      const bool isA = col < kTileM;
      const int c = isA ? col : col - kTileM;
      const int j = (isA ? j1lo : j2lo) + c - sn.jlo;
      const bool in = j >= 0 && j < sn.jhi - sn.jlo;
      const __nv_bfloat16 *src = in ? Yd + (int64_t)d * yd_plane + sn.yd_off + (int64_t)j * npad + k0 + 8 * kc : Yd;
      // B: per K-slab the S planes one after the other (plane d = rows 32 d .. 32 d + 31 of an
      // S * 32-row operand), so that planes 0 .. S - 1 - t form one K-major operand of
      // 32 (S - t) rows for the MMA of A's plane t
      const uint32_t dst = base + (isA ? (uint32_t)d * kAPlane + tc_off(c, 8 * kc, kTileM)
                                       : (uint32_t)S * kAPlane + tc_off(32 * d + c, 8 * kc, 32 * S));
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(in ? 16 : 0)
                   : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };

  // per thread: tensor-memory lane quarter and its 16 of the tile's 32 columns
  const int quarter = warp & 3, chalf = warp >> 2;
  const int row = 32 * quarter + lane;                        // tile row (j1 - j1lo)
  // Block sums of digit group d are integers of magnitude below 7 * 32 * 2^14 <
  // 2^22 (balanced digits), so v + 1.5 * 2^23 is exact and its bit pattern is
  // 0x4B400000 + v: one FP32 add and one 32-bit integer add per value fold a
  // block into gs (wrapping; the 0x4B400000 per block is taken out at the fold,
  // exact while the true sum stays below 2^31: at most 256 blocks).
  uint32_t gs[S][16];
  double dacc[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    dacc[c] = 0.0;
#pragma unroll
    for (int d = 0; d < S; ++d) gs[d][c] = 0u;
  }
  uint32_t nfold = 0;
  auto fold = [&]() {                      // exact: int64 Horner words, then one FP64 value per output
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      Groups<S> g;
#pragma unroll
      for (int d = 0; d < S; ++d) {
        g.accumulate(d, (int)(gs[d][c] - nfold * 0x4B400000u));
        gs[d][c] = 0u;
      }
      dacc[c] += g.value_wide();
    }
    nfold = 0;
  };

  auto flush = [&](int nb) -> bool {       // fold block nb's accumulators (buffer nb & 1)
    if (!mbar_wait(smem_u32(&mbar[nb & 1]), (uint32_t)((nb >> 1) & 1), poll_limit)) return false;
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    const uint32_t tb = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(nb & 1) * kBufCols + 16 * chalf;
#pragma unroll
    for (int d = 0; d < S; ++d) {
      uint32_t v[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(tb + 32u * d));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
      for (int c = 0; c < 16; ++c) gs[d][c] += __float_as_uint(__uint_as_float(v[c]) + 12582912.0f);
    }
    if (++nfold == 256) fold();
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    return true;
  };

  // Three stages, two blocks in flight ahead of the tensor cores: in iteration
  // nb the MMAs of block nb are issued, block nb - 1 is folded (its MMAs are
  // then complete, so its stage is free) and block nb + 2 is fetched into
  // that stage while block nb + 1's copies finish.  Every iteration commits
  // exactly one copy group (possibly empty), so `wait_group 1` always means
  // "all but the newest group", i.e. block nb + 1.
  int li0 = 0, k00 = -32;
  bool have = advance(li0, k00);
  int li1 = li0, k01 = k00;
  bool h1 = have && advance(li1, k01);
  int li2 = li1, k02 = k01;
  bool h2 = h1 && advance(li2, k02);
  if (have) fetch(li0, k00, 0);
  else asm volatile("cp.async.commit_group;\n" ::: "memory");
  if (h1) fetch(li1, k01, 1);
  else asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 1;\n" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");   // the copies, seen by the tensor cores
  __syncthreads();
  int nb = 0;
  while (have) {
    if (abort_flag) break;
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n");
      const uint32_t st = smem0 + (uint32_t)(nb % kStages) * kStageBytes;
      const uint32_t dbuf = tmem + (uint32_t)(nb & 1) * kBufCols;
      // For A's plane t, one MMA covers every B plane t' < S - t at once: N = 32 (S - t) and the
      // output columns 32 (t + t') of group t + t', i.e. TMEM columns 32 t .. 32 S: 2 S MMAs per block
#pragma unroll
      for (int ta = 0; ta < S; ++ta) {
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
          const uint64_t da = smem_desc(st + (uint32_t)ta * kAPlane + (uint32_t)ks * (kTileM * 32));
          const uint64_t db = smem_desc(st + (uint32_t)S * kAPlane + (uint32_t)ks * (kTileN * S * 32));
          mma_tc(dbuf + 32u * ta, da, db, idesc_n(kTileN * (S - ta)), (ta > 0 || ks > 0) ? 1u : 0u);
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
          smem_u32(&mbar[nb & 1])));
    }
    if (nb >= 1 && !flush(nb - 1)) {
      atomicOr(status, kStatusTimeout);
      abort_flag = 1;
    }
    // stage (nb + 2) % 3 held block nb - 1, whose MMAs this thread has seen complete
    if (h2) fetch(li2, k02, (nb + 2) % kStages);
    else asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    have = h1;
    h1 = h2;
    li1 = li2;
    k01 = k02;
    if (h2) h2 = advance(li2, k02);
    ++nb;
  }
  __syncthreads();
  const bool ok = !abort_flag && (nb == 0 || flush(nb - 1));
  if (!ok && !abort_flag) atomicOr(status, kStatusTimeout);
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols));
  if (!ok || abort_flag) return;

  fold();
  // epilogue: row j1 of the tile, columns j2 = j2lo + 16 chalf + c; the balanced
  // digits were cut against twice each column bound: 2^(Ej + 1) per operand
  const int32_t *perm = P.perm_cols + sd.col_off;
  const int *ce = colexp + sd.col_off;
  const int j1 = j1lo + row;
  if (j1 < sd.m && j1 >= j2lo) {
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const int j2 = j2lo + 16 * chalf + c;
      if (j2 >= sd.m || j1 < j2) continue;
      double v = dacc[c];
      const int e = (ce[j1] + 1 - 1022) + (ce[j2] + 1 - 1022);
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

}  // namespace

int tc_smem_bytes(int S) { return kStages * S * (kTileM + kTileN) * 32 * 2; }

int launch_syrk_tc(const sc_ctx &c, int S_, int64_t base, int64_t count, void *ws, double *F, void *stream) {
  if (count <= 0) return (int)cudaGetLastError();
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint8_t *w = static_cast<uint8_t *>(ws);
  const int *colexp = reinterpret_cast<const int *>(w + c.ws.colexp_off);
  const __nv_bfloat16 *Yd = reinterpret_cast<const __nv_bfloat16 *>(w + c.ws.yd_off);
  uint32_t *status = reinterpret_cast<uint32_t *>(w + c.ws.status_off);
  PlanPtrs p = c.ptrs();
  p.syrk_tasks += base;
  const long long limit = c.poll_limit > 0 ? (long long)c.poll_limit : (1LL << 26);
#define TC(S)                                                                                                     \
  {                                                                                                               \
    const int smem = tc_smem_bytes(S);                                                                            \
    cudaError_t e = cudaFuncSetAttribute(syrk_tc_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);  \
    if (e != cudaSuccess) return (int)e;                                                                          \
    syrk_tc_kernel<S><<<(unsigned)count, kTcThreads, smem, st>>>(p, Yd, c.ws.yd_plane, colexp, F, status, limit); \
  }
  switch (S_) {
    case 3: TC(3); break;
    case 4: TC(4); break;
    case 5: TC(5); break;
    case 6: TC(6); break;
    default: TC(7); break;
  }
#undef TC
  return (int)cudaGetLastError();
}

}  // namespace sc
