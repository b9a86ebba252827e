// Internal plan layout shared by the host planner (sc_plan.cpp), the C ABI
// (sc_api.cu) and the kernels (sc_kernels.cu).
//
// Vocabulary (paper Sec. 3): n dofs, m multipliers (columns of B^T), the column
// pivot of a column is its first nonzero row in L's ordering; columns are
// processed in "sorted" order (by pivot, via the etree postorder rank).  The
// blocks of the factor splitting are the supernodes of L: a supernode s is a
// chain of consecutive columns c0..c0+ns-1 whose patterns below the diagonal
// block coincide; its "pruned rows" R_s (rs of them) are the nonempty rows
// below the diagonal block.  Y restricted to the rows of s is nonzero only on
// the sorted column range [jlo, jhi) and is stored densely there, row-major
// (ns x ws, ws = jhi - jlo).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include "sc.h"

namespace sc {

constexpr int kChunk = 32;      // column chunk width of the TRSM / SYRK tasks
constexpr int kTile = 32;       // F tile edge
constexpr int kThreads = 128;   // threads per CTA of the assembly kernels
constexpr int kGridSMs = 152;   // SMs of a GB300: the round length of the TRSM task order (sc_plan.cpp)

// bits of the workspace status word
enum : uint32_t { kStatusNotSpd = 1u, kStatusTimeout = 2u };

// Per-subdomain kernel variant: 0 = FP64; S (3..7) = split precision with S
// digits and 32x32 SYRK blocks (mma.sync); kVarTile | S = the same digits
// with 128x32 SYRK tiles on tcgen05.  One launch group per variant.
constexpr int kVarTile = 8;
constexpr int kNumVariants = 16;
inline int var_digits(int v) { return v & 7; }

struct SubDev {
  int64_t F_off;     // doubles, start of F_i (tile-packed lower)
  int64_t L_off;     // start of L_i's values in the concatenated value array
  int32_t n, m, nt;  // nt = ceil(m / 32)
  int32_t col_off;   // offset of this subdomain's m entries in perm_cols / lambda
  int32_t lcp_off;   // offset of this subdomain's n entries in lcp / invdiag
  int32_t pad;
};

struct SnDev {
  int64_t y_off;     // doubles, start of Y_s in the Y region
  int64_t rmap_off;  // first entry of this supernode in rmap
  // split precision: first 32-wide row of this supernode in the L digit
  // region; block b (rows kb+kw .. ns+rs-1, kb = 32 b) starts at row
  // ld_off + b (ns + rs) - 16 b (b + 1)
  int64_t ld_off;
  int64_t yd_off;    // split precision: start of Y_s's digits (column-major, rows padded to 32)
  int32_t sub;       // subdomain
  int32_t c0, ns, rs;
  int32_t jlo, jhi;  // sorted column range on which Y_s is nonzero
  int32_t lcp_off;   // global column index of c0 (index into lcp / invdiag)
  int32_t cut_off;   // first entry of this supernode in cuts (one per 32-row block)
};

struct TrsmTask {
  int32_t sub, c_lo, w;       // sorted columns [c_lo, c_lo + w)
  int32_t list_off, list_len; // supernodes touched, ascending (children first)
  int32_t seed_lo, seed_hi;   // seeds of these columns
  int32_t pad;
};

// A 32x32 block of F (sorted chunks q1 >= q2, supernodes active on both), or
// for a tcgen05 variant a 128x32 tile: rows = chunks q1 .. q1 + 3 (q1 a
// multiple of 4), columns = chunk q2, supernodes = the union over its chunk
// pairs on or below the diagonal.
struct SyrkTask {
  int32_t sub, q1, q2;
  int32_t list_off, list_len;
  int32_t pad[3];
};

struct Seed {
  int64_t y_off;  // doubles in the Y region
  double value;   // entry of B^T (+1 / -1)
};

struct ApplyTask {
  int32_t sub, I;
};

// Symbolic analysis of one subdomain (sc_plan.cpp, steps 1-5): validated
// patterns, fundamental supernodes of L and the pivot-sorted B^T columns.
struct SubPlan {
  // supernodes (local)
  std::vector<int32_t> sn_c0, sn_ns, sn_rs, sn_jlo, sn_jhi;
  std::vector<int64_t> sn_rows_off;  // offset of pattern(c0) in L_rowind
  std::vector<int32_t> snode_of;     // column -> supernode
  std::vector<int32_t> sparent;
  std::vector<int32_t> perm_cols;    // sorted -> original column
  // within-supernode pivot cut: columns entering s from below (entry row 0)
  // and columns whose first nonzero on s is at local row e > 0
  std::vector<int32_t> maxq0;
  std::vector<std::vector<std::pair<int32_t, int32_t>>> inner;
};

// Returns an empty string on success, else the reason (prefixed "subdomain idx: ").
// A supernode s is reached (Y is nonzero on it) iff sn_jhi[s] > sn_jlo[s].
std::string analyze(int32_t idx, const sc_subdomain_desc &d, SubPlan &P);

// Device pointers into the uploaded plan blob.
struct PlanPtrs {
  const SubDev *subs;
  const SnDev *sns;
  const int64_t *lcp;        // absolute index of L(c, c) for every column of every subdomain
  const int64_t *rmap;       // per pruned row: Y offset of (row, column jlo of its source supernode)
  const TrsmTask *trsm_tasks;
  const int32_t *trsm_list;
  const SyrkTask *syrk_tasks;
  const int32_t *syrk_list;
  const Seed *seeds;
  const int32_t *perm_cols;  // sorted position -> user column, per subdomain
  const int32_t *lambda;     // user column -> global multiplier, per subdomain
  const ApplyTask *apply_tasks;
  const int32_t *active_cols; // global column indices whose reciprocal diagonal is needed
  const int32_t *cuts;       // per supernode and 32-row block: sorted columns >= cut are zero there
  const int32_t *sblk;       // (active supernode, 32-row block) pairs, for the split-precision packing
};

struct Section {
  size_t off = 0, bytes = 0;
};

// Per-subdomain plan counters, the structural features of the learned variant
// choice (sc_subdomain_features).
struct SubFeat {
  double n, m, nnzL, supernodes, max_supernode, flops_trsm, flops_syrk, flops_dense, y_doubles;
};

// First kHeaderBytes (512) bytes of the plan blob: a self-describing header, so that the
// host copy (sc_export_plan) can be inspected or stored.  Sections follow in
// the order of the arrays below, each 256-byte aligned.
constexpr int kNumSections = 15;
struct PlanHeader {
  uint32_t magic;      // 'SCPL'
  uint32_t version;    // 1
  int32_t nsub;
  int32_t chunk;       // kChunk
  int64_t n_sns, n_trsm, n_syrk, n_apply, n_cols, n_active_cols;
  uint64_t sec_off[kNumSections];   // subs sns lcp rmap trsm trsm_list syrk syrk_list seeds perm lambda apply active cuts sblk
  uint64_t sec_bytes[kNumSections];
};
constexpr size_t kHeaderBytes = 512;
static_assert(sizeof(PlanHeader) <= kHeaderBytes, "plan header must fit its reserved bytes");

// Workspace layout (bytes from ws_dev): [status 256 B][invdiag][Y], and for
// split precision also [column exponents][Y digit planes][L digit planes][L row exponents]
struct WsLayout {
  size_t status_off = 0;
  size_t invd_off = 256;
  size_t y_off = 0;
  size_t colexp_off = 0, yd_off = 0, ld_off = 0, lexp_off = 0;
  int64_t yd_plane = 0;     // elements per Y digit plane
  int64_t ld_rows = 0;      // 32-wide rows per L digit plane
  size_t total = 0;
};

}  // namespace sc

struct sc_ctx {
  std::string err;
  int32_t precision = SC_FP64;       // SC_SPLIT_BF16 when any subdomain runs split
  int32_t n_slices = 0;              // largest digit count of any subdomain (plane sizing)
  std::vector<int8_t> sub_var;       // per subdomain: 0 = FP64, 3..7 = split digits, kVarTile | S = tcgen05 SYRK
  int64_t poll_limit = 0;            // polls of a bounded device wait (0 = default)
  int64_t ws_limit = 0;              // workspace bytes per wave (0 = one wave)
  int32_t persistent = 0;            // FP64 TRSM/SYRK as work-queue kernels (sc_options.persistent)
  // per wave, launch groups by variant (index 0 = FP64, 3..7 = digits): first item, count
  struct WaveGroups {
    int64_t trsm[sc::kNumVariants][2] = {}, syrk[sc::kNumVariants][2] = {}, sblk[sc::kNumVariants][2] = {};
  };
  std::vector<WaveGroups> waves;
  std::vector<int32_t> sub_wave;     // wave of every subdomain
  int32_t nsub = 0;
  int64_t n_dual = 0;
  std::vector<uint8_t> blob;     // plan tables, 256-byte aligned sections
  sc::Section s_subs, s_sns, s_lcp, s_rmap, s_trsm, s_trsm_list, s_syrk, s_syrk_list, s_seeds,
      s_perm, s_lambda, s_apply, s_active, s_cuts, s_sblk;
  int64_t n_sns = 0, n_trsm = 0, n_syrk = 0, n_apply = 0, n_cols = 0, n_active_cols = 0, n_sblk = 0;
  std::vector<int64_t> F_offsets, L_offsets;
  std::vector<sc::SubFeat> sub_feat;    // per subdomain, in batch order
  std::vector<int64_t> diag_index;      // per column of every subdomain: index of L(c, c) in the values
  std::vector<int32_t> n, m;
  sc::WsLayout ws;
  sc_sizes sizes{};
  sc_stats stats{};
  bool has_lambda = true;
  void *plan_dev = nullptr;
  size_t plan_dev_bytes = 0;
  void *stage_events[4] = {nullptr, nullptr, nullptr, nullptr};  // cudaEvent_t, stage timing
  bool stage_recorded = false;
  // created on first use by a batch with several variant groups
  void *aux_streams[sc::kNumVariants] = {}, *aux_done[sc::kNumVariants] = {}, *fork_event = nullptr;
  std::vector<int> groups(int w) const;   // variants present in wave w
  ~sc_ctx();

  sc::PlanPtrs ptrs() const;
};

namespace sc {

sc_status fail(sc_ctx *ctx, sc_status st, const std::string &msg);

// kernel launchers (sc_kernels.cu); return cudaError_t as int
int launch_prep(const sc_ctx &c, const double *Lv, double *invd, uint32_t *status, double *F,
                void *ws, void *stream);
// one variant group (0 = FP64, 3..7 = digits) of wave w: its TRSM half and its SYRK half
int launch_group_trsm(const sc_ctx &c, int w, int v, const double *Lv, const double *invd, void *ws, double *Y,
                      void *stream);
int launch_group_syrk(const sc_ctx &c, int w, int v, const double *Y, void *ws, double *F, void *stream);
// every variant group of wave w: one after the other on `stream`, or (aux, several
// groups) each on its own stream forked from and joined back into `stream`
int launch_groups(sc_ctx &c, int w, const double *Lv, const double *invd, void *ws, double *Y, double *F,
                  void *stream, bool aux);
// split-precision launchers: one variant group of one wave (S digits, items [base, base + count))
int launch_lpack_split(const sc_ctx &c, int S, int64_t base, int64_t count, const double *Lv, void *ws, void *stream);
int launch_trsm_split(const sc_ctx &c, int S, int64_t base, int64_t count, const double *Lv, const double *invd,
                      void *ws, double *Y, void *stream);
int launch_colexp_reset(const sc_ctx &c, void *ws, void *stream);
// balanced: digits in [-128, 128] against twice the column bound (the tcgen05 SYRK's planes)
int launch_yslice_group(const sc_ctx &c, int S, int64_t base, int64_t count, const double *Y, void *ws,
                        void *stream, bool balanced);
int launch_syrk_split(const sc_ctx &c, int S, int64_t base, int64_t count, void *ws, double *F, void *stream);
// the 128x32-tile SYRK on tcgen05 (sc_syrk_tc.cu); tc_smem_bytes: its dynamic shared memory
int launch_syrk_tc(const sc_ctx &c, int S, int64_t base, int64_t count, void *ws, double *F, void *stream);
int tc_smem_bytes(int S);
int launch_apply(const sc_ctx &c, const double *F, const double *lam, double *q, void *stream);
int launch_export(const sc_ctx &c, const double *F, int32_t i, double *dst, int32_t ld, void *stream);

}  // namespace sc
