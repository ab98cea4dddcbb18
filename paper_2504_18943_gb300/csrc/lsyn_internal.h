// Internal declarations shared by the host driver (lsyn_api.cu) and the
// kernel translation units (kernels_w32.cu, kernels_w64.cu).
#pragma once

#include <cstdint>
#include <string>
#include <cuda_runtime.h>

namespace lsyn {

// This thread's message for lsyn_last_error(NULL).
std::string& thread_error();

// Operator codes stored in provenance records.
enum : uint32_t {
  kAtom = 0, kNot = 1, kAnd = 2, kOr = 3, kNext = 4, kFuture = 5, kGlobally = 6, kUntil = 7
};

// A candidate is named by a 64-bit descriptor: op in bits 60..63, the left
// child's cache id (or the proposition, for atoms) in bits 30..59 and the right
// child's id in bits 0..29. Cache ids therefore stay below 2^30.
constexpr uint32_t kIdBits = 30;
constexpr uint32_t kIdMask = (1u << kIdBits) - 1u;
constexpr uint32_t kMaxEntries = (1u << kIdBits) - 2u;

__host__ __device__ inline uint64_t pack_desc(uint32_t op, uint32_t left, uint32_t right) {
  return (uint64_t(op) << 60) | (uint64_t(left & kIdMask) << 30) | uint64_t(right & kIdMask);
}
__host__ __device__ inline uint32_t desc_op(uint64_t d) { return uint32_t(d >> 60); }
__host__ __device__ inline uint32_t desc_left(uint64_t d) { return uint32_t(d >> 30) & kIdMask; }
__host__ __device__ inline uint32_t desc_right(uint64_t d) { return uint32_t(d) & kIdMask; }

// Hash-table slot: 0 = empty; otherwise tag (high 32 bits of the CM hash) in
// the high word and, in the low word, id + 1 of a published entry, or one of:
constexpr uint32_t kSlotPending = 0xFFFFFFFFu;  // claimed, CM not yet published
constexpr uint32_t kSlotTomb = 0xFFFFFFFEu;     // claimed, but the arena was full

// Device-side counters of one context. The fields from `level_begin` on are
// cleared at the start of every level.
// Device counters of one language cache. Fields are grouped by how they are
// used into 128-byte lines of their own: every warp bumps the id counter, polls
// the flags and (rarely) appends to the deferred list, and operations on one
// line are served one after another at one L2 slice, so a flag that shared the
// counter's line waited behind its atomics.
// Kinds of launch whose counts are kept apart: the unary and the binary
// operators of a level, and everything else (atoms, deferred re-examination,
// the batch kernels).
constexpr int kLaunchKinds = 4;
constexpr unsigned kKindUnary = 0, kKindBinary = 1, kKindOther = 2;

struct alignas(128) DevCounters {
  // ---- the id counter (an atomic per warp chunk) ----
  unsigned int n_entries;        // arena fill (may exceed max_entries when full)
  unsigned int pad0[31];
  // ---- flags polled by every warp, written rarely ----
  unsigned long long sol;        // smallest descriptor of a separating candidate
  unsigned int level_begin;      // marker (unused)
  unsigned int full;             // an insert found the arena full
  unsigned int solved;           // a separating candidate was found (early exit flag)
  unsigned int error;            // internal consistency codes (probe overflow, hole log)
  unsigned long long t0;         // the GPU's global timer (ns) when the level began
  unsigned int timed_out;        // a kernel stopped because the level's time budget was spent
  unsigned int pad1[23];
  // ---- deferred lists and the hole log ----
  unsigned int defer_n[2];       // deferred-list fills (ping-pong)
  unsigned int defer_overflow;   // a deferred list overflowed: exactness lost
  unsigned int holes_n;          // id ranges reserved but left unused (hole log fill)
  unsigned int pad2[28];
  // ---- per-level totals (an atomic per warp at exit) and the hole plan ----
  // Split by the kind of launch that counted them (CacheView::kind), so that
  // one read of the counters after a level gives every launch's share.
  unsigned long long built_k[kLaunchKinds];     // candidates built in this level
  unsigned long long inserted_k[kLaunchKinds];  // new entries written in this level
  unsigned int moves_n;          // hole moves planned on the device (k_hole_plan)
  unsigned int pad3[15];
  __host__ __device__ unsigned long long built() const {
    unsigned long long t = 0;
    for (int i = 0; i < kLaunchKinds; ++i) t += built_k[i];
    return t;
  }
  __host__ __device__ unsigned long long inserted() const {
    unsigned long long t = 0;
    for (int i = 0; i < kLaunchKinds; ++i) t += inserted_k[i];
    return t;
  }
  // ---- tile counters of the persistent launches ----
  unsigned long long work[8];
  unsigned int pad4[16];
};
static_assert(sizeof(DevCounters) == 640, "DevCounters: five 128-byte lines");

// Everything a kernel needs to probe, compare and insert (passed by value).
struct CacheView {
  uint4* arena;                  // [max_entries][vecs]
  unsigned long long* prov;      // [max_entries] descriptors
  unsigned long long* table;     // [table_mask + 1] slots
  unsigned long long table_mask;
  unsigned int max_entries;
  unsigned int vecs;             // 16-byte vectors per CM (padded)
  DevCounters* ctr;
  const uint4* lenmask;          // [vecs]: bits 0..len-1 of every trace word
  const uint4* label;            // [vecs]: bit 0 = 1 for positive traces
  const uint4* care;             // [vecs]: bit 0 = 1 for real (not padding) traces
  const uint4* hkey;             // [vecs]: per-32-bit-word hash keys
  const uint4* hmul;             // [vecs]: per-32-bit-word odd hash multipliers
  const uint4* atoms;            // [n_props][vecs]
  unsigned long long* defer_out; // deferred descriptors written by this launch
  unsigned int* defer_out_n;
  unsigned int defer_cap;
  unsigned int* slotpos;         // [max_entries]: table slot of each entry (for hole fixup)
  unsigned int* homes;           // [max_entries]: low 32 bits of each entry's hash (table rebuilds)
  uint2* holes;                  // [hole_cap]: unused id ranges [x, y) left by warps
  unsigned int hole_cap;
  unsigned int chunk;            // ids a warp reserves per counter update (path B)
  int steps;                     // log-step count: 2^steps >= longest trace (at most the word width)
  int early_exit;                // 1: stop at the first separating candidate
  unsigned int planes;           // words per trace: plane j holds positions [j w, (j + 1) w) of every trace
  unsigned int plane_vecs;       // vectors of one plane (vecs = planes x plane_vecs, then padding)
  unsigned long long time_budget_ns;  // 0: none; else stop once the global timer passes ctr->t0 + this
  unsigned int kind;             // which DevCounters::built_k / inserted_k this launch counts into
};

// One split {i, j} of level k (i + j = k - 1) for the binary operators.
struct Split {
  uint32_t left_start, left_n;   // rows of the smaller level (staged operand)
  uint32_t right_start, right_n; // rows of the other level (streamed operand)
  uint32_t tri;                  // 1 when both sides are the same level: pairs a < b only (pairs = n(n-1)/2)
  uint32_t lt_tiles, rt_tiles;   // tiles along each side (k_binary_small_c: chunks of 8 rows, row groups)
  uint32_t group;                // k_binary_small_c: rows of the small side per work item
  unsigned long long tiles_begin;
  unsigned long long pairs_begin;
  unsigned long long pairs;
};

constexpr int kMaxSplits = 32;

struct BinaryPlan {
  int n_splits;
  uint32_t ops;                  // bit 0 and, bit 1 or, bit 2 U(a,b), bit 3 U(b,a)
  uint32_t tile;                 // rows per tile side (512-byte CMs: k_binary_c)
  uint32_t tile_fixed;           // 1: keep `tile` at every level (no halving at small levels)
  uint32_t work_slot;            // which DevCounters::work counter to use
  unsigned long long total_tiles;
  unsigned long long total_pairs;
  Split s[kMaxSplits];
};

// One problem of a batch level step (device array, built by the host per step).
constexpr int kBatchSplits = 8;  // binary splits of one level: levels up to 17

struct StepProblem {
  CacheView cv;
  uint32_t u_first, u_count, u_ops;        // unary work: rows of level k-1
  uint32_t b_ops, n_splits;                // binary work: splits of level k
  uint32_t d_n;                            // descriptor work: list length (atoms: n_props)
  const unsigned long long* d_list;        // NULL: implicit atom descriptors 0..d_n-1
  unsigned long long u_items_begin;        // prefix over problems, in work items
  unsigned long long b_items_begin;
  unsigned long long d_items_begin;
  Split s[kBatchSplits];
};

// Header of a batch step: item totals read by the persistent kernels, so one
// captured graph serves every step.
// The work-item counters (bumped by every warp) and the totals (read by every
// warp) each have a 128-byte line of their own, as in DevCounters.
struct alignas(128) StepHeader {
  unsigned long long total_u, total_b, total_d;
  int n;                       // problems in this step
  int rows;                    // unary rows / binary pairs per work item (2, 4 or 8)
  int pad0[24];
  struct alignas(128) Counter {
    unsigned long long v;
    unsigned long long pad[15];
  } work[3];                   // work-item counters: descriptors, unary, binary
};
static_assert(sizeof(StepHeader) == 512, "StepHeader: four 128-byte lines");

// Launch parameters chosen by the host.
struct LaunchCfg {
  cudaStream_t stream;
  int sms;                       // multiprocessor count
};

// Kernel launchers, instantiated for W = uint32_t and uint64_t.
template <typename W>
struct Kernels {
  // Path selection: returns 0 if vecs is not supported.
  static int path_for(unsigned vecs);
  // Level 1 (implicit descriptors ATOM 0..n-1) or a deferred list.
  static cudaError_t desc_list(const CacheView& cv, const unsigned long long* list,
                               const unsigned int* list_n, unsigned int list_cap,
                               unsigned int implicit_atoms, const LaunchCfg& lc);
  static cudaError_t unary(const CacheView& cv, uint32_t first, uint32_t count, uint32_t ops,
                           const LaunchCfg& lc);
  static cudaError_t binary(const CacheView& cv, const BinaryPlan& plan, const LaunchCfg& lc);
  // Batch step (problems at their own levels; all use whole warps of vectors):
  // reset counters, then descriptor (atoms / deferred), unary and binary work.
  static cudaError_t batch_begin(StepHeader* hdr, const StepProblem* steps, int n, const LaunchCfg& lc);
  // vpt: 16-byte vectors a lane loads together in the loops over a CM above 128 bytes (1 or 2).
  static cudaError_t batch_run(StepHeader* hdr, const StepProblem* steps, const LaunchCfg& lc, int blocks_per_sm,
                               int vpt);
  // Moves (problem index, src, dst) of a batch step; then each problem's entry count.
  static cudaError_t batch_fixup(const StepProblem* steps, const uint4* moves, unsigned n, const unsigned* dense_end,
                                 int n_problems, const LaunchCfg& lc);
  // Rebuild a table into a cleared one (new_cap slots, a power of two) from
  // the entries below live_end; error receives 4 if the new table overflows.
  static cudaError_t rehash(const unsigned long long* old_t, unsigned long long old_cap, unsigned long long* new_t,
                            unsigned long long new_cap, const unsigned* homes, unsigned* slotpos, unsigned live_end,
                            unsigned* error, const LaunchCfg& lc);
  // Move entries src -> dst (pairs), repointing their table slots.
  static cudaError_t fixup(const CacheView& cv, const uint2* moves, unsigned n, const LaunchCfg& lc);
  // Plan the hole moves of the level starting at id `start` on the device
  // (sets ctr->moves_n, ctr->n_entries = the dense end, ctr->holes_n = 0) and
  // run them; no host round trip. `bits` is scratch of 3 x hole_cap + 32 words.
  static cudaError_t close_holes(const CacheView& cv, unsigned start, unsigned* bits, uint2* moves, unsigned move_cap,
                                 const LaunchCfg& lc);
  // Evaluate a postorder node list on every trace word of every plane:
  // scratch [n_nodes][planes][plane words]; a CM of planes x plane_vecs vectors.
  static cudaError_t eval(const uint4* atoms, const uint4* lenmask, unsigned plane_vecs, unsigned planes,
                          const int4* nodes, int n_nodes, int steps, W* scratch, W* out, const LaunchCfg& lc);
};

}  // namespace lsyn
