// Host-side context of one specification, shared by the single-problem driver
// (lsyn_api.cu) and the batch driver (lsyn_batch.cu).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "lsyn.h"
#include "lsyn_internal.h"

namespace lsyn {

struct Alloc {
  lsyn_alloc_fn alloc = nullptr;
  lsyn_free_fn free = nullptr;
  void* user = nullptr;
  std::vector<void*> owned;
  void* get(size_t bytes) {
    if (bytes == 0) bytes = 16;
    void* p = nullptr;
    if (alloc) {
      p = alloc(bytes, user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    if (p) owned.push_back(p);
    return p;
  }
  void release_all() {
    for (void* p : owned) {
      if (free) free(p, user);
      else cudaFree(p);
    }
    owned.clear();
  }
};

// Bit reversal within a word: the ABI numbers positions from the least
// significant bit (bit t = position t); inside the library position 0 is the
// most significant bit, as the paper writes characteristic sequences.
inline uint32_t rev32(uint32_t x) {
  x = ((x >> 1) & 0x55555555u) | ((x & 0x55555555u) << 1);
  x = ((x >> 2) & 0x33333333u) | ((x & 0x33333333u) << 2);
  x = ((x >> 4) & 0x0F0F0F0Fu) | ((x & 0x0F0F0F0Fu) << 4);
  x = ((x >> 8) & 0x00FF00FFu) | ((x & 0x00FF00FFu) << 8);
  return (x >> 16) | (x << 16);
}

inline uint64_t rev64(uint64_t x) { return (uint64_t(rev32(uint32_t(x))) << 32) | rev32(uint32_t(x >> 32)); }

inline void reverse_words(void* data, size_t n_words, int word_bits) {
  if (word_bits == 32) {
    uint32_t* w = static_cast<uint32_t*>(data);
    for (size_t i = 0; i < n_words; ++i) w[i] = rev32(w[i]);
  } else {
    uint64_t* w = static_cast<uint64_t*>(data);
    for (size_t i = 0; i < n_words; ++i) w[i] = rev64(w[i]);
  }
}

struct Snap {
  DevCounters c;
};


// The plan of one level: the unary launch (rows of level k-1) and the binary
// splits, with the operand bytes each reads.
struct LevelPlan {
  uint32_t start = 0;            // first id of the new level
  uint32_t uops = 0;             // unary operators (bit 0 not, 1 X, 2 F, 3 G)
  uint32_t u_first = 0, u_count = 0;
  BinaryPlan plan;               // splits of the binary operators (plan.n_splits may be 0)
  double op_bytes_unary = 0, op_bytes_binary = 0;
  double cand_unary = 0;         // candidates the unary launch builds when it runs to the end
};

// Language-cache sizing for a byte budget: the hash-table capacity (a power of
// two, at most `load` of it in use) and the arena entries that fit beside it.
// Per entry the cache holds the CM (M bytes), its provenance (8), its table
// slot (4) and its hash's low word (4). Returns false if fewer than 64 fit.
bool cache_sizing(unsigned long long cache_bytes, size_t M, double load, unsigned long long* table_cap,
                  unsigned long long* entries);
constexpr size_t kEntryMetaBytes = 16;

// Hole moves: the id ranges [x, y) reserved in [start, total) but left unused
// by warps; returns the level's dense end and the (src, dst) moves that fill
// the holes below it with the entries above it.
uint32_t plan_hole_moves(const uint2* holes, unsigned n, uint32_t start, uint32_t total, std::vector<uint2>* mv);

}  // namespace lsyn

struct lsyn_ctx {
  using Alloc = lsyn::Alloc;
  using Snap = lsyn::Snap;
  using DevCounters = lsyn::DevCounters;
  using CacheView = lsyn::CacheView;
  int device = 0;
  cudaStream_t stream = nullptr;
  Alloc mem;
  uint32_t op_mask = LSYN_OPS_ALL;
  bool full_levels = false;
  bool timing = false;
  bool borrowed = false;   // owned by a batch or server: not driven or destroyed through the handle
  bool owns_host = false;  // h_snap / h_fbuf / h_fstatus are this context's pinned buffers
  double table_load = 0.5;
  unsigned tile_rows = 0;      // forced block-tile rows of the 512-byte binary launch (0: automatic)
  double time_limit_ms = 0;    // lsyn_solve's time limit (0: none)
  double solve_deadline_ms = 0;  // host clock (now_ms) at which the running lsyn_solve's limit passes (0: none)
  unsigned long long level_budget_ns = 0;  // the running level's time budget (CacheView::time_budget_ns)
  bool needs_reset = false;    // a level was interrupted by the time limit: only lsyn_reset helps
  // problem
  int n_props = 0, n_pos = 0, n_neg = 0, T = 0, word_bits = 32, max_len = 1, steps = 0;
  unsigned vecs = 0;
  unsigned planes = 1, plane_vecs = 0;  // words per trace, vectors per plane
  int path = 0;
  int sms = 1;
  // device memory
  uint4* arena = nullptr;
  unsigned long long* prov = nullptr;
  unsigned long long* table = nullptr;  // the table in use (the front table or the big one)
  unsigned long long table_cap = 0;
  // The front table: after a reset the first levels use a small table
  // (kFrontSlots slots, held in L2) while the big table, sized for the whole
  // cache, is cleared on a side stream; before the first level whose
  // candidates could load the front table past table_load the big table's
  // clear is joined and the entries are re-inserted into it.
  static constexpr unsigned long long kFrontSlots = 1ull << 20;
  unsigned long long* big_table = nullptr;
  unsigned long long big_cap = 0;
  unsigned long long* front_table = nullptr;
  unsigned long long front_cap = 0;  // 0: no front table (the big table is small)
  bool front_active = false;         // `table` is the front table
  bool big_clear_pending = false;    // the side stream's clear of the big table is not joined yet
  cudaStream_t side = nullptr;
  cudaEvent_t ev_side[2] = {};       // 0: the main stream reached the reset; 1: the big table is clear
  unsigned max_entries = 0;
  DevCounters* ctr = nullptr;
  uint4* consts = nullptr;  // [5][vecs]: lenmask, label, care, key, mul
  uint4* atoms = nullptr;   // [n_props][vecs]
  unsigned long long* defer[2] = {nullptr, nullptr};
  unsigned defer_cap = 0;
  unsigned* slotpos = nullptr;  // [max_entries]
  unsigned* homes = nullptr;    // [max_entries]
  uint2* holes = nullptr;       // [hole_cap]
  unsigned hole_cap = 0;
  uint2* moves = nullptr;       // [move_cap]
  unsigned* hole_bits = nullptr;  // [3 x hole_cap + 32] scratch of the device hole plan
  unsigned move_cap = 0;
  unsigned chunk = 1;
  char* fbuf = nullptr;
  int* fstatus = nullptr;
  static constexpr unsigned kFormulaCap = 1u << 16;
  // host mirrors
  Snap* h_snap = nullptr;  // pinned, kSnaps entries
  static constexpr int kSnaps = 80;
  char* h_fbuf = nullptr;  // pinned formula text
  int* h_fstatus = nullptr;
  std::vector<uint32_t> level_start, level_n;  // indexed by level
  int levels_done = 0;
  bool last_incomplete = false;
  unsigned long long constructed = 0;
  unsigned long long last_sol = ~0ull;
  cudaEvent_t ev[2 * 80] = {};
  bool events_ready = false;
  std::string err;

  lsyn_status fail(lsyn_status s, const std::string& msg) {
    err = msg;
    return s;
  }
  lsyn_status cuda_fail(cudaError_t e, const char* where) {
    err = std::string(where) + ": " + cudaGetErrorString(e);
    return LSYN_E_CUDA;
  }
  CacheView view(unsigned long long* defer_out, unsigned* defer_out_n) const {
    CacheView cv;
    cv.arena = arena;
    cv.prov = prov;
    cv.table = table;
    cv.table_mask = table_cap - 1;
    cv.max_entries = max_entries;
    cv.vecs = vecs;
    cv.ctr = ctr;
    cv.lenmask = consts;
    cv.label = consts + vecs;
    cv.care = consts + 2 * vecs;
    cv.hkey = consts + 3 * vecs;
    cv.hmul = consts + 4 * vecs;
    cv.atoms = atoms;
    cv.defer_out = defer_out;
    cv.defer_out_n = defer_out_n;
    cv.defer_cap = defer_cap;
    cv.slotpos = slotpos;
    cv.homes = homes;
    cv.holes = holes;
    cv.hole_cap = hole_cap;
    cv.chunk = chunk;
    cv.steps = steps;
    cv.early_exit = full_levels ? 0 : 1;
    cv.planes = planes;
    cv.plane_vecs = plane_vecs;
    cv.time_budget_ns = level_budget_ns;
    cv.kind = lsyn::kKindOther;
    return cv;
  }
};


namespace lsyn {
// Create a context; warp_layout forces whole warps of 16-byte vectors (the
// batch kernels need it).
lsyn_status ctx_create(const lsyn_problem* problem, const lsyn_config* config, bool warp_layout, lsyn_ctx** out);
// Validate a problem and fill a context's layout and sizing (max_entries and
// table_cap follow cache_bytes as in ctx_create) without device memory; the
// padded constants and atom rows are packed into `consts` / `atoms` if given.
lsyn_status ctx_shell(const lsyn_problem* problem, const lsyn_config* config, bool warp_layout, lsyn_ctx** out,
                      std::vector<uint32_t>* consts, std::vector<uint32_t>* atoms);
// Candidates level k builds given the sizes of levels 1..k-1 (sizes[i-1]).
int64_t level_candidate_count(const lsyn_ctx* c, int k);
// The plan of level k (= levels_done + 1); also sets the id chunk size.
void ctx_level_plan(lsyn_ctx* c, int k, LevelPlan* lp);
// Record level k from its final counters (after deferred passes and fixup):
// total = the dense end of the arena. Fills the level fields of `out`.
lsyn_status ctx_commit_level(lsyn_ctx* c, int k, const DevCounters& h, uint32_t total, unsigned long long deferred,
                             const LevelPlan& lp, lsyn_level_stats* out);
// Write the formula of descriptor *root_ptr (device) into out.
lsyn_status ctx_reconstruct(lsyn_ctx* c, const unsigned long long* root_ptr, char* out, size_t cap);
// Formula text of n descriptors in one launch: item i (device array) names a
// provenance array and the device word holding the root descriptor; its text
// goes to buf + i * cap (device), status[i] = 0 if it fit.
struct FormulaItem {
  const unsigned long long* prov;
  const unsigned long long* root;
};
// Clear the per-level counters (as the start of lsyn_enumerate_level does).
cudaError_t launch_level_begin(DevCounters* c, cudaStream_t stream);
cudaError_t reconstruct_many(const FormulaItem* items, int n, char* buf, unsigned cap, int* status,
                             cudaStream_t stream);
double now_ms();
}  // namespace lsyn
