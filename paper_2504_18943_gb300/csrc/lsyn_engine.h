// The multi-problem scheduler behind lsyn_batch_* and the server.
//
// Jobs (one specification each) wait in a FIFO queue and are admitted into
// slots. Every admitted job advances level by level through the bottom-up
// enumeration (the listing of paragraph "A generic program synthesiser") in
// one of two lanes:
//  * small levels go into batch steps: one persistent launch per word size
//    over a packed work list of every such job, on a high-priority stream;
//    jobs join and leave between steps (continuous batching);
//  * a level with more candidates than the solo threshold runs in the
//    large-level lane: the one-problem kernels on a stream of their own, one
//    job's level after another in admission order, driven by a non-blocking
//    state machine (launch with the first deferred pass and the level's hole
//    close queued behind it; further deferred passes; commit; answer) that
//    the host advances between batch steps. While small levels are in the
//    system the large-level launches leave `light_sms` SMs to them.
//
// Memory. A slot owns growable Segments (lsyn_pool.h) for one language cache:
// CM arena, provenance, table slot and hash word of each entry, two hash
// tables (one is rebuilt into the other when the table must grow), deferred
// lists and the problem's constants. Before each level the scheduler predicts
// the level's new entries from its candidate count and the unique ratio of the
// previous level and grows the arrays to hold them; the table keeps at most
// `table_load` of its slots in use. A job never has more entries than
// lsyn_create would give it for the same cache_bytes, so its levels, status
// and answer size equal the one-problem path's. If a level outgrows the
// prediction (the arena fills below that cap) and no solution settles it, the
// level is undone (the table is rebuilt without its entries) and run again with
// room for every candidate. When the pool cannot hold a job's growth, the job
// waits; if nothing can run, finished caches kept for export are dropped, then
// the youngest admitted jobs are evicted (their caches dropped, the jobs
// queued again) until the oldest fits. A job alone in the pool that still does
// not fit is capped at what the pool gives it (status LSYN_E_CACHE_FULL, noted
// in its error text).
#pragma once

#include <cstdint>
#include <deque>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "lsyn.h"
#include "lsyn_ctx.h"
#include "lsyn_internal.h"
#include "lsyn_pool.h"

namespace lsyn {

struct Job {
  Job() = default;
  Job(const Job&) = delete;
  Job& operator=(const Job&) = delete;
  ~Job() { delete c; }  // a shell: it owns no device memory
  uint64_t ticket = 0;
  int max_size = 0;
  double t_submit = 0, t_admit = 0, t_done = 0;
  uint64_t seq = 0;  // admission order (older first)
  // shell context (layout, level bookkeeping); device pointers point into a slot
  lsyn_ctx* c = nullptr;
  std::vector<uint32_t> consts, atoms;  // packed on the host, uploaded at admission
  unsigned long long cap_entries = 0;   // the one-problem entry limit for cache_bytes
  int slot = -1;
  bool redo = false;                    // re-run the current level with room for every candidate
  bool heavy = false;                   // its next level belongs to the large-level lane
  bool in_flight = false;               // a large level of it is on the GPU
  bool paused = false;                  // its last growth did not fit the pool
  double ratio = 1.0;                   // unique / candidates of the last complete level
  int evictions = 0, redos = 0;
  bool capped = false;
  bool resident = false;                // cache still on the device (export)
  enum State { kQueued, kActive, kDone } state = kQueued;
  // result
  lsyn_status status = LSYN_PENDING;
  int found = 0, size = 0, exact = 0, levels_done = 0;
  int64_t constructed = 0, unique = 0;
  std::string formula, err;
};

class Engine {
 public:
  Engine() = default;
  Engine(const Engine&) = delete;
  Engine& operator=(const Engine&) = delete;
  ~Engine();

  // keep_finished: a finished job keeps its slot and cache (for export) until
  // its memory is needed (batch); otherwise its slot is freed at once (server).
  lsyn_status init(const lsyn_config* cfg, const lsyn_batch_tuning* tune, int max_active, bool keep_finished);
  // Copy and validate a problem into a job (not yet queued). Thread-safe.
  lsyn_status make_job(const lsyn_problem* p, int max_size, Job* j) const;
  void enqueue(Job* j, double t_submit);
  // Admit queued jobs into free slots while the pool can hold their first levels.
  lsyn_status admit();
  // Advance both lanes once. With may_block, waits for the large-level lane
  // when nothing else can move. *progressed says whether anything moved.
  lsyn_status pump(bool may_block, bool* progressed);
  bool busy() const { return !queue_.empty() || !active_.empty(); }
  // A large level is on the GPU (its track waits for an event).
  bool lanes_busy() const;
  // Jobs finished since the last call.
  std::vector<Job*> take_done();
  // Drop every job (queued, active or resident) and free their slots.
  void clear();

  lsyn_batch_tuning tune() const { return tune_; }
  // Applies the launch-shape fields of t (not max_active, pool_bytes, lanes);
  // call between solves, with t checked by valid_tuning.
  void set_tune(const lsyn_batch_tuning& t);
  static bool valid_tuning(const lsyn_batch_tuning& t, std::string* e);
  const BlockPool& pool() const { return pool_; }
  int device() const { return device_; }
  int sm_count() const { return sms_; }
  size_t peak_in_use() const { return peak_; }
  uint64_t steps_run() const { return steps_; }
  uint64_t evictions() const { return evictions_; }
  uint64_t redos() const { return redos_; }
  uint64_t large_levels() const { return large_levels_; }
  int active_count() const { return int(active_.size()); }
  int queued_count() const { return int(queue_.size()); }
  // Step trace (the last kTraceCap batch steps, oldest first).
  static constexpr size_t kTraceCap = 4096;
  std::vector<lsyn_step_trace> trace() const;
  void clear_trace() { trace_.clear(); trace_head_ = 0; }
  std::string err;

 private:
  struct Slot {
    Segment arena, prov, slotpos, homes, misc, defer[2], table[2];
    int cur_table = 0;
    unsigned long long tcap = 0;   // slots of the current table
    bool reserved = false;
    Job* job = nullptr;
  };
  struct Plan {                    // one job's small level in a batch step
    Job* j;
    int k;
    LevelPlan lp;
    unsigned long long deferred = 0;
    int cur = 0;
    uint32_t total = 0;
    bool undo = false;
  };
  // A track of the large-level lane: one level of one job at a time.
  struct Lane {
    enum Stage { kIdle, kRun, kAnswer };
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    Job* j = nullptr;
    Stage stage = kIdle;
    int k = 0;
    LevelPlan lp;
    int cur = 0, passes = 0;
    bool closed = false;           // the holes of every pass so far are closed
    bool first = false;            // the first event of the level has not been handled
    unsigned long long deferred = 0;
    uint32_t total = 0;
    DevCounters* snap = nullptr;   // pinned [2]: after the level's kernels, latest
    uint2* d_moves = nullptr;      // device [move_cap]
    unsigned* d_bits = nullptr;    // device [3 x hole_cap + 32]: hole plan scratch
    unsigned* h_val = nullptr;     // pinned scratch word
    FormulaItem* h_item = nullptr; // pinned, one item
    FormulaItem* d_item = nullptr;
    char* d_text = nullptr;        // device [kTextCap]
    char* h_text = nullptr;        // pinned [kTextCap]
    int* d_tst = nullptr;
    int* h_tst = nullptr;
    Segment* old_table = nullptr;  // unmapped once the lane's first event has passed
    double t0 = 0, t_launched = 0;
    bool ran = false;
    lsyn_step_trace rec{};
  };
  static constexpr unsigned kTextCap = 1024;  // formula text of a job (sizes up to 17 need about 120 bytes)

  lsyn_config cfg_{};
  lsyn_batch_tuning tune_{};
  bool keep_finished_ = false;
  int device_ = 0, sms_ = 1;
  cudaStream_t stream_ = nullptr;  // batch steps (high priority)
  bool own_stream_ = false;
  BlockPool pool_;
  std::vector<Slot> slots_;
  std::deque<Job*> queue_;
  std::vector<Job*> active_;       // admitted, unfinished
  std::vector<Job*> done_;
  uint64_t next_seq_ = 0;
  size_t peak_ = 0;
  uint64_t steps_ = 0, evictions_ = 0, redos_ = 0, large_levels_ = 0;
  std::vector<Lane> lanes_;        // the large-level lane's tracks
  // device and pinned step state of the batch lane
  Alloc mem_;
  DevCounters* ctrs_ = nullptr;
  DevCounters* h_ctrs_ = nullptr;
  uint2* holes_ = nullptr;
  unsigned hole_cap_ = 1u << 16;
  uint2* h_holes_ = nullptr;       // pinned staging for the step's hole logs
  size_t h_holes_cap_ = 0;
  StepHeader* d_hdr_ = nullptr;
  StepHeader* h_hdr_ = nullptr;
  StepProblem* d_steps_ = nullptr;
  StepProblem* h_steps_ = nullptr;
  uint4* d_moves_ = nullptr;
  uint4* h_moves_ = nullptr;       // pinned [move_cap]
  unsigned move_cap_ = 1u << 22;
  unsigned* d_dense_ = nullptr;
  unsigned* h_dense_ = nullptr;
  unsigned* h_stage_ = nullptr;    // pinned per-slot scratch for counter writes
  FormulaItem* d_items_ = nullptr; // answers of a step, one launch
  FormulaItem* h_items_ = nullptr;
  char* d_texts_ = nullptr;
  char* h_texts_ = nullptr;
  int* d_tst_ = nullptr;
  int* h_tst_ = nullptr;
  char* fbuf_ = nullptr;           // lsyn_entry_formula on a job's handle
  int* fstatus_ = nullptr;
  char* h_fbuf_ = nullptr;
  int* h_fstatus_ = nullptr;
  std::map<std::tuple<int, int, int>, std::pair<cudaGraph_t, cudaGraphExec_t>> graphs_;  // (bits, bucket, sms)
  std::vector<Segment*> trim_after_sync_;
  std::vector<lsyn_step_trace> trace_;
  size_t trace_head_ = 0;
  lsyn_step_trace cur_{};

  bool reserve_slot(Slot& s, const Job* j, std::string* e);
  void trim_slot(Slot& s);
  lsyn_status bind(Job* j, int slot);
  void unbind(Job* j, bool keep_cache);
  void evict(Job* j);
  void finish(Job* j, lsyn_status st);
  bool release_finished();
  void drop_graphs();
  unsigned long long candidates(const Job* j, int k) const;
  unsigned long long solo_min() const { return tune_.solo_candidates ? tune_.solo_candidates : (1ull << 19); }
  // unary rows / binary pairs per work item of a batch step
  unsigned rows_per_item() const { return tune_.rows_per_item > 0 ? unsigned(tune_.rows_per_item) : 8u; }
  // load up to which a job's table fills before it is rebuilt larger (its entry limit does not depend on it)
  double table_load(const Job* j) const {
    return tune_.table_load_pct > 0 ? double(tune_.table_load_pct) / 100.0 : j->c->table_load;
  }
  int light_sms() const;
  unsigned long long predict_entries(const Job* j, int k, unsigned long long cand) const;
  size_t growth_cost(const Job* j, unsigned long long entries) const;
  // ln: the lane track the growth is for (its stream), or null for the batch stream
  lsyn_status grow(Job* j, unsigned long long entries, Lane* ln, bool* ok);
  lsyn_status rebuild_table(Job* j, unsigned long long tcap, uint32_t live_end, cudaStream_t st, Segment** old);
  lsyn_status relieve(bool* progressed);
  // batch lane
  lsyn_status batch_step(bool* progressed);
  lsyn_status run_group(std::vector<Plan>& g, int word_bits, int sms);
  lsyn_status launch_step(int word_bits, int n, int sms);
  lsyn_status launch_plain(int word_bits, int n, int sms);
  lsyn_status answer(const std::vector<Job*>& solved);
  // large-level lane
  lsyn_status lane_advance(Lane& L, bool* progressed);
  lsyn_status lane_launch(Lane& L, Job* j, bool* progressed);
  lsyn_status lane_commit(Lane& L);
  void lane_fail(Lane& L, lsyn_status s, const std::string& m);
  void note_peak() { if (pool_.in_use() > peak_) peak_ = pool_.in_use(); }
  void record(const lsyn_step_trace& t);
  void lane_done(Lane& L);  // close the track's trace record and free it
};

}  // namespace lsyn
