// The multi-problem scheduler behind lsyn_batch_* and the server.
//
// Jobs (one specification each) wait in a FIFO queue and are admitted into
// slots. A step advances every admitted job by one level of the bottom-up
// enumeration (the listing of paragraph "A generic program synthesiser") in one
// persistent launch per word size over a packed work list; between steps jobs
// finish, new ones are admitted (continuous batching), and caches grow.
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
// waits for a later step; if nothing can run, the youngest admitted jobs are
// evicted (their caches dropped, the jobs queued again) until the oldest fits.
// A job alone in the pool that still does not fit is capped at what the pool
// gives it (status LSYN_E_CACHE_FULL, noted in its error text).
#pragma once

#include <cstdint>
#include <deque>
#include <map>
#include <string>
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
  // Copy and validate a problem into a job (not yet queued).
  lsyn_status make_job(const lsyn_problem* p, int max_size, Job* j);
  void enqueue(Job* j, double t_submit);
  // Admit queued jobs into free slots while the pool can hold their first levels.
  lsyn_status admit();
  // One level of every admitted job (jobs that finish move to done()).
  lsyn_status step();
  bool busy() const { return !queue_.empty() || !active_.empty(); }
  // Jobs finished since the last call.
  std::vector<Job*> take_done();
  // Drop every job (queued, active or resident) and free their slots.
  void clear();
  // Release a finished job's slot (its cache).
  void release_job(Job* j);

  lsyn_batch_tuning tune() const { return tune_; }
  void set_tune(const lsyn_batch_tuning& t);
  int sms() const { return sms_; }
  cudaStream_t stream() const { return stream_; }
  const BlockPool& pool() const { return pool_; }
  size_t peak_in_use() const { return peak_; }
  uint64_t steps_run() const { return steps_; }
  uint64_t evictions() const { return evictions_; }
  uint64_t redos() const { return redos_; }
  int active_count() const { return int(active_.size()); }
  int queued_count() const { return int(queue_.size()); }
  std::string err;

 private:
  struct Slot {
    Segment arena, prov, slotpos, homes, misc, defer[2], table[2];
    int cur_table = 0;
    unsigned long long tcap = 0;   // slots of the current table
    bool reserved = false;
    Job* job = nullptr;
  };
  struct Plan {                    // one job's level in a step
    Job* j;
    int k;
    LevelPlan lp;
    unsigned long long deferred = 0;
    int cur = 0;
    uint32_t total = 0;
    bool undo = false;
    bool solo = false;               // its operators run as one-problem launches
  };

  lsyn_config cfg_{};
  lsyn_batch_tuning tune_{};
  bool keep_finished_ = false;
  int device_ = 0, sms_ = 1;
  cudaStream_t stream_ = nullptr;
  bool own_stream_ = false;
  BlockPool pool_;
  std::vector<Slot> slots_;
  std::deque<Job*> queue_;
  std::vector<Job*> active_;       // admitted, unfinished
  std::vector<Job*> done_;
  uint64_t next_seq_ = 0;
  size_t peak_ = 0;
  uint64_t steps_ = 0, evictions_ = 0, redos_ = 0;
  // device and pinned step state
  Alloc mem_;
  DevCounters* ctrs_ = nullptr;
  DevCounters* h_ctrs_ = nullptr;
  uint2* holes_ = nullptr;
  unsigned hole_cap_ = 1u << 16;
  StepHeader* d_hdr_ = nullptr;
  StepHeader* h_hdr_ = nullptr;
  StepProblem* d_steps_ = nullptr;
  StepProblem* h_steps_ = nullptr;
  uint4* d_moves_ = nullptr;
  unsigned move_cap_ = 1u << 22;
  unsigned* d_dense_ = nullptr;
  unsigned* h_dense_ = nullptr;
  unsigned* h_stage_ = nullptr;    // pinned per-slot scratch for counter writes
  char* fbuf_ = nullptr;
  int* fstatus_ = nullptr;
  char* h_fbuf_ = nullptr;
  int* h_fstatus_ = nullptr;
  std::map<std::pair<int, int>, std::pair<cudaGraph_t, cudaGraphExec_t>> graphs_;  // (word bits, bucket)
  std::vector<Segment*> trim_after_sync_;

  bool reserve_slot(Slot& s, const Job* j, std::string* e);
  void trim_slot(Slot& s, bool all);
  lsyn_status bind(Job* j, int slot);
  void unbind(Job* j, bool keep_cache);
  void evict(Job* j);
  void finish(Job* j, lsyn_status st);
  unsigned long long predict_entries(const Job* j, int k, unsigned long long cand) const;
  size_t growth_cost(const Job* j, unsigned long long entries) const;
  lsyn_status grow(Job* j, unsigned long long entries, bool* ok);
  lsyn_status rebuild_table(Job* j, unsigned long long tcap, uint32_t live_end);
  lsyn_status run_group(std::vector<Plan>& g, int word_bits);
  lsyn_status launch_step(int word_bits, int n, const std::vector<Plan>& g);
  lsyn_status launch_plain(int word_bits, int n);
  void note_peak() { if (pool_.in_use() > peak_) peak_ = pool_.in_use(); }
};

}  // namespace lsyn
