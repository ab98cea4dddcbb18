// Multi-problem scheduler: admission, cache growth, batch steps and the
// large-level lane (see lsyn_engine.h for the design).
#include "lsyn_engine.h"

#include <algorithm>
#include <cstring>
#include <new>

namespace lsyn {
namespace {

unsigned long long pow2_at_least(unsigned long long x) {
  unsigned long long p = 1;
  while (p < x) p <<= 1;
  return p;
}

unsigned long long pow2_at_most(unsigned long long x) {
  unsigned long long p = 1;
  while (p * 2 <= x) p <<= 1;
  return x ? p : 0;
}

constexpr size_t kSmallBytes = 4u << 20;  // constants + atom rows: (5 + 32) * 64 KiB at most, rounded
constexpr unsigned kDeferMin = 1u << 16, kDeferMax = 1u << 23;

unsigned defer_cap_for(unsigned long long entries) {
  return unsigned(std::max<unsigned long long>(kDeferMin, std::min<unsigned long long>(kDeferMax, entries / 16)));
}

template <typename T>
bool pinned(T** p, size_t n) {
  if (cudaMallocHost(reinterpret_cast<void**>(p), sizeof(T) * std::max<size_t>(n, 1)) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return false;
  }
  return true;
}

}  // namespace

// ---------------------------------------------------------------------------
// Setup and teardown
// ---------------------------------------------------------------------------

Engine::~Engine() {
  if (stream_) cudaStreamSynchronize(stream_);
  for (Lane& L : lanes_)
    if (L.stream) cudaStreamSynchronize(L.stream);
  drop_graphs();
  for (Slot& s : slots_) {
    s.arena.release(pool_);
    s.prov.release(pool_);
    s.slotpos.release(pool_);
    s.homes.release(pool_);
    s.misc.release(pool_);
    s.defer[0].release(pool_);
    s.defer[1].release(pool_);
    s.table[0].release(pool_);
    s.table[1].release(pool_);
  }
  mem_.release_all();
  for (void* p : {static_cast<void*>(h_ctrs_), static_cast<void*>(h_hdr_), static_cast<void*>(h_steps_),
                  static_cast<void*>(h_dense_), static_cast<void*>(h_stage_), static_cast<void*>(h_items_),
                  static_cast<void*>(h_texts_), static_cast<void*>(h_tst_), static_cast<void*>(h_fbuf_),
                  static_cast<void*>(h_fstatus_), static_cast<void*>(h_holes_)})
    if (p) cudaFreeHost(p);
  for (Lane& L : lanes_) {
    for (void* p : {static_cast<void*>(L.snap), static_cast<void*>(L.h_val), static_cast<void*>(L.h_item),
                    static_cast<void*>(L.h_text), static_cast<void*>(L.h_tst)})
      if (p) cudaFreeHost(p);
    if (L.ev) cudaEventDestroy(L.ev);
    if (L.stream) cudaStreamDestroy(L.stream);
  }
  if (own_stream_ && stream_) cudaStreamDestroy(stream_);
}

lsyn_status Engine::init(const lsyn_config* cfg, const lsyn_batch_tuning* tune, int max_active, bool keep_finished) {
  memset(&cfg_, 0, sizeof(cfg_));
  cfg_.device = -1;
  if (cfg) cfg_ = *cfg;
  if (!cfg_.cache_bytes) cfg_.cache_bytes = 1ull << 30;
  memset(&tune_, 0, sizeof(tune_));
  if (tune) tune_ = *tune;
  if (tune_.blocks_per_sm < 1) tune_.blocks_per_sm = 4;
  if (max_active < 1) { err = "max_active must be positive"; return LSYN_E_INVAL; }
  if (!valid_tuning(tune_, &err)) return LSYN_E_INVAL;
  tune_.max_active = max_active;
  keep_finished_ = keep_finished;
  cudaError_t e;
  auto cuda = [&](cudaError_t x) {
    err = cudaGetErrorString(x);
    return LSYN_E_CUDA;
  };
  if (cfg_.device >= 0 && (e = cudaSetDevice(cfg_.device)) != cudaSuccess) return cuda(e);
  if ((e = cudaGetDevice(&device_)) != cudaSuccess) return cuda(e);
  if ((e = cudaDeviceGetAttribute(&sms_, cudaDevAttrMultiProcessorCount, device_)) != cudaSuccess) return cuda(e);
  int prio_lo = 0, prio_hi = 0;
  if ((e = cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi)) != cudaSuccess) return cuda(e);
  stream_ = static_cast<cudaStream_t>(cfg_.stream);
  if (!stream_) {  // high priority; the legacy default stream could not be captured into a graph either
    if ((e = cudaStreamCreateWithPriority(&stream_, cudaStreamNonBlocking, prio_hi)) != cudaSuccess) return cuda(e);
    own_stream_ = true;
  }
  cfg_.stream = stream_;
  lanes_.resize(size_t(std::max(1, std::min(tune_.lanes > 0 ? tune_.lanes : 4, 8))));
  tune_.lanes = int32_t(lanes_.size());
  for (Lane& L : lanes_) {
    if ((e = cudaStreamCreateWithPriority(&L.stream, cudaStreamNonBlocking, prio_lo)) != cudaSuccess) return cuda(e);
    if ((e = cudaEventCreateWithFlags(&L.ev, cudaEventDisableTiming)) != cudaSuccess) return cuda(e);
  }
  size_t free_b = 0, total_b = 0;
  if ((e = cudaMemGetInfo(&free_b, &total_b)) != cudaSuccess) return cuda(e);
  const size_t budget = tune_.pool_bytes ? size_t(tune_.pool_bytes) : size_t(double(free_b) * 0.9);
  if (!pool_.init(device_, budget, &err)) return LSYN_E_CUDA;
  tune_.pool_bytes = pool_.budget();

  const int n = max_active;
  const int cap_steps = int(pow2_at_least((unsigned long long)n));
  slots_.resize(size_t(n));
  mem_.alloc = cfg_.alloc;
  mem_.free = cfg_.free;
  mem_.user = cfg_.alloc_user;
  ctrs_ = static_cast<DevCounters*>(mem_.get(sizeof(DevCounters) * size_t(n)));
  holes_ = static_cast<uint2*>(mem_.get(sizeof(uint2) * size_t(hole_cap_) * size_t(n)));
  d_hdr_ = static_cast<StepHeader*>(mem_.get(sizeof(StepHeader)));
  d_steps_ = static_cast<StepProblem*>(mem_.get(sizeof(StepProblem) * size_t(cap_steps)));
  d_moves_ = static_cast<uint4*>(mem_.get(sizeof(uint4) * size_t(move_cap_)));
  d_dense_ = static_cast<unsigned*>(mem_.get(sizeof(unsigned) * size_t(n)));
  d_items_ = static_cast<FormulaItem*>(mem_.get(sizeof(FormulaItem) * size_t(n)));
  d_texts_ = static_cast<char*>(mem_.get(size_t(kTextCap) * size_t(n)));
  d_tst_ = static_cast<int*>(mem_.get(sizeof(int) * size_t(n)));
  fbuf_ = static_cast<char*>(mem_.get(lsyn_ctx::kFormulaCap));
  fstatus_ = static_cast<int*>(mem_.get(sizeof(int)));
  if (!ctrs_ || !holes_ || !d_hdr_ || !d_steps_ || !d_moves_ || !d_dense_ || !d_items_ || !d_texts_ || !d_tst_ ||
      !fbuf_ || !fstatus_) {
    err = "device allocation failed";
    return LSYN_E_NOMEM;
  }
  for (Lane& L : lanes_) {
    L.d_moves = static_cast<uint2*>(mem_.get(sizeof(uint2) * size_t(move_cap_)));
    L.d_bits = static_cast<unsigned*>(mem_.get(sizeof(unsigned) * (3 * size_t(hole_cap_) + 32)));
    L.d_item = static_cast<FormulaItem*>(mem_.get(sizeof(FormulaItem)));
    L.d_text = static_cast<char*>(mem_.get(kTextCap));
    L.d_tst = static_cast<int*>(mem_.get(sizeof(int)));
    if (!L.d_moves || !L.d_bits || !L.d_item || !L.d_text || !L.d_tst || !pinned(&L.snap, 2) ||
        !pinned(&L.h_val, 1) || !pinned(&L.h_item, 1) || !pinned(&L.h_text, kTextCap) || !pinned(&L.h_tst, 1)) {
      err = "lane allocation failed";
      return LSYN_E_NOMEM;
    }
  }
  h_holes_cap_ = hole_cap_;
  if (!pinned(&h_ctrs_, size_t(n)) || !pinned(&h_hdr_, 1) || !pinned(&h_steps_, size_t(cap_steps)) ||
      !pinned(&h_dense_, size_t(n)) || !pinned(&h_stage_, size_t(n)) || !pinned(&h_items_, size_t(n)) ||
      !pinned(&h_texts_, size_t(kTextCap) * size_t(n)) || !pinned(&h_tst_, size_t(n)) ||
      !pinned(&h_fbuf_, lsyn_ctx::kFormulaCap) || !pinned(&h_fstatus_, 1) || !pinned(&h_holes_, h_holes_cap_)) {
    err = "pinned host allocation failed";
    return LSYN_E_NOMEM;
  }
  memset(h_steps_, 0, sizeof(StepProblem) * size_t(cap_steps));
  if ((e = cudaMemsetAsync(ctrs_, 0, sizeof(DevCounters) * size_t(n), stream_)) != cudaSuccess ||
      (e = cudaMemsetAsync(d_steps_, 0, sizeof(StepProblem) * size_t(cap_steps), stream_)) != cudaSuccess ||
      (e = cudaStreamSynchronize(stream_)) != cudaSuccess)
    return cuda(e);
  return LSYN_OK;
}

void Engine::drop_graphs() {
  for (auto& kv : graphs_) {
    if (kv.second.second) cudaGraphExecDestroy(kv.second.second);
    if (kv.second.first) cudaGraphDestroy(kv.second.first);
  }
  graphs_.clear();
}

bool Engine::valid_tuning(const lsyn_batch_tuning& t, std::string* e) {
  if (t.rows_per_item != 0 && t.rows_per_item != 2 && t.rows_per_item != 4 && t.rows_per_item != 8) {
    *e = "rows_per_item must be 0, 2, 4 or 8";
    return false;
  }
  if (t.words_per_thread < 0 || t.words_per_thread > 2) {
    *e = "words_per_thread must be 0, 1 or 2";
    return false;
  }
  if (t.table_load_pct != 0 && (t.table_load_pct < 25 || t.table_load_pct > 90)) {
    *e = "table_load_pct must be 0 or in 25..90";
    return false;
  }
  return true;
}

void Engine::set_tune(const lsyn_batch_tuning& t) {
  if (stream_) cudaStreamSynchronize(stream_);
  tune_.blocks_per_sm = t.blocks_per_sm > 0 ? t.blocks_per_sm : 4;
  tune_.use_graph = t.use_graph;
  tune_.predict_pct = t.predict_pct;
  tune_.solo_candidates = t.solo_candidates;
  tune_.light_sms = t.light_sms;  // the number of lane tracks is fixed at creation
  tune_.rows_per_item = t.rows_per_item;
  tune_.words_per_thread = t.words_per_thread;
  tune_.table_load_pct = t.table_load_pct;
  drop_graphs();  // the launch shape is part of each graph
}

lsyn_status Engine::make_job(const lsyn_problem* p, int max_size, Job* j) const {
  // The constants and atom rows are packed once; they are all a (re)admission
  // needs. The layout (and so the entry limit) is the one-problem path's.
  j->max_size = max_size;
  lsyn_config cfg = cfg_;
  cfg.device = -1;  // may run on a caller's thread: leave its current device alone
  lsyn_status s = ctx_shell(p, &cfg, false, &j->c, &j->consts, &j->atoms);
  if (s != LSYN_OK) {
    j->err = thread_error();
    return s;
  }
  j->c->device = device_;
  j->c->sms = sms_;
  j->c->borrowed = true;
  j->c->owns_host = false;
  j->c->stream = stream_;
  j->cap_entries = j->c->max_entries;
  j->c->max_entries = 0;
  j->c->table_cap = 0;
  return LSYN_OK;
}

void Engine::enqueue(Job* j, double t_submit) {
  j->t_submit = t_submit;
  j->state = Job::kQueued;
  j->status = LSYN_PENDING;
  queue_.push_back(j);
}

std::vector<lsyn_step_trace> Engine::trace() const {
  std::vector<lsyn_step_trace> out;
  out.reserve(trace_.size());
  for (size_t i = 0; i < trace_.size(); ++i) out.push_back(trace_[(trace_head_ + i) % trace_.size()]);
  return out;
}

// ---------------------------------------------------------------------------
// Slots
// ---------------------------------------------------------------------------

// Address space for this job's largest cache (a slot keeps the largest
// reservation any of its jobs needed).
bool Engine::reserve_slot(Slot& s, const Job* j, std::string* e) {
  const unsigned long long cap = j->cap_entries + 64;
  const size_t M = size_t(j->c->vecs) * 16;
  const double load = std::min(j->c->table_load, table_load(j));
  const unsigned long long max_t = std::max(pow2_at_least((unsigned long long)(double(cap) / load) + 2),
                                            (unsigned long long)(pool_.granularity() / 8));
  auto fit = [&](Segment& sg, size_t bytes) {
    if (sg.reserved() && sg.reserved() >= bytes + bytes / 2) return true;
    sg.release(pool_);
    return sg.reserve(pool_, bytes, e);
  };
  if (!fit(s.arena, size_t(cap) * M) || !fit(s.prov, size_t(cap) * 8) || !fit(s.slotpos, size_t(cap) * 4) ||
      !fit(s.homes, size_t(cap) * 4) || !fit(s.misc, kSmallBytes) || !fit(s.defer[0], size_t(kDeferMax) * 8) ||
      !fit(s.defer[1], size_t(kDeferMax) * 8) || !fit(s.table[0], size_t(max_t) * 8) ||
      !fit(s.table[1], size_t(max_t) * 8))
    return false;
  s.reserved = true;
  return true;
}

// Keep a small warm mapping for the slot's next job. The slot's job has no
// work in flight in the large-level lane; the batch stream is drained first.
void Engine::trim_slot(Slot& s) {
  cudaStreamSynchronize(stream_);
  const size_t g = pool_.granularity();
  s.arena.shrink(pool_, 2 * g);
  s.prov.shrink(pool_, g);
  s.slotpos.shrink(pool_, g);
  s.homes.shrink(pool_, g);
  s.misc.shrink(pool_, g);
  s.defer[0].shrink(pool_, g);
  s.defer[1].shrink(pool_, g);
  s.table[s.cur_table].shrink(pool_, g);
  s.table[1 - s.cur_table].shrink(pool_, 0);
  s.tcap = 0;
}

lsyn_status Engine::bind(Job* j, int slot) {
  Slot& s = slots_[size_t(slot)];
  if (!reserve_slot(s, j, &err)) return LSYN_E_CUDA;
  lsyn_ctx* c = j->c;
  const size_t M = size_t(c->vecs) * 16;
  if (!s.misc.grow(pool_, (5 + size_t(c->n_props)) * M, &err)) return LSYN_E_NOMEM;
  s.job = j;
  s.tcap = 0;
  j->slot = slot;
  c->arena = static_cast<uint4*>(s.arena.ptr());
  c->prov = static_cast<unsigned long long*>(s.prov.ptr());
  c->slotpos = static_cast<unsigned*>(s.slotpos.ptr());
  c->homes = static_cast<unsigned*>(s.homes.ptr());
  c->consts = static_cast<uint4*>(s.misc.ptr());
  c->atoms = c->consts + size_t(5) * c->vecs;
  c->defer[0] = static_cast<unsigned long long*>(s.defer[0].ptr());
  c->defer[1] = static_cast<unsigned long long*>(s.defer[1].ptr());
  c->table = static_cast<unsigned long long*>(s.table[s.cur_table].ptr());
  c->table_cap = 0;
  c->max_entries = 0;
  c->defer_cap = 0;
  c->ctr = ctrs_ + slot;
  c->holes = holes_ + size_t(slot) * hole_cap_;
  c->hole_cap = hole_cap_;
  c->fbuf = fbuf_;
  c->fstatus = fstatus_;
  c->h_fbuf = h_fbuf_;
  c->h_fstatus = h_fstatus_;
  c->level_start.assign(1, 0);
  c->level_n.assign(1, 0);
  c->levels_done = 0;
  c->last_incomplete = false;
  c->constructed = 0;
  c->last_sol = ~0ull;
  j->redo = j->heavy = j->in_flight = j->paused = false;
  j->ratio = 1.0;
  cudaError_t e = cudaMemcpyAsync(c->consts, j->consts.data(), j->consts.size() * 4, cudaMemcpyHostToDevice, stream_);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->atoms, j->atoms.data(), j->atoms.size() * 4, cudaMemcpyHostToDevice, stream_);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->ctr, 0, sizeof(DevCounters), stream_);
  if (e != cudaSuccess) { err = cudaGetErrorString(e); return LSYN_E_CUDA; }
  j->state = Job::kActive;
  j->seq = next_seq_++;
  j->t_admit = now_ms();
  j->resident = true;
  active_.push_back(j);
  note_peak();
  return LSYN_OK;
}

void Engine::unbind(Job* j, bool keep_cache) {
  if (j->slot < 0 || keep_cache) return;
  Slot& s = slots_[size_t(j->slot)];
  trim_slot(s);
  s.job = nullptr;
  j->slot = -1;
  j->resident = false;
  lsyn_ctx* c = j->c;
  c->levels_done = 0;  // read-only calls on the handle now see no levels
  c->level_start.assign(1, 0);
  c->level_n.assign(1, 0);
  c->arena = nullptr;
  c->prov = nullptr;
  c->table = nullptr;
  c->max_entries = 0;
  c->table_cap = 0;
}

bool Engine::release_finished() {
  bool any = false;
  for (Slot& s : slots_)
    if (s.job && s.job->state == Job::kDone) {
      unbind(s.job, false);
      any = true;
    }
  return any;
}

void Engine::evict(Job* j) {
  active_.erase(std::remove(active_.begin(), active_.end(), j), active_.end());
  unbind(j, false);
  j->state = Job::kQueued;
  j->redo = j->heavy = j->paused = false;
  ++j->evictions;
  ++evictions_;
  queue_.push_front(j);
}

void Engine::finish(Job* j, lsyn_status st) {
  lsyn_ctx* c = j->c;
  j->status = st;
  j->t_done = now_ms();
  j->levels_done = c->levels_done;
  j->constructed = int64_t(c->constructed);
  j->unique = int64_t(c->level_start.back() + c->level_n.back());
  j->state = Job::kDone;
  j->in_flight = false;
  active_.erase(std::remove(active_.begin(), active_.end(), j), active_.end());
  done_.push_back(j);
  unbind(j, keep_finished_);
}

std::vector<Job*> Engine::take_done() {
  std::vector<Job*> out;
  out.swap(done_);
  return out;
}

void Engine::clear() {
  if (stream_) cudaStreamSynchronize(stream_);
  for (Lane& L : lanes_) {
    if (L.stream) cudaStreamSynchronize(L.stream);
    L.j = nullptr;
    L.stage = Lane::kIdle;
    L.old_table = nullptr;
  }
  for (Job* j : active_) {
    j->in_flight = false;
    unbind(j, false);
    j->state = Job::kDone;
  }
  active_.clear();
  queue_.clear();
  for (Slot& s : slots_)
    if (s.job) unbind(s.job, false);
  done_.clear();
}

lsyn_status Engine::admit() {
  if (queue_.empty()) return LSYN_OK;
  // memory the admitted jobs are predicted to need for their next level
  size_t reserve = 0;
  for (Job* j : active_) {
    const int k = j->c->levels_done + 1;
    const size_t g = growth_cost(j, predict_entries(j, k, candidates(j, k)));
    reserve += g == ~size_t(0) ? 0 : g;
  }
  size_t next_free = 0;
  while (!queue_.empty()) {
    while (next_free < slots_.size() && slots_[next_free].job) ++next_free;
    if (next_free >= slots_.size()) {
      // every slot is taken: free one kept only for a finished job's export
      for (size_t i = 0; i < slots_.size(); ++i)
        if (slots_[i].job && slots_[i].job->state == Job::kDone) {
          unbind(slots_[i].job, false);
          next_free = i;
          break;
        }
      if (next_free >= slots_.size()) break;
    }
    Job* j = queue_.front();
    // first levels: constants, warm arrays and a table (a few blocks)
    const size_t M = size_t(j->c->vecs) * 16;
    const size_t first = (5 + size_t(j->c->n_props)) * M + 16 * pool_.granularity();
    if (!active_.empty() && pool_.available() < reserve + first) break;
    queue_.pop_front();
    lsyn_status s = bind(j, int(next_free));
    if (s != LSYN_OK) {
      slots_[next_free].job = nullptr;
      j->slot = -1;
      active_.erase(std::remove(active_.begin(), active_.end(), j), active_.end());
      if (s != LSYN_E_NOMEM) return s;
      if (!active_.empty()) {  // wait for memory
        j->state = Job::kQueued;
        queue_.push_front(j);
        err.clear();
        break;
      }
      j->err = "the memory pool cannot hold this problem's constants";
      j->status = LSYN_E_NOMEM;
      j->state = Job::kDone;
      j->t_done = now_ms();
      done_.push_back(j);
      err.clear();
      continue;
    }
    reserve += first;
  }
  return LSYN_OK;
}

// ---------------------------------------------------------------------------
// Cache growth
// ---------------------------------------------------------------------------

unsigned long long Engine::candidates(const Job* j, int k) const {
  return (unsigned long long)std::max<int64_t>(0, level_candidate_count(j->c, k));
}

int Engine::light_sms() const {
  const int want = tune_.light_sms > 0 ? tune_.light_sms : std::max(1, sms_ / 8);
  return std::max(1, std::min(want, sms_ - 1));
}

unsigned long long Engine::predict_entries(const Job* j, int k, unsigned long long cand) const {
  const lsyn_ctx* c = j->c;
  const unsigned long long start = c->level_start.back() + c->level_n.back();
  unsigned long long add = cand;
  if (k >= 3 && !j->redo) {
    const double margin = (tune_.predict_pct > 0 ? tune_.predict_pct : 150) / 100.0;
    const double r = std::min(1.0, margin * j->ratio);
    add = std::min<unsigned long long>(
        cand, (unsigned long long)(double(cand) * r) + (tune_.predict_pct > 0 ? 1ull : 1024ull));
  }
  return std::min<unsigned long long>(j->cap_entries, start + add + 1);
}

size_t Engine::growth_cost(const Job* j, unsigned long long entries) const {
  if (j->slot < 0) return 0;
  const Slot& s = slots_[size_t(j->slot)];
  const lsyn_ctx* c = j->c;
  const size_t M = size_t(c->vecs) * 16;
  entries = std::min<unsigned long long>(entries, j->cap_entries);
  size_t cost = 0;
  auto add = [&](size_t x) { cost = (x == ~size_t(0) || cost == ~size_t(0)) ? ~size_t(0) : cost + x; };
  const size_t cap = size_t(j->cap_entries);
  add(s.arena.grow_cost(pool_, size_t(entries) * M, cap * M));
  add(s.prov.grow_cost(pool_, size_t(entries) * 8, cap * 8));
  add(s.slotpos.grow_cost(pool_, size_t(entries) * 4, cap * 4));
  add(s.homes.grow_cost(pool_, size_t(entries) * 4, cap * 4));
  const size_t dbytes = size_t(defer_cap_for(entries)) * 8;
  const size_t dlimit = size_t(defer_cap_for(cap)) * 8;
  add(s.defer[0].grow_cost(pool_, dbytes, dlimit));
  add(s.defer[1].grow_cost(pool_, dbytes, dlimit));
  const unsigned long long want_t = pow2_at_least((unsigned long long)(double(entries) / table_load(j)) + 1);
  if (want_t > s.tcap || j->redo) {
    const size_t tb = size_t(std::max(want_t, s.tcap)) * 8;
    add(s.tcap == 0 ? s.table[s.cur_table].grow_cost(pool_, tb) : s.table[1 - s.cur_table].grow_cost(pool_, tb));
  }
  return cost;
}

lsyn_status Engine::rebuild_table(Job* j, unsigned long long tcap, uint32_t live_end, cudaStream_t st,
                                  Segment** old) {
  Slot& s = slots_[size_t(j->slot)];
  lsyn_ctx* c = j->c;
  const LaunchCfg lc{st, sms_};
  const bool fresh = s.tcap == 0;
  Segment& dst = fresh ? s.table[s.cur_table] : s.table[1 - s.cur_table];
  if (!dst.grow(pool_, size_t(tcap) * 8, &err)) return LSYN_E_NOMEM;
  tcap = std::max(tcap, pow2_at_most(dst.mapped() / 8));  // a larger table costs only its clearing
  auto* nt = static_cast<unsigned long long*>(dst.ptr());
  cudaError_t e = cudaMemsetAsync(nt, 0, size_t(tcap) * 8, st);
  if (e == cudaSuccess && !fresh) {
    auto* ot = static_cast<unsigned long long*>(s.table[s.cur_table].ptr());
    e = c->word_bits == 32
            ? Kernels<uint32_t>::rehash(ot, s.tcap, nt, tcap, c->homes, c->slotpos, live_end, &c->ctr->error, lc)
            : Kernels<uint64_t>::rehash(ot, s.tcap, nt, tcap, c->homes, c->slotpos, live_end, &c->ctr->error, lc);
  }
  if (e != cudaSuccess) { err = std::string("table rebuild: ") + cudaGetErrorString(e); return LSYN_E_CUDA; }
  if (!fresh) {
    *old = &s.table[s.cur_table];
    s.cur_table = 1 - s.cur_table;
  }
  s.tcap = tcap;
  c->table = nt;
  c->table_cap = tcap;
  return LSYN_OK;
}

// Grow a job's arrays (and table) to hold `entries`, on stream st. *ok = false
// (with nothing to undo) when the pool cannot hold it now.
lsyn_status Engine::grow(Job* j, unsigned long long entries, Lane* ln, bool* ok) {
  *ok = false;
  const cudaStream_t st = ln ? ln->stream : stream_;
  Slot& s = slots_[size_t(j->slot)];
  lsyn_ctx* c = j->c;
  const size_t M = size_t(c->vecs) * 16;
  entries = std::max<unsigned long long>(1, std::min<unsigned long long>(entries, j->cap_entries));
  const size_t cost = growth_cost(j, entries);
  if (cost == ~size_t(0) || cost > pool_.available()) return LSYN_OK;
  std::string e2;
  const size_t cap = size_t(j->cap_entries);
  const size_t dbytes = size_t(defer_cap_for(entries)) * 8;
  const size_t dlimit = size_t(defer_cap_for(cap)) * 8;
  if (!s.arena.grow(pool_, size_t(entries) * M, &e2, cap * M) ||
      !s.prov.grow(pool_, size_t(entries) * 8, &e2, cap * 8) ||
      !s.slotpos.grow(pool_, size_t(entries) * 4, &e2, cap * 4) ||
      !s.homes.grow(pool_, size_t(entries) * 4, &e2, cap * 4) || !s.defer[0].grow(pool_, dbytes, &e2, dlimit) ||
      !s.defer[1].grow(pool_, dbytes, &e2, dlimit))
    return LSYN_OK;  // the pool ran short (another size class was needed): try again later
  const unsigned long long live = c->level_start.back() + c->level_n.back();
  const unsigned long long want_t = pow2_at_least((unsigned long long)(double(entries) / table_load(j)) + 1);
  if (want_t > s.tcap || j->redo) {
    Segment* old = nullptr;
    lsyn_status r = rebuild_table(j, std::max(want_t, s.tcap), uint32_t(live), st, &old);
    if (r == LSYN_E_NOMEM) return LSYN_OK;
    if (r != LSYN_OK) return r;
    if (old) {
      if (ln) ln->old_table = old;
      else trim_after_sync_.push_back(old);
    }
  }
  if (j->redo) {
    // the undone level's entries are gone from the table; the arena restarts at its first id
    unsigned* v = ln ? ln->h_val : &h_stage_[j->slot];
    *v = uint32_t(live);
    cudaError_t e = cudaMemcpyAsync(&c->ctr->n_entries, v, sizeof(unsigned), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) { err = cudaGetErrorString(e); return LSYN_E_CUDA; }
  }
  unsigned long long have = j->cap_entries;
  have = std::min<unsigned long long>(have, s.arena.mapped() / M);
  have = std::min<unsigned long long>(have, s.prov.mapped() / 8);
  have = std::min<unsigned long long>(have, s.slotpos.mapped() / 4);
  have = std::min<unsigned long long>(have, s.homes.mapped() / 4);
  have = std::min<unsigned long long>(have, (unsigned long long)(double(s.tcap) * table_load(j)));
  c->max_entries = unsigned(have);
  c->defer_cap = unsigned(std::min<size_t>(kDeferMax, std::min(s.defer[0].mapped(), s.defer[1].mapped()) / 8));
  note_peak();
  *ok = true;
  return LSYN_OK;
}

// Nothing moved and jobs wait for memory: drop finished caches, then evict the
// youngest jobs not in flight until the oldest waiting one fits; alone, cap it.
lsyn_status Engine::relieve(bool* progressed) {
  Job* oldest = nullptr;
  for (Job* j : active_)
    if (j->paused && !j->in_flight && (!oldest || j->seq < oldest->seq)) oldest = j;
  if (!oldest) return LSYN_OK;
  auto retry = [&](bool* ok) {
    // on the batch stream; a large level launched later waits for it (below)
    const int k = oldest->c->levels_done + 1;
    return grow(oldest, predict_entries(oldest, k, candidates(oldest, k)), nullptr, ok);
  };
  bool ok = false;
  if (release_finished()) *progressed = true;
  lsyn_status s = retry(&ok);
  if (s != LSYN_OK) return s;
  while (!ok) {
    Job* young = nullptr;
    for (Job* j : active_)
      if (j != oldest && !j->in_flight && (!young || j->seq > young->seq)) young = j;
    if (!young) break;
    evict(young);
    *progressed = true;
    if ((s = retry(&ok)) != LSYN_OK) return s;
  }
  if (ok) {
    oldest->paused = false;
    *progressed = true;
    cudaError_t e = cudaStreamSynchronize(stream_);  // the growth's table rebuild, before any other stream uses it
    if (e != cudaSuccess) { err = cudaGetErrorString(e); return LSYN_E_CUDA; }
    return LSYN_OK;
  }
  lsyn_ctx* c = oldest->c;
  const unsigned long long live = c->level_start.back() + c->level_n.back();
  if (c->max_entries >= live && slots_[size_t(oldest->slot)].tcap > 0 && !oldest->redo) {
    oldest->capped = true;
    oldest->cap_entries = c->max_entries;
    oldest->paused = false;
    oldest->err = "the memory pool could not hold this cache: capped at " + std::to_string(c->max_entries) + " entries";
  } else {
    oldest->err = "the memory pool cannot hold this problem's next level";
    finish(oldest, LSYN_E_NOMEM);
  }
  *progressed = true;
  return LSYN_OK;
}

// ---------------------------------------------------------------------------
// The loop
// ---------------------------------------------------------------------------

lsyn_status Engine::pump(bool may_block, bool* progressed) {
  cudaSetDevice(device_);
  bool moved = false;
  auto advance_all = [&]() {
    for (Lane& L : lanes_) {
      lsyn_status r = lane_advance(L, &moved);
      if (r != LSYN_OK) return r;
    }
    return LSYN_OK;
  };
  lsyn_status s = advance_all();
  if (s == LSYN_OK) s = batch_step(&moved);
  if (s == LSYN_OK) s = advance_all();
  if (s == LSYN_OK && !moved) {
    if (lanes_busy()) {
      if (may_block) {
        for (Lane& L : lanes_)
          if (L.stage != Lane::kIdle) {
            cudaEventSynchronize(L.ev);
            break;
          }
        s = advance_all();
      }
    } else {
      s = relieve(&moved);
    }
  }
  *progressed = moved;
  return s;
}

// ---------------------------------------------------------------------------
// Batch lane
// ---------------------------------------------------------------------------

lsyn_status Engine::batch_step(bool* progressed) {
  const double t0 = now_ms();
  std::sort(active_.begin(), active_.end(), [](const Job* a, const Job* b) { return a->seq < b->seq; });
  std::vector<Job*> runnable;
  const std::vector<Job*> order = active_;
  const size_t done0 = done_.size();
  for (Job* j : order) {
    if (j->heavy || j->in_flight) continue;
    const int k = j->c->levels_done + 1;
    if (k > j->max_size) {
      finish(j, LSYN_NOT_FOUND);
      *progressed = true;
      continue;
    }
    const unsigned long long cand = candidates(j, k);
    if (k >= 2 && cand > solo_min()) {
      j->heavy = true;
      continue;
    }
    bool ok = false;
    lsyn_status s = grow(j, predict_entries(j, k, cand), nullptr, &ok);
    if (s != LSYN_OK) return s;
    if (!ok && release_finished()) {  // caches kept only for export go first
      if ((s = grow(j, predict_entries(j, k, cand), nullptr, &ok)) != LSYN_OK) return s;
    }
    j->paused = !ok;
    if (ok) runnable.push_back(j);
  }
  if (runnable.empty()) return LSYN_OK;
  memset(&cur_, 0, sizeof(cur_));
  cur_.step = int64_t(steps_);
  cur_.lane = 0;
  cur_.plan_ms = now_ms() - t0;
  cur_.solo = lanes_busy() ? 1 : 0;
  const int sms = lanes_busy() ? light_sms() : sms_;
  for (int wb : {64, 32}) {
    std::vector<Plan> g;
    for (Job* j : runnable)
      if (j->state == Job::kActive && j->c->word_bits == wb) g.push_back(Plan{j, j->c->levels_done + 1, LevelPlan()});
    if (g.empty()) continue;
    lsyn_status s = run_group(g, wb, sms);
    if (s != LSYN_OK) return s;
  }
  cudaError_t e = cudaStreamSynchronize(stream_);
  if (e != cudaSuccess) { err = std::string("step sync: ") + cudaGetErrorString(e); return LSYN_E_CUDA; }
  for (Segment* sg : trim_after_sync_) {
    bool current = false;
    for (Slot& sl : slots_)
      if (&sl.table[sl.cur_table] == sg) current = true;
    if (!current) sg->shrink(pool_, 0);
  }
  trim_after_sync_.clear();
  ++steps_;
  *progressed = true;
  cur_.finished = int32_t(done_.size() - done0);
  cur_.pool_in_use = pool_.in_use();
  cur_.settle_ms = now_ms() - t0 - cur_.plan_ms - cur_.run_ms;
  record(cur_);
  return LSYN_OK;
}

void Engine::record(const lsyn_step_trace& t) {
  if (trace_.size() < kTraceCap) {
    trace_.push_back(t);
  } else {
    trace_[trace_head_] = t;
    trace_head_ = (trace_head_ + 1) % kTraceCap;
  }
}

void Engine::lane_done(Lane& L) {
  L.rec.settle_ms = now_ms() - L.t_launched - L.rec.run_ms;
  L.rec.pool_in_use = pool_.in_use();
  L.rec.finished = L.j && L.j->state == Job::kDone ? 1 : 0;
  record(L.rec);
  if (L.j) L.j->in_flight = false;
  L.j = nullptr;
  L.stage = Lane::kIdle;
}

bool Engine::lanes_busy() const {
  for (const Lane& L : lanes_)
    if (L.stage != Lane::kIdle) return true;
  return false;
}

lsyn_status Engine::launch_step(int word_bits, int n, int sms) {
  LaunchCfg lc{stream_, sms};
  cudaError_t e;
  if (tune_.use_graph) {
    const int bucket = int(pow2_at_least((unsigned long long)n));
    auto& gr = graphs_[std::make_tuple(word_bits, bucket, sms)];
    if (!gr.second) {
      e = cudaStreamBeginCapture(stream_, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) { err = std::string("graph capture: ") + cudaGetErrorString(e); return LSYN_E_CUDA; }
      cudaMemcpyAsync(d_hdr_, h_hdr_, sizeof(StepHeader), cudaMemcpyHostToDevice, stream_);
      cudaMemcpyAsync(d_steps_, h_steps_, sizeof(StepProblem) * size_t(bucket), cudaMemcpyHostToDevice, stream_);
      if (word_bits == 32) {
        Kernels<uint32_t>::batch_begin(d_hdr_, d_steps_, bucket, lc);
        Kernels<uint32_t>::batch_run(d_hdr_, d_steps_, lc, tune_.blocks_per_sm, tune_.words_per_thread);
      } else {
        Kernels<uint64_t>::batch_begin(d_hdr_, d_steps_, bucket, lc);
        Kernels<uint64_t>::batch_run(d_hdr_, d_steps_, lc, tune_.blocks_per_sm, tune_.words_per_thread);
      }
      cudaMemcpyAsync(h_ctrs_, ctrs_, sizeof(DevCounters) * slots_.size(), cudaMemcpyDeviceToHost, stream_);
      e = cudaStreamEndCapture(stream_, &gr.first);
      if (e != cudaSuccess) { err = std::string("graph capture: ") + cudaGetErrorString(e); return LSYN_E_CUDA; }
      e = cudaGraphInstantiate(&gr.second, gr.first, 0);
      if (e != cudaSuccess) { err = std::string("graph instantiate: ") + cudaGetErrorString(e); return LSYN_E_CUDA; }
    }
    e = cudaGraphLaunch(gr.second, stream_);
    if (e != cudaSuccess) { err = std::string("graph launch: ") + cudaGetErrorString(e); return LSYN_E_CUDA; }
  } else {
    e = cudaMemcpyAsync(d_hdr_, h_hdr_, sizeof(StepHeader), cudaMemcpyHostToDevice, stream_);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_steps_, h_steps_, sizeof(StepProblem) * size_t(n), cudaMemcpyHostToDevice, stream_);
    if (e == cudaSuccess)
      e = word_bits == 32 ? Kernels<uint32_t>::batch_begin(d_hdr_, d_steps_, n, lc)
                          : Kernels<uint64_t>::batch_begin(d_hdr_, d_steps_, n, lc);
    if (e == cudaSuccess)
      e = word_bits == 32 ? Kernels<uint32_t>::batch_run(d_hdr_, d_steps_, lc, tune_.blocks_per_sm, tune_.words_per_thread)
                          : Kernels<uint64_t>::batch_run(d_hdr_, d_steps_, lc, tune_.blocks_per_sm, tune_.words_per_thread);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h_ctrs_, ctrs_, sizeof(DevCounters) * slots_.size(), cudaMemcpyDeviceToHost, stream_);
    if (e != cudaSuccess) { err = std::string("batch step: ") + cudaGetErrorString(e); return LSYN_E_CUDA; }
  }
  e = cudaStreamSynchronize(stream_);
  if (e != cudaSuccess) { err = std::string("batch step sync: ") + cudaGetErrorString(e); return LSYN_E_CUDA; }
  return LSYN_OK;
}

// Deferred-only passes reuse the step arrays without the counter reset.
lsyn_status Engine::launch_plain(int word_bits, int n, int sms) {
  LaunchCfg lc{stream_, sms};
  cudaError_t e = cudaMemcpyAsync(d_hdr_, h_hdr_, sizeof(StepHeader), cudaMemcpyHostToDevice, stream_);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_steps_, h_steps_, sizeof(StepProblem) * size_t(n), cudaMemcpyHostToDevice, stream_);
  if (e == cudaSuccess)
    e = word_bits == 32 ? Kernels<uint32_t>::batch_run(d_hdr_, d_steps_, lc, tune_.blocks_per_sm, tune_.words_per_thread)
                        : Kernels<uint64_t>::batch_run(d_hdr_, d_steps_, lc, tune_.blocks_per_sm, tune_.words_per_thread);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h_ctrs_, ctrs_, sizeof(DevCounters) * slots_.size(), cudaMemcpyDeviceToHost, stream_);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream_);
  if (e != cudaSuccess) { err = std::string("batch pass: ") + cudaGetErrorString(e); return LSYN_E_CUDA; }
  return LSYN_OK;
}

// Formula text of every job answered in a step: one launch, one copy back.
lsyn_status Engine::answer(const std::vector<Job*>& solved) {
  const int n = int(solved.size());
  if (!n) return LSYN_OK;
  for (int i = 0; i < n; ++i) h_items_[i] = FormulaItem{solved[size_t(i)]->c->prov, &solved[size_t(i)]->c->ctr->sol};
  cudaError_t e = cudaMemcpyAsync(d_items_, h_items_, sizeof(FormulaItem) * size_t(n), cudaMemcpyHostToDevice, stream_);
  if (e == cudaSuccess) e = reconstruct_many(d_items_, n, d_texts_, kTextCap, d_tst_, stream_);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h_texts_, d_texts_, size_t(kTextCap) * size_t(n), cudaMemcpyDeviceToHost, stream_);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_tst_, d_tst_, sizeof(int) * size_t(n), cudaMemcpyDeviceToHost, stream_);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream_);
  if (e != cudaSuccess) { err = std::string("answers: ") + cudaGetErrorString(e); return LSYN_E_CUDA; }
  for (int i = 0; i < n; ++i) {
    Job* j = solved[size_t(i)];
    if (h_tst_[i] != 0) {
      j->err = "formula too deep or too long to print";
      finish(j, LSYN_E_STATE);
      continue;
    }
    j->formula.assign(h_texts_ + size_t(i) * kTextCap, strnlen(h_texts_ + size_t(i) * kTextCap, kTextCap));
    j->found = 1;
    j->size = j->c->levels_done;
    j->exact = 1;
    finish(j, LSYN_OK);
  }
  return LSYN_OK;
}

lsyn_status Engine::run_group(std::vector<Plan>& g, int word_bits, int sms) {
  const int n = int(g.size());
  const unsigned R = rows_per_item();
  const unsigned long long warps = (unsigned long long)sms * unsigned(tune_.blocks_per_sm) * 8ull;
  // 1. plan every job's level and pack the step array
  unsigned long long tu = 0, tb = 0, td = 0;
  for (int i = 0; i < n; ++i) {
    Plan& p = g[size_t(i)];
    lsyn_ctx* c = p.j->c;
    ctx_level_plan(c, p.k, &p.lp);
    if (p.lp.plan.n_splits > kBatchSplits) {
      err = "too many splits for a batch level";
      return LSYN_E_UNSUPPORTED;
    }
    // Warps move between problems and return their unused ids at each move:
    // size the id chunk by this job's expected inserts over the launch's warps.
    const unsigned long long cand = candidates(p.j, p.k);
    c->chunk = unsigned(std::max(1ull, std::min<unsigned long long>(c->chunk, (cand + 32ull) / (8ull * warps))));
    StepProblem& sp = h_steps_[i];
    memset(&sp, 0, sizeof(sp));
    sp.cv = c->view(c->defer[0], &c->ctr->defer_n[0]);
    sp.d_items_begin = td;
    sp.u_items_begin = tu;
    sp.b_items_begin = tb;
    if (p.k == 1) {
      sp.d_n = unsigned(c->n_props);
      sp.d_list = nullptr;
      td += (sp.d_n + 31u) / 32u;
    } else {
      sp.u_first = p.lp.u_first;
      sp.u_count = p.lp.u_count;
      sp.u_ops = p.lp.uops;
      tu += (sp.u_count + R - 1u) / R;
      sp.b_ops = p.lp.plan.ops;
      sp.n_splits = uint32_t(p.lp.plan.n_splits);
      for (int t = 0; t < p.lp.plan.n_splits; ++t) sp.s[t] = p.lp.plan.s[t];
      tb += (p.lp.plan.total_pairs + R - 1ull) / R;
    }
  }
  memset(h_hdr_, 0, sizeof(StepHeader));
  h_hdr_->total_u = tu;
  h_hdr_->total_b = tb;
  h_hdr_->total_d = td;
  h_hdr_->n = n;
  h_hdr_->rows = int(R);
  const double tr = now_ms();
  lsyn_status s = launch_step(word_bits, n, sms);
  if (s != LSYN_OK) return s;
  cur_.run_ms += now_ms() - tr;
  cur_.active += n;
  for (const Plan& p : g) cur_.candidates += h_ctrs_[p.j->slot].built();

  // 2. deferred candidates of every job, one launch per pass
  for (int pass = 0;; ++pass) {
    std::vector<int> need;
    for (int i = 0; i < n; ++i) {
      const Plan& p = g[size_t(i)];
      const DevCounters& h = h_ctrs_[p.j->slot];
      if (h.defer_overflow) { err = "deferred list overflow"; return LSYN_E_STATE; }
      if (h.error) { err = "consistency check " + std::to_string(h.error) + " failed"; return LSYN_E_STATE; }
      if (std::min(h.defer_n[p.cur], p.j->c->defer_cap)) need.push_back(i);
    }
    if (need.empty()) break;
    if (pass >= 48) { err = "deferred candidates did not settle"; return LSYN_E_STATE; }
    ++cur_.passes;
    unsigned long long td2 = 0;
    for (size_t q = 0; q < need.size(); ++q) {
      Plan& p = g[size_t(need[q])];
      lsyn_ctx* c = p.j->c;
      const unsigned cnt = std::min(h_ctrs_[p.j->slot].defer_n[p.cur], c->defer_cap);
      p.deferred += cnt;
      cudaError_t e = cudaMemsetAsync(&c->ctr->defer_n[1 - p.cur], 0, sizeof(unsigned), stream_);
      if (e != cudaSuccess) { err = cudaGetErrorString(e); return LSYN_E_CUDA; }
      StepProblem& sp = h_steps_[q];
      memset(&sp, 0, sizeof(sp));
      sp.cv = c->view(c->defer[1 - p.cur], &c->ctr->defer_n[1 - p.cur]);
      sp.cv.early_exit = 0;  // a deferred candidate must be settled even after a solution
      sp.d_list = c->defer[p.cur];
      sp.d_n = cnt;
      sp.d_items_begin = td2;
      td2 += (cnt + 31u) / 32u;
      p.cur = 1 - p.cur;
    }
    memset(h_hdr_, 0, sizeof(StepHeader));
    h_hdr_->total_d = td2;
    h_hdr_->n = int(need.size());
    h_hdr_->rows = int(R);
    if ((s = launch_plain(word_bits, int(need.size()), sms)) != LSYN_OK) return s;
  }

  // 3. levels that outgrew the prediction are undone (unless a solution settles them)
  for (Plan& p : g) {
    lsyn_ctx* c = p.j->c;
    const DevCounters& h = h_ctrs_[p.j->slot];
    p.undo = h.full && c->max_entries < p.j->cap_entries && (!h.solved || c->full_levels);
    p.total = std::min(h.n_entries, c->max_entries);
  }

  // 4. hole fixups of the kept levels: stage the hole logs, plan, one launch
  size_t n_holes = 0;
  for (const Plan& p : g) {
    const DevCounters& h = h_ctrs_[p.j->slot];
    if (p.undo || !h.holes_n) continue;
    if (h.holes_n > hole_cap_) { err = "hole log overflow"; return LSYN_E_STATE; }
    n_holes += h.holes_n;
  }
  if (n_holes) {
    if (n_holes > h_holes_cap_) {
      cudaFreeHost(h_holes_);
      h_holes_cap_ = std::max(n_holes, 2 * h_holes_cap_);
      if (!pinned(&h_holes_, h_holes_cap_)) { err = "pinned host allocation failed"; return LSYN_E_NOMEM; }
    }
    std::vector<size_t> at(size_t(n), 0);
    size_t off = 0;
    for (int i = 0; i < n; ++i) {
      const Plan& p = g[size_t(i)];
      const DevCounters& h = h_ctrs_[p.j->slot];
      at[size_t(i)] = off;
      if (p.undo || !h.holes_n) continue;
      cudaError_t e = cudaMemcpyAsync(h_holes_ + off, p.j->c->holes, h.holes_n * sizeof(uint2), cudaMemcpyDeviceToHost,
                                      stream_);
      if (e != cudaSuccess) { err = cudaGetErrorString(e); return LSYN_E_CUDA; }
      off += h.holes_n;
    }
    cudaError_t e = cudaStreamSynchronize(stream_);
    if (e != cudaSuccess) { err = std::string("hole log copy: ") + cudaGetErrorString(e); return LSYN_E_CUDA; }
    std::vector<uint4> mv_all;
    for (int i = 0; i < n; ++i) {
      Plan& p = g[size_t(i)];
      lsyn_ctx* c = p.j->c;
      const DevCounters& h = h_ctrs_[p.j->slot];
      memset(&h_steps_[i], 0, sizeof(StepProblem));
      h_steps_[i].cv = c->view(c->defer[0], &c->ctr->defer_n[0]);
      h_dense_[i] = 0xFFFFFFFFu;
      if (p.undo || !h.holes_n) continue;
      std::vector<uint2> mv;
      const uint32_t dense = plan_hole_moves(h_holes_ + at[size_t(i)], h.holes_n, p.lp.start, p.total, &mv);
      for (const uint2& m : mv) mv_all.push_back(make_uint4(unsigned(i), m.x, m.y, 0));
      p.total = dense;
      h_dense_[i] = dense;
    }
    if (mv_all.size() > move_cap_) { err = "too many hole moves"; return LSYN_E_STATE; }
    e = cudaMemcpyAsync(d_steps_, h_steps_, sizeof(StepProblem) * size_t(n), cudaMemcpyHostToDevice, stream_);
    if (e == cudaSuccess && !mv_all.empty())
      e = cudaMemcpyAsync(d_moves_, mv_all.data(), mv_all.size() * sizeof(uint4), cudaMemcpyHostToDevice, stream_);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_dense_, h_dense_, sizeof(unsigned) * size_t(n), cudaMemcpyHostToDevice, stream_);
    LaunchCfg lc{stream_, sms};
    if (e == cudaSuccess)
      e = word_bits == 32
              ? Kernels<uint32_t>::batch_fixup(d_steps_, d_moves_, unsigned(mv_all.size()), d_dense_, n, lc)
              : Kernels<uint64_t>::batch_fixup(d_steps_, d_moves_, unsigned(mv_all.size()), d_dense_, n, lc);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h_ctrs_, ctrs_, sizeof(DevCounters) * slots_.size(), cudaMemcpyDeviceToHost, stream_);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream_);
    if (e != cudaSuccess) { err = std::string("batch fixup: ") + cudaGetErrorString(e); return LSYN_E_CUDA; }
  }

  // 5. commit, answer, or schedule the redo
  std::vector<Job*> solved;
  for (Plan& p : g) {
    Job* j = p.j;
    lsyn_ctx* c = j->c;
    const DevCounters h = h_ctrs_[j->slot];
    if (p.undo) {
      j->redo = true;
      ++j->redos;
      ++redos_;
      continue;
    }
    if (h.error) { err = "hole fixup found an inconsistent slot"; return LSYN_E_STATE; }
    lsyn_level_stats st;
    s = ctx_commit_level(c, p.k, h, p.total, p.deferred, p.lp, &st);
    if (s != LSYN_OK) { err = c->err; return s; }
    j->redo = false;
    if (st.candidates > 0 && !st.early_exit) j->ratio = double(st.unique) / double(st.candidates);
    if (st.solved) {
      solved.push_back(j);
    } else if (st.cache_full) {
      if (j->err.empty()) j->err = "language cache full at level " + std::to_string(p.k);
      finish(j, LSYN_E_CACHE_FULL);
    }
  }
  return answer(solved);
}

// ---------------------------------------------------------------------------
// Large-level lane
// ---------------------------------------------------------------------------

void Engine::lane_fail(Lane& L, lsyn_status s, const std::string& m) {
  Job* j = L.j;
  if (!j) return;
  j->in_flight = false;
  j->err = m;
  finish(j, s);
  lane_done(L);
}

lsyn_status Engine::lane_launch(Lane& L, Job* j, bool* progressed) {
  const double t0 = now_ms();
  lsyn_ctx* c = j->c;
  const int k = c->levels_done + 1;
  const unsigned long long cand = candidates(j, k);
  bool ok = false;
  lsyn_status s = grow(j, predict_entries(j, k, cand), &L, &ok);
  if (s != LSYN_OK) return s;
  if (!ok && release_finished()) {
    *progressed = true;
    if ((s = grow(j, predict_entries(j, k, cand), &L, &ok)) != LSYN_OK) return s;
  }
  j->paused = !ok;
  if (!ok) return LSYN_OK;
  ctx_level_plan(c, k, &L.lp);
  // leave SMs to the batch steps while small levels are in the system
  bool light = !queue_.empty();
  for (const Job* x : active_) light = light || (!x->heavy && x != j);
  const LaunchCfg lc{L.stream, light ? sms_ - light_sms() : sms_};
  const CacheView cv = c->view(c->defer[0], &c->ctr->defer_n[0]);
  // CMs above 512 bytes (path D): the unary launch and the deferred passes
  // reserve exactly each batch's ids, as on the one-problem path. Ids a warp
  // leaves unused count against the job's entries until the level closes, so
  // chunks held by many warps (a deferred pass spreads a short list over many
  // warps) could fill a cache at its cap that the one-problem path fits.
  CacheView uv = cv;
  if (c->vecs > 32u) uv.chunk = 1;
  cudaError_t e = launch_level_begin(c->ctr, L.stream);
  if (e == cudaSuccess && L.lp.uops && L.lp.u_count)
    e = c->word_bits == 32 ? Kernels<uint32_t>::unary(uv, L.lp.u_first, L.lp.u_count, L.lp.uops, lc)
                           : Kernels<uint64_t>::unary(uv, L.lp.u_first, L.lp.u_count, L.lp.uops, lc);
  if (e == cudaSuccess && L.lp.plan.n_splits > 0)
    e = c->word_bits == 32 ? Kernels<uint32_t>::binary(cv, L.lp.plan, lc)
                           : Kernels<uint64_t>::binary(cv, L.lp.plan, lc);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&L.snap[0], c->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, L.stream);
  // The first pass over the deferred candidates and the hole close are queued
  // behind the level's kernels (both read their counts on the device).
  if (e == cudaSuccess) e = cudaMemsetAsync(&c->ctr->defer_n[1], 0, sizeof(unsigned), L.stream);
  if (e == cudaSuccess) {
    CacheView rv = c->view(c->defer[1], &c->ctr->defer_n[1]);
    rv.early_exit = 0;  // a deferred candidate must be settled even after a solution
    if (c->vecs > 32u) rv.chunk = 1;
    e = c->word_bits == 32 ? Kernels<uint32_t>::desc_list(rv, c->defer[0], &c->ctr->defer_n[0], c->defer_cap, 0, lc)
                           : Kernels<uint64_t>::desc_list(rv, c->defer[0], &c->ctr->defer_n[0], c->defer_cap, 0, lc);
  }
  if (e == cudaSuccess)
    e = c->word_bits == 32 ? Kernels<uint32_t>::close_holes(cv, L.lp.start, L.d_bits, L.d_moves, move_cap_, lc)
                           : Kernels<uint64_t>::close_holes(cv, L.lp.start, L.d_bits, L.d_moves, move_cap_, lc);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&L.snap[1], c->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, L.stream);
  if (e == cudaSuccess) e = cudaEventRecord(L.ev, L.stream);
  if (e != cudaSuccess) { err = std::string("large level: ") + cudaGetErrorString(e); return LSYN_E_CUDA; }
  L.j = j;
  L.k = k;
  L.cur = 1;
  L.closed = true;
  L.first = true;
  L.passes = 0;
  L.deferred = 0;
  L.total = 0;
  L.stage = Lane::kRun;
  ++large_levels_;
  j->in_flight = true;
  L.t0 = t0;
  L.t_launched = now_ms();
  L.ran = false;
  memset(&L.rec, 0, sizeof(L.rec));
  L.rec.step = int64_t(steps_);
  L.rec.lane = 1;
  L.rec.active = 1;
  L.rec.level = k;
  L.rec.plan_ms = L.t_launched - t0;
  *progressed = true;
  return LSYN_OK;
}

lsyn_status Engine::lane_commit(Lane& L) {
  Job* j = L.j;
  lsyn_ctx* c = j->c;
  lsyn_level_stats st;
  lsyn_status s = ctx_commit_level(c, L.k, L.snap[1], L.total, L.deferred, L.lp, &st);
  if (s != LSYN_OK) {
    lane_fail(L, s, c->err);
    return LSYN_OK;
  }
  j->redo = false;
  if (st.candidates > 0 && !st.early_exit) j->ratio = double(st.unique) / double(st.candidates);
  if (st.solved) {
    *L.h_item = FormulaItem{c->prov, &c->ctr->sol};
    cudaError_t e = cudaMemcpyAsync(L.d_item, L.h_item, sizeof(FormulaItem), cudaMemcpyHostToDevice,
                                    L.stream);
    if (e == cudaSuccess) e = reconstruct_many(L.d_item, 1, L.d_text, kTextCap, L.d_tst, L.stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(L.h_text, L.d_text, kTextCap, cudaMemcpyDeviceToHost, L.stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(L.h_tst, L.d_tst, sizeof(int), cudaMemcpyDeviceToHost, L.stream);
    if (e == cudaSuccess) e = cudaEventRecord(L.ev, L.stream);
    if (e != cudaSuccess) { err = std::string("answer: ") + cudaGetErrorString(e); return LSYN_E_CUDA; }
    L.stage = Lane::kAnswer;
    return LSYN_OK;
  }
  j->in_flight = false;
  if (st.cache_full) {
    if (j->err.empty()) j->err = "language cache full at level " + std::to_string(L.k);
    finish(j, LSYN_E_CACHE_FULL);
  } else {
    j->heavy = candidates(j, L.k + 1) > solo_min();
  }
  lane_done(L);
  return LSYN_OK;
}

lsyn_status Engine::lane_advance(Lane& L, bool* progressed) {
  if (L.stage == Lane::kIdle) {
    Job* pick = nullptr;
    for (Job* j : active_)
      if (j->heavy && !j->in_flight && (!pick || j->seq < pick->seq)) pick = j;
    if (!pick) return LSYN_OK;
    if (pick->c->levels_done + 1 > pick->max_size) {
      finish(pick, LSYN_NOT_FOUND);
      *progressed = true;
      return LSYN_OK;
    }
    return lane_launch(L, pick, progressed);
  }
  const cudaError_t q = cudaEventQuery(L.ev);
  if (q == cudaErrorNotReady) return LSYN_OK;
  if (q != cudaSuccess) { err = std::string("large level: ") + cudaGetErrorString(q); return LSYN_E_CUDA; }
  *progressed = true;
  if (L.old_table) {  // the rebuild that replaced it has run
    bool current = false;
    for (Slot& sl : slots_)
      if (&sl.table[sl.cur_table] == L.old_table) current = true;
    if (!current) L.old_table->shrink(pool_, 0);
    L.old_table = nullptr;
  }
  Job* j = L.j;
  lsyn_ctx* c = j->c;
  const LaunchCfg lc{L.stream, sms_};
  const DevCounters& h = L.snap[1];
  if (!L.ran) {
    L.ran = true;
    L.rec.run_ms = now_ms() - L.t_launched;
    L.rec.candidates = h.built();
  }
  cudaError_t e = cudaSuccess;
  switch (L.stage) {
    case Lane::kRun: {
      if (L.first) {  // the level's own deferred candidates were settled by the queued first pass
        L.first = false;
        const unsigned n0 = std::min(L.snap[0].defer_n[0], c->defer_cap);
        if (n0) {
          L.deferred += n0;
          ++L.passes;
          ++L.rec.passes;
        }
      }
      if (h.defer_overflow) { lane_fail(L, LSYN_E_STATE, "deferred list overflow"); return LSYN_OK; }
      if (h.error) { lane_fail(L, LSYN_E_STATE, "consistency check " + std::to_string(h.error) + " failed"); return LSYN_OK; }
      const unsigned nd = std::min(h.defer_n[L.cur], c->defer_cap);
      if (nd) {
        if (L.passes >= 48) { lane_fail(L, LSYN_E_STATE, "deferred candidates did not settle"); return LSYN_OK; }
        const int cur = L.cur;
        e = cudaMemsetAsync(&c->ctr->defer_n[1 - cur], 0, sizeof(unsigned), L.stream);
        CacheView rv = c->view(c->defer[1 - cur], &c->ctr->defer_n[1 - cur]);
        rv.early_exit = 0;  // a deferred candidate must be settled even after a solution
        if (c->vecs > 32u) rv.chunk = 1;  // as the level's first pass
        if (e == cudaSuccess)
          e = c->word_bits == 32 ? Kernels<uint32_t>::desc_list(rv, c->defer[cur], &c->ctr->defer_n[cur], nd, 0, lc)
                                 : Kernels<uint64_t>::desc_list(rv, c->defer[cur], &c->ctr->defer_n[cur], nd, 0, lc);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(&L.snap[1], c->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, L.stream);
        if (e == cudaSuccess) e = cudaEventRecord(L.ev, L.stream);
        if (e != cudaSuccess) { err = std::string("deferred pass: ") + cudaGetErrorString(e); return LSYN_E_CUDA; }
        L.cur = 1 - cur;
        ++L.passes;
        ++L.rec.passes;
        L.deferred += nd;
        L.closed = false;
        return LSYN_OK;
      }
      if (h.full && c->max_entries < j->cap_entries && (!h.solved || c->full_levels)) {
        j->redo = true;  // outgrew its prediction: undo and run again with room for every candidate
        ++j->redos;
        ++redos_;
        lane_done(L);
        return LSYN_OK;
      }
      if (!L.closed) {  // close the holes the later passes left
        const CacheView cv = c->view(c->defer[0], &c->ctr->defer_n[0]);
        e = c->word_bits == 32 ? Kernels<uint32_t>::close_holes(cv, L.lp.start, L.d_bits, L.d_moves, move_cap_, lc)
                               : Kernels<uint64_t>::close_holes(cv, L.lp.start, L.d_bits, L.d_moves, move_cap_, lc);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(&L.snap[1], c->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, L.stream);
        if (e == cudaSuccess) e = cudaEventRecord(L.ev, L.stream);
        if (e != cudaSuccess) { err = std::string("hole fixup: ") + cudaGetErrorString(e); return LSYN_E_CUDA; }
        L.closed = true;
        return LSYN_OK;
      }
      L.total = std::min(h.n_entries, c->max_entries);
      return lane_commit(L);
    }
    case Lane::kAnswer: {
      j->in_flight = false;
      if (*L.h_tst != 0) {
        j->err = "formula too deep or too long to print";
        finish(j, LSYN_E_STATE);
      } else {
        j->formula.assign(L.h_text, strnlen(L.h_text, kTextCap));
        j->found = 1;
        j->size = c->levels_done;
        j->exact = 1;
        finish(j, LSYN_OK);
      }
      lane_done(L);
      return LSYN_OK;
    }
    default:
      return LSYN_OK;
  }
}

}  // namespace lsyn
