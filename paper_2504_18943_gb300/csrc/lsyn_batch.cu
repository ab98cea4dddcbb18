// Batched solving: many independent specifications enumerated together.
//
// Every problem keeps its own language cache (arena, provenance, table) and
// sits at its own level. A batch step advances every unfinished problem by one
// level: the host plans each problem's level (as lsyn_enumerate_level does),
// packs the plans into one step array, and a single persistent launch
// (k_batch_run) works through the atoms / unary / binary work of all of them
// from one packed work list. Counters of all problems are contiguous, so a step
// needs one device-to-host copy to decide what comes next; deferred
// candidates and hole fixups are batched the same way. The upload, the reset,
// the persistent launch and the copy back can be replayed from a captured CUDA
// graph (lsyn_batch_tuning.use_graph).
#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lsyn.h"
#include "lsyn_ctx.h"
#include "lsyn_device.cuh"
#include "lsyn_internal.h"

using namespace lsyn;

struct lsyn_batch {
  int n = 0;
  int word_bits = 64;
  int device = 0;
  int sms = 1;
  cudaStream_t stream = nullptr;
  std::vector<lsyn_ctx*> ctx;
  Alloc mem;
  DevCounters* ctrs = nullptr;    // device [n]
  DevCounters* h_ctrs = nullptr;  // pinned [n]
  uint2* holes = nullptr;         // device [n][hole_cap]
  unsigned hole_cap = 0;
  StepHeader* d_hdr = nullptr;
  StepProblem* d_steps = nullptr;
  StepHeader* h_hdr = nullptr;    // pinned
  StepProblem* h_steps = nullptr; // pinned [n]
  uint4* d_moves = nullptr;
  unsigned move_cap = 0;
  unsigned* d_dense = nullptr;    // device [n]
  unsigned* h_dense = nullptr;    // pinned [n]
  lsyn_batch_tuning tune;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  bool own_stream = false;
  std::string err;

  lsyn_status fail(lsyn_status s, const std::string& m) {
    err = m;
    return s;
  }
  lsyn_status cuda_fail(cudaError_t e, const char* where) {
    err = std::string(where) + ": " + cudaGetErrorString(e);
    return LSYN_E_CUDA;
  }
};

namespace {

thread_local std::string g_batch_error;

lsyn_status run_step(lsyn_batch* b, int n_active) {
  LaunchCfg lc{b->stream, b->sms};
  cudaError_t e;
  if (b->tune.use_graph) {
    if (!b->graph_exec) {
      e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return b->cuda_fail(e, "graph capture");
      cudaMemcpyAsync(b->d_hdr, b->h_hdr, sizeof(StepHeader), cudaMemcpyHostToDevice, b->stream);
      cudaMemcpyAsync(b->d_steps, b->h_steps, sizeof(StepProblem) * b->n, cudaMemcpyHostToDevice, b->stream);
      if (b->word_bits == 32) {
        Kernels<uint32_t>::batch_begin(b->d_hdr, b->d_steps, b->n, lc);
        Kernels<uint32_t>::batch_run(b->d_hdr, b->d_steps, lc, b->tune.blocks_per_sm);
      } else {
        Kernels<uint64_t>::batch_begin(b->d_hdr, b->d_steps, b->n, lc);
        Kernels<uint64_t>::batch_run(b->d_hdr, b->d_steps, lc, b->tune.blocks_per_sm);
      }
      cudaMemcpyAsync(b->h_ctrs, b->ctrs, sizeof(DevCounters) * b->n, cudaMemcpyDeviceToHost, b->stream);
      e = cudaStreamEndCapture(b->stream, &b->graph);
      if (e != cudaSuccess) return b->cuda_fail(e, "graph capture");
      e = cudaGraphInstantiate(&b->graph_exec, b->graph, 0);
      if (e != cudaSuccess) return b->cuda_fail(e, "graph instantiate");
    }
    e = cudaGraphLaunch(b->graph_exec, b->stream);
    if (e != cudaSuccess) return b->cuda_fail(e, "graph launch");
  } else {
    e = cudaMemcpyAsync(b->d_hdr, b->h_hdr, sizeof(StepHeader), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b->d_steps, b->h_steps, sizeof(StepProblem) * n_active, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
      e = b->word_bits == 32 ? Kernels<uint32_t>::batch_begin(b->d_hdr, b->d_steps, n_active, lc)
                             : Kernels<uint64_t>::batch_begin(b->d_hdr, b->d_steps, n_active, lc);
    if (e == cudaSuccess)
      e = b->word_bits == 32 ? Kernels<uint32_t>::batch_run(b->d_hdr, b->d_steps, lc, b->tune.blocks_per_sm)
                             : Kernels<uint64_t>::batch_run(b->d_hdr, b->d_steps, lc, b->tune.blocks_per_sm);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b->h_ctrs, b->ctrs, sizeof(DevCounters) * b->n, cudaMemcpyDeviceToHost, b->stream);
    if (e != cudaSuccess) return b->cuda_fail(e, "batch step");
  }
  e = cudaStreamSynchronize(b->stream);
  return e == cudaSuccess ? LSYN_OK : b->cuda_fail(e, "batch step sync");
}

// Deferred-only or hole passes reuse the step arrays without the reset kernel.
lsyn_status run_plain(lsyn_batch* b, int n_active) {
  LaunchCfg lc{b->stream, b->sms};
  cudaError_t e = cudaMemcpyAsync(b->d_hdr, b->h_hdr, sizeof(StepHeader), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_steps, b->h_steps, sizeof(StepProblem) * n_active, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = b->word_bits == 32 ? Kernels<uint32_t>::batch_run(b->d_hdr, b->d_steps, lc, b->tune.blocks_per_sm)
                           : Kernels<uint64_t>::batch_run(b->d_hdr, b->d_steps, lc, b->tune.blocks_per_sm);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->h_ctrs, b->ctrs, sizeof(DevCounters) * b->n, cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  return e == cudaSuccess ? LSYN_OK : b->cuda_fail(e, "batch pass");
}

}  // namespace

extern "C" {

void lsyn_batch_destroy(lsyn_batch* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (lsyn_ctx* c : b->ctx) lsyn_destroy(c);
  b->mem.release_all();
  if (b->h_ctrs) cudaFreeHost(b->h_ctrs);
  if (b->h_hdr) cudaFreeHost(b->h_hdr);
  if (b->h_steps) cudaFreeHost(b->h_steps);
  if (b->h_dense) cudaFreeHost(b->h_dense);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

lsyn_status lsyn_batch_problem(lsyn_batch* b, int32_t i, lsyn_ctx** out) {
  if (!b || !out || i < 0 || i >= b->n) return LSYN_E_INVAL;
  *out = b->ctx[i];
  return LSYN_OK;
}

const char* lsyn_batch_last_error(const lsyn_batch* b) { return b ? b->err.c_str() : g_batch_error.c_str(); }

lsyn_status lsyn_batch_create(const lsyn_problem* problems, int32_t n, const lsyn_config* config,
                              const lsyn_batch_tuning* tuning, lsyn_batch** out) {
  g_batch_error.clear();
  if (!out || !problems || n < 1) {
    g_batch_error = "problems, n >= 1 and out are required";
    return LSYN_E_INVAL;
  }
  *out = nullptr;
  for (int i = 1; i < n; ++i)
    if (problems[i].word_bits != problems[0].word_bits) {
      g_batch_error = "every problem of a batch must use the same word_bits";
      return LSYN_E_INVAL;
    }
  lsyn_batch* b = new (std::nothrow) lsyn_batch;
  if (!b) return LSYN_E_NOMEM;
  b->n = n;
  b->word_bits = problems[0].word_bits;
  memset(&b->tune, 0, sizeof(b->tune));
  if (tuning) b->tune = *tuning;
  if (b->tune.blocks_per_sm < 1) b->tune.blocks_per_sm = 4;
  lsyn_config cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.device = -1;
  if (config) cfg = *config;
  auto bail = [&](lsyn_status st, const std::string& msg) {
    g_batch_error = msg;
    lsyn_batch_destroy(b);
    return st;
  };
  cudaError_t e;
  if (cfg.device >= 0 && (e = cudaSetDevice(cfg.device)) != cudaSuccess) return bail(LSYN_E_CUDA, cudaGetErrorString(e));
  if ((e = cudaGetDevice(&b->device)) != cudaSuccess) return bail(LSYN_E_CUDA, cudaGetErrorString(e));
  cudaDeviceProp prop;
  if ((e = cudaGetDeviceProperties(&prop, b->device)) != cudaSuccess) return bail(LSYN_E_CUDA, cudaGetErrorString(e));
  b->sms = prop.multiProcessorCount;
  b->stream = static_cast<cudaStream_t>(cfg.stream);
  if (!b->stream) {  // the legacy default stream cannot be captured into a graph
    if ((e = cudaStreamCreate(&b->stream)) != cudaSuccess) return bail(LSYN_E_CUDA, cudaGetErrorString(e));
    b->own_stream = true;
    cfg.stream = b->stream;
  }
  b->mem.alloc = cfg.alloc;
  b->mem.free = cfg.free;
  b->mem.user = cfg.alloc_user;
  b->hole_cap = 16384;
  b->move_cap = 1u << 22;
  b->ctrs = static_cast<DevCounters*>(b->mem.get(sizeof(DevCounters) * n));
  b->holes = static_cast<uint2*>(b->mem.get(sizeof(uint2) * size_t(b->hole_cap) * n));
  b->d_hdr = static_cast<StepHeader*>(b->mem.get(sizeof(StepHeader)));
  b->d_steps = static_cast<StepProblem*>(b->mem.get(sizeof(StepProblem) * n));
  b->d_moves = static_cast<uint4*>(b->mem.get(sizeof(uint4) * size_t(b->move_cap)));
  b->d_dense = static_cast<unsigned*>(b->mem.get(sizeof(unsigned) * n));
  if (!b->ctrs || !b->holes || !b->d_hdr || !b->d_steps || !b->d_moves || !b->d_dense)
    return bail(LSYN_E_NOMEM, "device allocation failed");
  if (cudaMallocHost(&b->h_ctrs, sizeof(DevCounters) * n) != cudaSuccess ||
      cudaMallocHost(&b->h_hdr, sizeof(StepHeader)) != cudaSuccess ||
      cudaMallocHost(&b->h_steps, sizeof(StepProblem) * n) != cudaSuccess ||
      cudaMallocHost(&b->h_dense, sizeof(unsigned) * n) != cudaSuccess) {
    cudaGetLastError();
    return bail(LSYN_E_NOMEM, "pinned host allocation failed");
  }
  memset(b->h_steps, 0, sizeof(StepProblem) * n);
  if ((e = cudaMemsetAsync(b->ctrs, 0, sizeof(DevCounters) * n, b->stream)) != cudaSuccess)
    return bail(LSYN_E_CUDA, cudaGetErrorString(e));
  b->ctx.assign(n, nullptr);
  for (int i = 0; i < n; ++i) {
    lsyn_status s = ctx_create(&problems[i], &cfg, true, &b->ctx[i]);
    if (s != LSYN_OK) return bail(s, "problem " + std::to_string(i) + ": " + thread_error());
    // The batch owns the counters and hole logs, contiguous for one-copy steps.
    b->ctx[i]->ctr = b->ctrs + i;
    b->ctx[i]->holes = b->holes + size_t(i) * b->hole_cap;
    b->ctx[i]->hole_cap = b->hole_cap;
  }
  if ((e = cudaStreamSynchronize(b->stream)) != cudaSuccess) return bail(LSYN_E_CUDA, cudaGetErrorString(e));
  *out = b;
  return LSYN_OK;
}

lsyn_status lsyn_batch_solve(lsyn_batch* b, int32_t max_size, lsyn_result* results, int32_t* statuses) {
  if (!b || !results || !statuses) return LSYN_E_INVAL;
  if (max_size < 1 || max_size > 17) return b->fail(LSYN_E_INVAL, "max_size must be in 1..17 for a batch");
  cudaSetDevice(b->device);
  const double t0 = now_ms();
  const int n = b->n;
  std::vector<int> running(n, 1), cur(n, 0);
  std::vector<unsigned long long> deferred(n, 0);
  std::vector<LevelPlan> lp(n);
  std::vector<int> act, slot_of(n, -1);
  for (int i = 0; i < n; ++i) {
    lsyn_status s = lsyn_reset(b->ctx[i]);
    if (s != LSYN_OK) return b->fail(s, b->ctx[i]->err);
    b->ctx[i]->ctr = b->ctrs + i;
    results[i].found = results[i].size = results[i].exact = 0;
    results[i].levels_done = 0;
    results[i].constructed = results[i].unique = 0;
    results[i].launches = 0;
    results[i].ms = 0;
    statuses[i] = LSYN_PENDING;
  }
  cudaError_t e = cudaMemsetAsync(b->ctrs, 0, sizeof(DevCounters) * n, b->stream);
  if (e != cudaSuccess) return b->cuda_fail(e, "reset");
  int steps_run = 0;
  while (true) {
    // 1. plan the next level of every running problem
    act.clear();
    for (int i = 0; i < n; ++i) {
      if (!running[i]) continue;
      lsyn_ctx* c = b->ctx[i];
      const int k = c->levels_done + 1;
      if (k > max_size) {
        running[i] = 0;
        statuses[i] = LSYN_NOT_FOUND;
        results[i].ms = now_ms() - t0;
        continue;
      }
      ctx_level_plan(c, k, &lp[i]);
      if (lp[i].plan.n_splits > kBatchSplits) return b->fail(LSYN_E_UNSUPPORTED, "too many splits for a batch level");
      // In a batch, warps move between problems and return their unused ids
      // at each move: size this problem's id chunk by its own expected inserts
      // (about half its candidates) over the warps of the launch.
      {
        const unsigned long long cand = 4ull * lp[i].u_count + 4ull * lp[i].plan.total_pairs + 32ull;
        const unsigned long long warps = (unsigned long long)b->sms * b->tune.blocks_per_sm * 8ull;
        c->chunk = unsigned(std::max(1ull, std::min<unsigned long long>(c->chunk, cand / (2ull * 4ull * warps))));
      }
      slot_of[i] = int(act.size());
      act.push_back(i);
    }
    if (act.empty()) break;
    unsigned long long tu = 0, tb = 0, td = 0;
    for (size_t j = 0; j < act.size(); ++j) {
      const int i = act[j];
      lsyn_ctx* c = b->ctx[i];
      const int k = c->levels_done + 1;
      StepProblem& sp = b->h_steps[j];
      memset(&sp, 0, sizeof(sp));
      sp.cv = c->view(c->defer[0], &c->ctr->defer_n[0]);
      sp.d_items_begin = td;
      sp.u_items_begin = tu;
      sp.b_items_begin = tb;
      if (k == 1) {
        sp.d_n = unsigned(c->n_props);
        sp.d_list = nullptr;
        td += (sp.d_n + 31u) / 32u;
      } else {
        sp.u_first = lp[i].u_first;
        sp.u_count = lp[i].u_count;
        sp.u_ops = lp[i].uops;
        tu += (sp.u_count + 7u) / 8u;
        sp.b_ops = lp[i].plan.ops;
        sp.n_splits = uint32_t(lp[i].plan.n_splits);
        for (int t = 0; t < lp[i].plan.n_splits; ++t) sp.s[t] = lp[i].plan.s[t];
        tb += (lp[i].plan.total_pairs + 7ull) / 8ull;
      }
      cur[i] = 0;
      deferred[i] = 0;
    }
    memset(b->h_hdr, 0, sizeof(StepHeader));
    b->h_hdr->total_u = tu;
    b->h_hdr->total_b = tb;
    b->h_hdr->total_d = td;
    b->h_hdr->n = int(act.size());
    lsyn_status s = run_step(b, int(act.size()));
    if (s != LSYN_OK) return s;
    ++steps_run;

    // 2. deferred candidates, problem by problem in one pass
    for (int pass = 0;; ++pass) {
      std::vector<int> need;
      for (int i : act) {
        const DevCounters& h = b->h_ctrs[i];
        if (h.defer_overflow) return b->fail(LSYN_E_STATE, "deferred list overflow in problem " + std::to_string(i));
        if (h.error)
          return b->fail(LSYN_E_STATE, "consistency check " + std::to_string(h.error) + " failed in problem " +
                                           std::to_string(i));
        if (std::min(h.defer_n[cur[i]], b->ctx[i]->defer_cap)) need.push_back(i);
      }
      if (need.empty()) break;
      if (pass >= 48) return b->fail(LSYN_E_STATE, "deferred candidates did not settle");
      unsigned long long td2 = 0;
      for (size_t j = 0; j < need.size(); ++j) {
        const int i = need[j];
        lsyn_ctx* c = b->ctx[i];
        const unsigned cnt = std::min(b->h_ctrs[i].defer_n[cur[i]], c->defer_cap);
        deferred[i] += cnt;
        e = cudaMemsetAsync(&c->ctr->defer_n[1 - cur[i]], 0, sizeof(unsigned), b->stream);
        if (e != cudaSuccess) return b->cuda_fail(e, "memset");
        StepProblem& sp = b->h_steps[j];
        memset(&sp, 0, sizeof(sp));
        sp.cv = c->view(c->defer[1 - cur[i]], &c->ctr->defer_n[1 - cur[i]]);
        sp.cv.early_exit = 0;
        sp.d_list = c->defer[cur[i]];
        sp.d_n = cnt;
        sp.d_items_begin = td2;
        td2 += (cnt + 31u) / 32u;
        cur[i] = 1 - cur[i];
      }
      memset(b->h_hdr, 0, sizeof(StepHeader));
      b->h_hdr->total_d = td2;
      b->h_hdr->n = int(need.size());
      if ((s = run_plain(b, int(need.size()))) != LSYN_OK) return s;
    }

    // 3. hole fixups
    std::vector<uint4> mv_all;
    bool any_holes = false;
    std::vector<uint32_t> total(n, 0);
    for (size_t j = 0; j < act.size(); ++j) {
      const int i = act[j];
      lsyn_ctx* c = b->ctx[i];
      const DevCounters& h = b->h_ctrs[i];
      total[i] = std::min(h.n_entries, c->max_entries);
      b->h_dense[j] = 0xFFFFFFFFu;
      if (!h.holes_n) continue;
      if (h.holes_n > b->hole_cap) return b->fail(LSYN_E_STATE, "hole log overflow");
      std::vector<uint2> hr(h.holes_n);
      e = cudaMemcpyAsync(hr.data(), c->holes, hr.size() * sizeof(uint2), cudaMemcpyDeviceToHost, b->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
      if (e != cudaSuccess) return b->cuda_fail(e, "hole log copy");
      std::vector<uint2> mv;
      const uint32_t dense = plan_hole_moves(hr.data(), unsigned(hr.size()), lp[i].start, total[i], &mv);
      for (const uint2& m : mv) mv_all.push_back(make_uint4(unsigned(j), m.x, m.y, 0));
      total[i] = dense;
      b->h_dense[j] = dense;
      any_holes = true;
    }
    if (any_holes) {
      if (mv_all.size() > b->move_cap) return b->fail(LSYN_E_STATE, "too many hole moves");
      // the step array still describes `act` (index j): rebuild it (deferred passes reused it)
      for (size_t j = 0; j < act.size(); ++j) {
        const int i = act[j];
        lsyn_ctx* c = b->ctx[i];
        memset(&b->h_steps[j], 0, sizeof(StepProblem));
        b->h_steps[j].cv = c->view(c->defer[0], &c->ctr->defer_n[0]);
      }
      e = cudaMemcpyAsync(b->d_steps, b->h_steps, sizeof(StepProblem) * act.size(), cudaMemcpyHostToDevice, b->stream);
      if (e == cudaSuccess && !mv_all.empty())
        e = cudaMemcpyAsync(b->d_moves, mv_all.data(), mv_all.size() * sizeof(uint4), cudaMemcpyHostToDevice, b->stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_dense, b->h_dense, sizeof(unsigned) * act.size(), cudaMemcpyHostToDevice, b->stream);
      LaunchCfg lc{b->stream, b->sms};
      if (e == cudaSuccess)
        e = b->word_bits == 32
                ? Kernels<uint32_t>::batch_fixup(b->d_steps, b->d_moves, unsigned(mv_all.size()), b->d_dense,
                                                 int(act.size()), lc)
                : Kernels<uint64_t>::batch_fixup(b->d_steps, b->d_moves, unsigned(mv_all.size()), b->d_dense,
                                                 int(act.size()), lc);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->h_ctrs, b->ctrs, sizeof(DevCounters) * n, cudaMemcpyDeviceToHost, b->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
      if (e != cudaSuccess) return b->cuda_fail(e, "batch fixup");
    }

    // 4. commit every problem's level
    for (int i : act) {
      lsyn_ctx* c = b->ctx[i];
      const int k = c->levels_done + 1;
      const DevCounters h = b->h_ctrs[i];
      if (h.error) return b->fail(LSYN_E_STATE, "hole fixup found an inconsistent slot in problem " + std::to_string(i));
      lsyn_level_stats st;
      s = ctx_commit_level(c, k, h, total[i], deferred[i], lp[i], &st);
      if (s != LSYN_OK) return b->fail(s, "problem " + std::to_string(i) + ": " + c->err);
      results[i].levels_done = k;
      results[i].constructed = int64_t(c->constructed);
      results[i].unique = int64_t(c->level_start.back() + c->level_n.back());
      if (st.solved) {
        s = ctx_reconstruct(c, &c->ctr->sol, results[i].formula, results[i].formula_cap);
        if (s != LSYN_OK) return b->fail(s, "problem " + std::to_string(i) + ": " + c->err);
        results[i].found = 1;
        results[i].size = k;
        results[i].exact = 1;
        results[i].ms = now_ms() - t0;
        statuses[i] = LSYN_OK;
        running[i] = 0;
      } else if (st.cache_full) {
        results[i].ms = now_ms() - t0;
        statuses[i] = LSYN_E_CACHE_FULL;
        running[i] = 0;
      }
    }
  }
  for (int i = 0; i < n; ++i) results[i].launches = steps_run;
  return LSYN_OK;
}

lsyn_status lsyn_batch_autotune(lsyn_batch* b, int32_t max_size, lsyn_batch_tuning* out) {
  if (!b) return LSYN_E_INVAL;
  const int n = b->n;
  std::vector<lsyn_result> res(n);
  std::vector<int32_t> st(n);
  std::vector<std::vector<char>> fbuf(n, std::vector<char>(4096));
  for (int i = 0; i < n; ++i) {
    memset(&res[i], 0, sizeof(lsyn_result));
    res[i].formula = fbuf[i].data();
    res[i].formula_cap = fbuf[i].size();
  }
  const lsyn_batch_tuning saved = b->tune;
  lsyn_batch_tuning best = saved;
  double best_ms = 1e300;
  const int blocks[] = {2, 4, 6, 8};
  for (int g = 0; g < 2; ++g) {
    for (int bl : blocks) {
      lsyn_batch_tuning t = saved;
      t.blocks_per_sm = bl;
      t.use_graph = g;
      if (b->graph_exec) { cudaGraphExecDestroy(b->graph_exec); b->graph_exec = nullptr; }
      if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
      b->tune = t;
      const double t0 = now_ms();
      lsyn_status s = lsyn_batch_solve(b, max_size, res.data(), st.data());
      const double ms = now_ms() - t0;
      if (s != LSYN_OK) { b->tune = saved; return s; }
      if (ms < best_ms) { best_ms = ms; best = t; }
    }
  }
  if (b->graph_exec) { cudaGraphExecDestroy(b->graph_exec); b->graph_exec = nullptr; }
  if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
  b->tune = best;
  if (out) *out = best;
  return LSYN_OK;
}

}  // extern "C"
