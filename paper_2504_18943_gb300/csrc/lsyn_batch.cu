// Batched solving (lsyn_batch_*): every problem of the batch is a job of one
// scheduler (lsyn_engine.h) that admits all of them (or tuning->max_active at
// a time) and steps them together until each is answered.
#include <algorithm>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "lsyn.h"
#include "lsyn_engine.h"

using namespace lsyn;

struct lsyn_batch {
  Engine eng;
  std::vector<std::unique_ptr<Job>> jobs;
  std::vector<unsigned long long> caps;  // each job's entry limit
  std::string err;
};

namespace {
thread_local std::string g_batch_error;
}

extern "C" {

void lsyn_batch_destroy(lsyn_batch* b) {
  if (!b) return;
  b->eng.clear();
  delete b;
}

lsyn_status lsyn_batch_problem(lsyn_batch* b, int32_t i, lsyn_ctx** out) {
  if (!b || !out || i < 0 || i >= int32_t(b->jobs.size())) return LSYN_E_INVAL;
  *out = b->jobs[size_t(i)]->c;
  return LSYN_OK;
}

lsyn_status lsyn_batch_trace(const lsyn_batch* b, lsyn_step_trace* out, int32_t cap, int32_t* n_out) {
  if (!b || !n_out || cap < 0 || (cap > 0 && !out)) return LSYN_E_INVAL;
  const std::vector<lsyn_step_trace> t = b->eng.trace();
  const size_t n = std::min(t.size(), size_t(cap));
  for (size_t i = 0; i < n; ++i) out[i] = t[i];
  *n_out = int32_t(n);
  return LSYN_OK;
}

const char* lsyn_batch_last_error(const lsyn_batch* b) { return b ? b->err.c_str() : g_batch_error.c_str(); }

lsyn_status lsyn_batch_stats(const lsyn_batch* b, lsyn_sched_stats* out) {
  if (!b || !out) return LSYN_E_INVAL;
  memset(out, 0, sizeof(*out));
  int64_t done = 0;
  for (const auto& j : b->jobs) done += j->state == Job::kDone ? 1 : 0;
  out->submitted = int64_t(b->jobs.size());
  out->completed = done;
  out->active = b->eng.active_count();
  out->queued = b->eng.queued_count();
  out->steps = int64_t(b->eng.steps_run());
  out->evictions = int64_t(b->eng.evictions());
  out->redos = int64_t(b->eng.redos());
  out->large_levels = int64_t(b->eng.large_levels());
  out->pool_bytes = b->eng.pool().budget();
  out->pool_in_use = b->eng.pool().in_use();
  out->pool_peak = b->eng.peak_in_use();
  return LSYN_OK;
}

lsyn_status lsyn_batch_create(const lsyn_problem* problems, int32_t n, const lsyn_config* config,
                              const lsyn_batch_tuning* tuning, lsyn_batch** out) {
  g_batch_error.clear();
  if (!out || !problems || n < 1) {
    g_batch_error = "problems, n >= 1 and out are required";
    return LSYN_E_INVAL;
  }
  *out = nullptr;
  std::unique_ptr<lsyn_batch> b(new (std::nothrow) lsyn_batch);
  if (!b) return LSYN_E_NOMEM;
  const int max_active = tuning && tuning->max_active > 0 ? std::min(n, tuning->max_active) : n;
  lsyn_status s = b->eng.init(config, tuning, max_active, true);
  if (s != LSYN_OK) {
    g_batch_error = b->eng.err;
    return s;
  }
  b->jobs.reserve(size_t(n));
  for (int i = 0; i < n; ++i) {
    b->jobs.emplace_back(new (std::nothrow) Job);
    if (!b->jobs.back()) return LSYN_E_NOMEM;
    s = b->eng.make_job(&problems[i], 17, b->jobs.back().get());
    if (s != LSYN_OK) {
      g_batch_error = "problem " + std::to_string(i) + ": " + b->jobs.back()->err;
      return s;
    }
    b->caps.push_back(b->jobs.back()->cap_entries);
  }
  *out = b.release();
  return LSYN_OK;
}

lsyn_status lsyn_batch_solve(lsyn_batch* b, int32_t max_size, lsyn_result* results, int32_t* statuses) {
  if (!b || !results || !statuses) return LSYN_E_INVAL;
  if (max_size < 1 || max_size > 17) {
    b->err = "max_size must be in 1..17 for a batch";
    return LSYN_E_INVAL;
  }
  b->err.clear();
  b->eng.clear();  // drop the caches of an earlier solve
  b->eng.clear_trace();
  const double t0 = now_ms();
  const uint64_t steps0 = b->eng.steps_run();
  for (size_t i = 0; i < b->jobs.size(); ++i) {
    Job* j = b->jobs[i].get();
    j->max_size = max_size;
    j->cap_entries = b->caps[i];
    j->found = j->size = j->exact = j->levels_done = 0;
    j->constructed = j->unique = 0;
    j->formula.clear();
    j->err.clear();
    j->redo = false;
    j->capped = false;
    j->evictions = j->redos = 0;
    b->eng.enqueue(j, t0);
  }
  while (b->eng.busy()) {
    bool moved = false;
    lsyn_status s = b->eng.admit();
    if (s == LSYN_OK) s = b->eng.pump(true, &moved);
    if (s != LSYN_OK) {
      b->err = b->eng.err;
      b->eng.clear();
      return s;
    }
  }
  b->eng.take_done();
  lsyn_status ret = LSYN_OK;
  for (size_t i = 0; i < b->jobs.size(); ++i) {
    const Job* j = b->jobs[i].get();
    lsyn_result& r = results[i];
    statuses[i] = j->status;
    r.found = j->found;
    r.size = j->size;
    r.exact = j->exact;
    r.levels_done = j->levels_done;
    r.constructed = j->constructed;
    r.unique = j->unique;
    r.ms = j->t_done - t0;
    r.launches = int32_t(b->eng.steps_run() - steps0);
    if (j->found) {
      if (!r.formula || r.formula_cap < j->formula.size() + 1) {
        b->err = "formula buffer of problem " + std::to_string(i) + " too small";
        ret = LSYN_E_INVAL;
      } else {
        memcpy(r.formula, j->formula.c_str(), j->formula.size() + 1);
      }
    } else if (r.formula && r.formula_cap) {
      r.formula[0] = '\0';
    }
  }
  return ret;
}

lsyn_status lsyn_batch_autotune(lsyn_batch* b, int32_t max_size, lsyn_batch_tuning* out) {
  if (!b) return LSYN_E_INVAL;
  const size_t n = b->jobs.size();
  std::vector<lsyn_result> res(n);
  std::vector<int32_t> st(n);
  std::vector<std::vector<char>> fbuf(n, std::vector<char>(lsyn_ctx::kFormulaCap));
  for (size_t i = 0; i < n; ++i) {
    memset(&res[i], 0, sizeof(lsyn_result));
    res[i].formula = fbuf[i].data();
    res[i].formula_cap = fbuf[i].size();
  }
  // the defaults written out, so that the result names every value it chose
  lsyn_batch_tuning saved = b->eng.tune();
  if (!saved.rows_per_item) saved.rows_per_item = 8;
  if (!saved.words_per_thread) saved.words_per_thread = 1;
  if (!saved.table_load_pct)
    saved.table_load_pct = std::max(25, std::min(90, int32_t(b->jobs.empty() ? 50 : b->jobs[0]->c->table_load * 100.0 + 0.5)));
  auto time_it = [&](const lsyn_batch_tuning& t, double* ms) {
    b->eng.set_tune(t);
    const double t0 = now_ms();
    lsyn_status s = lsyn_batch_solve(b, max_size, res.data(), st.data());
    *ms = now_ms() - t0;
    return s;
  };
  // one untimed solve warms the pool and the launch paths
  double ms = 0;
  lsyn_status s = time_it(saved, &ms);
  if (s != LSYN_OK) return s;
  lsyn_batch_tuning best = saved;
  double best_ms = 1e300;
  if ((s = time_it(best, &best_ms)) != LSYN_OK) return s;
  const int sms = b->eng.sm_count();  // of the batch's device
  // Coordinate descent: one parameter at a time, keep the fastest value. The
  // first three axes are the kernel's shape: formulas per warp (rows / pairs
  // per work item), words per thread (vectors a lane loads together on CMs
  // above 128 bytes) and table sizing (the load up to which tables fill);
  // then the launch: blocks per SM, graph replay, the large-level threshold
  // and the SMs kept for batch steps.
  const int32_t rows[3] = {2, 4, 8};
  const int32_t wpt[2] = {1, 2};
  const int32_t load_pct[3] = {25, 50, 75};
  const int32_t blocks[3] = {2, 4, 8};
  const uint64_t solo[3] = {1ull << 17, 1ull << 19, 1ull << 21};
  const int32_t light[3] = {std::max(1, sms / 16), std::max(1, sms / 8), std::max(1, sms / 4)};
  for (int axis = 0; axis < 7; ++axis) {
    std::vector<lsyn_batch_tuning> cand;
    for (int v = 0; v < 3; ++v) {
      lsyn_batch_tuning t = best;
      switch (axis) {
        case 0: t.rows_per_item = rows[v]; break;
        case 1:
          if (v == 2) continue;
          t.words_per_thread = wpt[v];
          break;
        case 2: t.table_load_pct = load_pct[v]; break;
        case 3: t.blocks_per_sm = blocks[v]; break;
        case 4:
          if (v == 2) continue;
          t.use_graph = v;
          break;
        case 5: t.solo_candidates = solo[v]; break;
        default: t.light_sms = light[v]; break;
      }
      cand.push_back(t);
    }
    for (const lsyn_batch_tuning& t : cand) {
      if ((s = time_it(t, &ms)) != LSYN_OK) {
        b->eng.set_tune(saved);
        return s;
      }
      if (ms < best_ms) {
        best_ms = ms;
        best = b->eng.tune();
      }
    }
  }
  b->eng.set_tune(best);
  if (out) *out = b->eng.tune();
  return LSYN_OK;
}

}  // extern "C"
