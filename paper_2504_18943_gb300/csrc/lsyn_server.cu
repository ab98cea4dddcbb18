// Serving (lsyn_server_*, lsyn_submit, lsyn_poll, lsyn_wait): a host thread
// runs the scheduler's step loop (lsyn_engine.h) over the problems submitted so
// far. Submissions are validated and packed on the caller's thread, handed to
// the loop through an inbox and admitted between steps; answers are kept by
// ticket until polled.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>
#include <algorithm>

#include "lsyn.h"
#include "lsyn_engine.h"

using namespace lsyn;

struct lsyn_server {
  Engine eng;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::unique_ptr<Job>> inbox;
  std::unordered_map<uint64_t, std::unique_ptr<Job>> running;
  std::unordered_map<uint64_t, std::unique_ptr<Job>> finished;
  uint64_t next_ticket = 1;
  bool stop = false;
  lsyn_status fatal = LSYN_OK;
  std::string err;
  lsyn_sched_stats stats{};
  std::vector<lsyn_step_trace> trace;  // snapshot of the engine's trace, updated by the loop
  std::thread th;
  int device = 0;

  void loop();
};

namespace {
thread_local std::string g_server_error;

lsyn_status deliver(const Job& j, lsyn_result* out) {
  out->found = j.found;
  out->size = j.size;
  out->exact = j.exact;
  out->levels_done = j.levels_done;
  out->constructed = j.constructed;
  out->unique = j.unique;
  out->ms = j.t_done - j.t_submit;
  out->launches = 0;
  if (j.found) {
    if (!out->formula || out->formula_cap < j.formula.size() + 1) return LSYN_E_INVAL;
    memcpy(out->formula, j.formula.c_str(), j.formula.size() + 1);
  } else if (out->formula && out->formula_cap) {
    out->formula[0] = '\0';
  }
  return j.status;
}
}  // namespace

void lsyn_server::loop() {
  cudaSetDevice(device);
  int64_t last_steps = 0;
  while (true) {
    {
      std::unique_lock<std::mutex> lk(mu);
      cv_work.wait(lk, [&] { return stop || !inbox.empty() || eng.busy(); });
      if (stop) return;
      while (!inbox.empty()) {
        std::unique_ptr<Job> j = std::move(inbox.front());
        inbox.pop_front();
        eng.enqueue(j.get(), j->t_submit);
        running[j->ticket] = std::move(j);
      }
    }
    bool moved = false;
    lsyn_status s = eng.admit();
    if (s == LSYN_OK && eng.busy()) s = eng.pump(false, &moved);
    std::vector<Job*> done = eng.take_done();
    std::unique_lock<std::mutex> lk(mu);
    for (Job* j : done) {
      auto it = running.find(j->ticket);
      if (it == running.end()) continue;
      finished[j->ticket] = std::move(it->second);
      running.erase(it);
      ++stats.completed;
    }
    stats.active = eng.active_count();
    stats.queued = eng.queued_count() + int64_t(inbox.size());
    stats.steps = int64_t(eng.steps_run());
    stats.evictions = int64_t(eng.evictions());
    stats.redos = int64_t(eng.redos());
    stats.large_levels = int64_t(eng.large_levels());
    stats.pool_in_use = eng.pool().in_use();
    stats.pool_peak = eng.peak_in_use();
    if (stats.steps != last_steps) {
      trace = eng.trace();
      last_steps = stats.steps;
    }
    if (s != LSYN_OK) {
      fatal = s;
      err = eng.err;
      eng.clear();
      cv_done.notify_all();
      return;
    }
    if (!done.empty()) cv_done.notify_all();
    // Nothing moved. While a large level is on the GPU, poll it closely (a
    // timed wait sleeps for its duration plus the timer slack, and a heavy
    // problem passes here once per level); otherwise wait for a submission
    // or look again shortly.
    if (!moved && done.empty()) {
      if (eng.lanes_busy()) {
        lk.unlock();
        std::this_thread::yield();
      } else {
        cv_work.wait_for(lk, std::chrono::microseconds(100), [&] { return stop || !inbox.empty(); });
      }
    }
  }
}

extern "C" {

lsyn_status lsyn_server_create(const lsyn_config* config, const lsyn_batch_tuning* tuning, lsyn_server** out) {
  g_server_error.clear();
  if (!out) {
    g_server_error = "out is NULL";
    return LSYN_E_INVAL;
  }
  *out = nullptr;
  std::unique_ptr<lsyn_server> sv(new (std::nothrow) lsyn_server);
  if (!sv) return LSYN_E_NOMEM;
  const int max_active = tuning && tuning->max_active > 0 ? tuning->max_active : 256;
  lsyn_status s = sv->eng.init(config, tuning, max_active, false);
  if (s != LSYN_OK) {
    g_server_error = sv->eng.err;
    return s;
  }
  cudaGetDevice(&sv->device);
  sv->stats.pool_bytes = sv->eng.pool().budget();
  try {
    sv->th = std::thread([p = sv.get()] { p->loop(); });
  } catch (...) {
    g_server_error = "cannot start the server thread";
    return LSYN_E_NOMEM;
  }
  *out = sv.release();
  return LSYN_OK;
}

void lsyn_server_destroy(lsyn_server* sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv_work.notify_all();
  if (sv->th.joinable()) sv->th.join();
  cudaSetDevice(sv->device);
  sv->eng.clear();
  delete sv;
}

const char* lsyn_server_last_error(const lsyn_server* sv) { return sv ? sv->err.c_str() : g_server_error.c_str(); }

lsyn_status lsyn_submit(lsyn_server* sv, const lsyn_problem* problem, int32_t max_size, uint64_t* ticket) {
  if (!sv || !ticket) return LSYN_E_INVAL;
  if (max_size < 1 || max_size > 17) {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->err = "max_size must be in 1..17";
    return LSYN_E_INVAL;
  }
  const double t = now_ms();
  std::unique_ptr<Job> j(new (std::nothrow) Job);
  if (!j) return LSYN_E_NOMEM;
  lsyn_status s = sv->eng.make_job(problem, max_size, j.get());
  std::lock_guard<std::mutex> lk(sv->mu);
  if (s != LSYN_OK) {
    sv->err = j->err;
    return s;
  }
  if (sv->fatal != LSYN_OK || sv->stop) {
    sv->err = "the server stopped: " + sv->err;
    return LSYN_E_STATE;
  }
  j->t_submit = t;
  j->ticket = sv->next_ticket++;
  *ticket = j->ticket;
  sv->inbox.push_back(std::move(j));
  ++sv->stats.submitted;
  sv->cv_work.notify_one();
  return LSYN_OK;
}

lsyn_status lsyn_poll(lsyn_server* sv, uint64_t ticket, lsyn_result* out) {
  if (!sv || !out) return LSYN_E_INVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->finished.find(ticket);
  if (it != sv->finished.end()) {
    const lsyn_status s = deliver(*it->second, out);
    if (s == LSYN_E_INVAL && it->second->status != LSYN_E_INVAL) {
      sv->err = "formula buffer too small";
      return LSYN_E_INVAL;
    }
    sv->finished.erase(it);
    return s;
  }
  if (sv->running.count(ticket)) return sv->fatal != LSYN_OK ? sv->fatal : LSYN_PENDING;
  for (const auto& j : sv->inbox)
    if (j->ticket == ticket) return sv->fatal != LSYN_OK ? sv->fatal : LSYN_PENDING;
  return LSYN_E_INVAL;
}

lsyn_status lsyn_wait(lsyn_server* sv, uint64_t ticket, int32_t timeout_ms, lsyn_result* out) {
  if (!sv || !out) return LSYN_E_INVAL;
  {
    std::unique_lock<std::mutex> lk(sv->mu);
    auto ready = [&] { return sv->finished.count(ticket) || sv->fatal != LSYN_OK; };
    if (timeout_ms < 0) {
      sv->cv_done.wait(lk, ready);
    } else if (!sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
      return LSYN_E_TIMEOUT;
    }
  }
  return lsyn_poll(sv, ticket, out);
}

lsyn_status lsyn_server_trace(lsyn_server* sv, lsyn_step_trace* out, int32_t cap, int32_t* n_out) {
  if (!sv || !n_out || cap < 0 || (cap > 0 && !out)) return LSYN_E_INVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  const size_t n = std::min(sv->trace.size(), size_t(cap));
  for (size_t i = 0; i < n; ++i) out[i] = sv->trace[sv->trace.size() - n + i];
  *n_out = int32_t(n);
  return LSYN_OK;
}

lsyn_status lsyn_server_stats(lsyn_server* sv, lsyn_sched_stats* out) {
  if (!sv || !out) return LSYN_E_INVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  *out = sv->stats;
  return LSYN_OK;
}

}  // extern "C"
