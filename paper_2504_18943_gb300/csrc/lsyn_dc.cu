// Divide-and-conquer (paragraph "Divide-and-conquer"): split a specification
// that cannot be solved in one go into (P_i, N_j), solve the parts
// recursively, recombine (phi_11 & phi_12) | (phi_21 & phi_22).
//
// The recursion runs breadth first: all parts pending at one depth form one
// batch of the scheduler (lsyn_engine.h), so the parts of a split are solved
// side by side on the GPU; a part without an answer is split for the next
// round. A part is "small enough to be solved in one go" when the scheduler
// answers it (a separating formula of size <= max_size within its cache).
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "lsyn.h"
#include "lsyn_engine.h"

using namespace lsyn;

namespace {

thread_local std::string g_dc_error;

enum Kind { kPending = 0, kLeaf = 1, kBoth = 2, kPosOnly = 3, kNegOnly = 4 };

struct Part {
  std::vector<int> pos, neg;  // trace indices of the whole specification
  int depth = 0;
  int kind = kPending;
  int child[4] = {-1, -1, -1, -1};
  std::string formula;
  int64_t size = 0;
};

// The halves of an index list: the first ceil(n / 2), then the rest.
void halves(const std::vector<int>& v, std::vector<int>* a, std::vector<int>* b) {
  const size_t h = (v.size() + 1) / 2;
  a->assign(v.begin(), v.begin() + long(h));
  b->assign(v.begin() + long(h), v.end());
}

// Formula text and size of part i from its children (post-order).
void compose(std::vector<Part>& parts, int i) {
  Part& p = parts[size_t(i)];
  if (p.kind == kLeaf) return;
  for (int c : p.child)
    if (c >= 0) compose(parts, c);
  auto f = [&](int k) -> const Part& { return parts[size_t(p.child[k])]; };
  if (p.kind == kBoth) {
    p.formula = "(| (& " + f(0).formula + " " + f(1).formula + ") (& " + f(2).formula + " " + f(3).formula + "))";
    p.size = 3 + f(0).size + f(1).size + f(2).size + f(3).size;
  } else if (p.kind == kPosOnly) {
    p.formula = "(| " + f(0).formula + " " + f(1).formula + ")";
    p.size = 1 + f(0).size + f(1).size;
  } else {
    p.formula = "(& " + f(0).formula + " " + f(1).formula + ")";
    p.size = 1 + f(0).size + f(1).size;
  }
}

}  // namespace

extern "C" lsyn_status lsyn_dc_solve(const lsyn_problem* problem, int32_t max_size, const lsyn_config* config,
                                     const lsyn_batch_tuning* tuning, lsyn_result* out, lsyn_dc_stats* stats) {
  g_dc_error.clear();
  if (!problem || !out) return LSYN_E_INVAL;
  if (max_size < 1 || max_size > 17) return LSYN_E_INVAL;
  lsyn_dc_stats st_local;
  lsyn_dc_stats& st = stats ? *stats : st_local;
  memset(&st, 0, sizeof(st));
  const double t0 = now_ms();
  // validate the whole specification once (the parts are subsets of it)
  {
    lsyn_ctx* c = nullptr;
    lsyn_status s = ctx_shell(problem, config, false, &c, nullptr, nullptr);
    if (s != LSYN_OK) {
      g_dc_error = thread_error();
      return s;
    }
    delete c;
  }
  const int T = problem->n_pos + problem->n_neg;
  const size_t wbytes = size_t(problem->word_bits / 8);
  const uint8_t* words = static_cast<const uint8_t*>(problem->atom_words);

  std::unique_ptr<Engine> eng(new (std::nothrow) Engine);
  if (!eng) return LSYN_E_NOMEM;
  lsyn_status s = eng->init(config, tuning, 256, false);
  if (s != LSYN_OK) {
    g_dc_error = eng->err;
    return s;
  }

  std::vector<Part> parts(1);
  for (int i = 0; i < problem->n_pos; ++i) parts[0].pos.push_back(i);
  for (int i = problem->n_pos; i < T; ++i) parts[0].neg.push_back(i);
  std::vector<int> round = {0};
  int64_t constructed = 0, unique = 0;
  while (!round.empty()) {
    ++st.rounds;
    // one sub-problem per pending part: its traces (positives first) copied out
    std::vector<std::unique_ptr<Job>> jobs;
    for (int pi : round) {
      const Part& p = parts[size_t(pi)];
      std::vector<int> idx(p.pos);
      idx.insert(idx.end(), p.neg.begin(), p.neg.end());
      const size_t n = idx.size();
      std::vector<int32_t> lens(n);
      std::vector<uint8_t> w(size_t(problem->n_props) * n * wbytes);
      for (size_t t = 0; t < n; ++t) {
        lens[t] = problem->lengths[idx[t]];
        for (int q = 0; q < problem->n_props; ++q)
          memcpy(&w[(size_t(q) * n + t) * wbytes], &words[(size_t(q) * size_t(T) + size_t(idx[t])) * wbytes], wbytes);
      }
      lsyn_problem sp = *problem;
      sp.n_pos = int(p.pos.size());
      sp.n_neg = int(p.neg.size());
      sp.lengths = lens.data();
      sp.atom_words = w.data();
      jobs.emplace_back(new (std::nothrow) Job);
      if (!jobs.back()) return LSYN_E_NOMEM;
      if ((s = eng->make_job(&sp, max_size, jobs.back().get())) != LSYN_OK) {
        g_dc_error = jobs.back()->err;
        return s;
      }
      eng->enqueue(jobs.back().get(), now_ms());
    }
    st.parts += int64_t(jobs.size());
    while (eng->busy()) {
      bool moved = false;
      if ((s = eng->admit()) == LSYN_OK) s = eng->pump(true, &moved);
      if (s != LSYN_OK) {
        g_dc_error = eng->err;
        eng->clear();
        return s;
      }
    }
    eng->take_done();
    std::vector<int> next;
    for (size_t r = 0; r < round.size(); ++r) {
      const int pi = round[r];
      const Job& j = *jobs[r];
      constructed += j.constructed;
      unique += j.unique;
      if (j.status == LSYN_OK) {
        Part& p = parts[size_t(pi)];
        p.kind = kLeaf;
        p.formula = j.formula;
        p.size = j.size;
        ++st.leaves;
        continue;
      }
      if (j.status != LSYN_NOT_FOUND && j.status != LSYN_E_CACHE_FULL) {
        g_dc_error = j.err;
        return j.status;
      }
      // not solvable in one go: split (the parts are appended, so re-fetch p)
      const std::vector<int> pos = parts[size_t(pi)].pos, neg = parts[size_t(pi)].neg;
      const int depth = parts[size_t(pi)].depth + 1;
      std::vector<int> p1, p2, n1, n2;
      halves(pos, &p1, &p2);
      halves(neg, &n1, &n2);
      int kind;
      std::vector<std::pair<const std::vector<int>*, const std::vector<int>*>> kids;
      if (pos.size() >= 2 && neg.size() >= 2) {
        kind = kBoth;  // phi_11, phi_12, phi_21, phi_22
        kids = {{&p1, &n1}, {&p1, &n2}, {&p2, &n1}, {&p2, &n2}};
      } else if (pos.size() >= 2) {
        kind = kPosOnly;
        kids = {{&p1, &neg}, {&p2, &neg}};
      } else if (neg.size() >= 2) {
        kind = kNegOnly;
        kids = {{&pos, &n1}, {&pos, &n2}};
      } else {
        out->found = 0;
        out->size = 0;
        out->exact = 0;
        out->constructed = constructed;
        out->unique = unique;
        out->ms = now_ms() - t0;
        if (out->formula && out->formula_cap) out->formula[0] = '\0';
        g_dc_error = "a part of one positive and one negative trace has no separating formula up to max_size";
        return LSYN_NOT_FOUND;
      }
      parts[size_t(pi)].kind = kind;
      ++st.splits;
      for (size_t k = 0; k < kids.size(); ++k) {
        Part c;
        c.pos = *kids[k].first;
        c.neg = *kids[k].second;
        c.depth = depth;
        parts.push_back(c);
        parts[size_t(pi)].child[k] = int(parts.size()) - 1;
        next.push_back(int(parts.size()) - 1);
        if (depth > st.depth) st.depth = depth;
      }
    }
    round.swap(next);
  }
  compose(parts, 0);
  const Part& root = parts[0];
  st.formula_len = int64_t(root.formula.size());
  out->found = 1;
  out->size = int32_t(root.size);
  out->exact = root.kind == kLeaf ? 1 : 0;
  out->levels_done = root.kind == kLeaf ? int32_t(root.size) : 0;
  out->constructed = constructed;
  out->unique = unique;
  out->ms = now_ms() - t0;
  out->launches = int32_t(eng->steps_run() + eng->large_levels());
  if (!out->formula || out->formula_cap < root.formula.size() + 1) {
    g_dc_error = "formula buffer too small (" + std::to_string(root.formula.size() + 1) + " bytes needed)";
    return LSYN_E_INVAL;
  }
  memcpy(out->formula, root.formula.c_str(), root.formula.size() + 1);
  return LSYN_OK;
}

extern "C" const char* lsyn_dc_last_error(void) { return g_dc_error.c_str(); }
