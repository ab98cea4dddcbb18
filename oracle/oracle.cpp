// Plain CPU oracle for bottom-up semantic enumeration of LTLf formulae.
//
// TEST INFRASTRUCTURE ONLY. Only the test-suite, the smoke check and the
// benchmark's CPU-baseline leg may build, load or call this file. The product
// path (the CUDA library and its binding) never does, and shares no code,
// header, table or helper with it.
//
// What it computes, and where the paper defines it ("GPU accelerated program
// synthesis: Enumerate semantics, not syntax!", arXiv 2504.18943):
//
//  * Formulae: the grammar of the section "Synthesising linear temporal logic
//    formulae from examples" (atoms, not, and, X, F, U), plus "or" (used by the
//    paper in its F argument and in "Divide-and-conquer") and G, read as
//    "not F not".
//  * Satisfaction tr, i |= phi over finite traces: same section. Positions at
//    or beyond the trace length never satisfy anything (section "Parallel
//    enumeration of LTLf formulae on GPUs", the argument for F).
//  * Characteristic sequence / matrix: same "Parallel enumeration" section.
//    Here a characteristic sequence is a string of '0'/'1' characters, one
//    per position of the trace; a characteristic matrix is the sequences of
//    all traces, in the fixed order (positives first), joined with ','.
//  * Observational equivalence: two formulae are the same search-space element
//    iff their characteristic matrices are equal ("Parallel enumeration").
//  * Bottom-up enumeration with a language cache: the listing of the paragraph
//    "A generic program synthesiser" (section "Program synthesis"). For every
//    operator, every split of size-1 into child sizes, every left and every
//    right program from the cache, build the candidate, return it if it
//    separates the specification, otherwise add it to the cache of its size
//    unless an equal characteristic matrix is already cached.
//  * Separation: phi separates (P, N) iff tr, 0 |= phi for every tr in P and
//    not for every tr in N ("Synthesising ... from examples").
//  * Size: the number of syntax-tree nodes; "not (b U a)" has size 4.
//
// Everything is done with strings, std::set and plain loops, position by
// position, exactly as the definitions read. There are no bit tricks, no
// log-step scans, no hashing and no parallelism.
//
// Operator mask bits (an interface shared with the tests): 0 not, 1 and,
// 2 or, 3 X, 4 F, 5 G, 6 U.

#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <set>
#include <string>
#include <thread>
#include <vector>

namespace {

enum Op { ATOM = 0, NOT, AND, OR, NEXT, FUTURE, GLOBALLY, UNTIL };
const int kMaskBit[8] = {-1, 0, 1, 2, 3, 4, 5, 6};
const char* kOpText[8] = {"p", "!", "&", "|", "X", "F", "G", "U"};

bool is_binary(int op) { return op == AND || op == OR || op == UNTIL; }
bool enabled(unsigned mask, int op) { return op == ATOM || ((mask >> kMaskBit[op]) & 1u); }

// A trace: holds[t][p] says that proposition p is in the letter at position t.
struct Trace {
  std::vector<std::vector<bool>> holds;
  int length() const { return (int)holds.size(); }
};

struct Spec {
  int n_props = 0;
  int n_pos = 0;
  std::vector<Trace> traces;  // positives first, then negatives
};

// ---------------------------------------------------------------------------
// Syntax trees and the text format "(op child ...)" / "pK"
// ---------------------------------------------------------------------------

struct Node {
  int op;
  int prop;   // for ATOM
  int a, b;   // child node indices (-1 if absent)
};

struct Tree {
  std::vector<Node> nodes;
  int root = -1;
};

struct Parser {
  const char* s;
  size_t i = 0;
  Tree* t;
  bool ok = true;
  void skip() { while (s[i] == ' ' || s[i] == '\t' || s[i] == '\n') ++i; }
  int add(Node n) { t->nodes.push_back(n); return (int)t->nodes.size() - 1; }
  int parse() {
    skip();
    if (s[i] == 'p') {
      ++i;
      if (s[i] < '0' || s[i] > '9') { ok = false; return -1; }
      int v = 0;
      while (s[i] >= '0' && s[i] <= '9') { v = v * 10 + (s[i] - '0'); ++i; }
      return add({ATOM, v, -1, -1});
    }
    if (s[i] != '(') { ok = false; return -1; }
    ++i;
    skip();
    int op = -1;
    for (int k = 1; k < 8; ++k)
      if (s[i] == kOpText[k][0]) op = k;
    if (op < 0) { ok = false; return -1; }
    ++i;
    int a = parse();
    if (!ok) return -1;
    int b = -1;
    if (is_binary(op)) { b = parse(); if (!ok) return -1; }
    skip();
    if (s[i] != ')') { ok = false; return -1; }
    ++i;
    return add({op, 0, a, b});
  }
};

bool parse_formula(const char* text, Tree* out) {
  Parser p{text, 0, out, true};
  out->nodes.clear();
  out->root = p.parse();
  if (!p.ok) return false;
  p.skip();
  return text[p.i] == '\0';
}

void print_tree(const Tree& t, int n, std::string* out) {
  const Node& x = t.nodes[n];
  if (x.op == ATOM) { *out += "p" + std::to_string(x.prop); return; }
  *out += "(";
  *out += kOpText[x.op];
  *out += " ";
  print_tree(t, x.a, out);
  if (x.b >= 0) { *out += " "; print_tree(t, x.b, out); }
  *out += ")";
}

// ---------------------------------------------------------------------------
// Satisfaction by the definition, recursively on the tree: tr, i |= phi.
// ---------------------------------------------------------------------------

bool sat(const Tree& t, int n, const Trace& tr, int i) {
  const int len = tr.length();
  if (i >= len) return false;  // nothing holds beyond the end of a finite trace
  const Node& x = t.nodes[n];
  switch (x.op) {
    case ATOM: return x.prop < (int)tr.holds[i].size() && tr.holds[i][x.prop];
    case NOT: return !sat(t, x.a, tr, i);
    case AND: return sat(t, x.a, tr, i) && sat(t, x.b, tr, i);
    case OR: return sat(t, x.a, tr, i) || sat(t, x.b, tr, i);
    case NEXT: return i + 1 < len && sat(t, x.a, tr, i + 1);
    case FUTURE:
      for (int j = i; j < len; ++j)
        if (sat(t, x.a, tr, j)) return true;
      return false;
    case GLOBALLY:
      for (int j = i; j < len; ++j)
        if (!sat(t, x.a, tr, j)) return false;
      return true;
    case UNTIL:
      for (int j = i; j < len; ++j) {
        if (!sat(t, x.b, tr, j)) continue;
        bool left_all = true;
        for (int k = i; k < j; ++k)
          if (!sat(t, x.a, tr, k)) { left_all = false; break; }
        if (left_all) return true;
      }
      return false;
  }
  return false;
}

// Characteristic matrix of a tree, by the recursive definition.
std::string cm_by_tree(const Spec& s, const Tree& t) {
  std::string out;
  for (size_t k = 0; k < s.traces.size(); ++k) {
    if (k) out += ',';
    const Trace& tr = s.traces[k];
    for (int i = 0; i < tr.length(); ++i) out += sat(t, t.root, tr, i) ? '1' : '0';
  }
  return out;
}

// ---------------------------------------------------------------------------
// The same operators on characteristic sequences (strings), used by the
// bottom-up enumerator: the value of op(children) depends only on the
// children's characteristic sequences, position by position.
// ---------------------------------------------------------------------------

using CM = std::vector<std::string>;  // one characteristic sequence per trace

std::string seq_atom(const Trace& tr, int p) {
  std::string r(tr.length(), '0');
  for (int i = 0; i < tr.length(); ++i) r[i] = tr.holds[i][p] ? '1' : '0';
  return r;
}

std::string seq_unary(int op, const std::string& a) {
  const int n = (int)a.size();
  std::string r(n, '0');
  for (int i = 0; i < n; ++i) {
    bool v = false;
    if (op == NOT) v = a[i] != '1';
    if (op == NEXT) v = i + 1 < n && a[i + 1] == '1';
    if (op == FUTURE) {
      v = false;
      for (int j = i; j < n; ++j) if (a[j] == '1') v = true;
    }
    if (op == GLOBALLY) {
      v = true;
      for (int j = i; j < n; ++j) if (a[j] != '1') v = false;
    }
    r[i] = v ? '1' : '0';
  }
  return r;
}

std::string seq_binary(int op, const std::string& a, const std::string& b) {
  const int n = (int)a.size();
  std::string r(n, '0');
  for (int i = 0; i < n; ++i) {
    bool v = false;
    if (op == AND) v = a[i] == '1' && b[i] == '1';
    if (op == OR) v = a[i] == '1' || b[i] == '1';
    if (op == UNTIL) {
      for (int j = i; j < n && !v; ++j) {
        if (b[j] != '1') continue;
        bool left_all = true;
        for (int k = i; k < j; ++k) if (a[k] != '1') left_all = false;
        if (left_all) v = true;
      }
    }
    r[i] = v ? '1' : '0';
  }
  return r;
}

std::string join(const CM& cm) {
  std::string out;
  for (size_t k = 0; k < cm.size(); ++k) {
    if (k) out += ',';
    out += cm[k];
  }
  return out;
}

bool separates(const Spec& s, const CM& cm) {
  for (size_t k = 0; k < s.traces.size(); ++k) {
    const bool at0 = !cm[k].empty() && cm[k][0] == '1';
    const bool positive = (int)k < s.n_pos;
    if (at0 != positive) return false;
  }
  return true;
}

bool separates_joined(const Spec& s, const std::string& joined) {
  CM cm;
  std::string cur;
  for (char c : joined) {
    if (c == ',') { cm.push_back(cur); cur.clear(); } else cur += c;
  }
  cm.push_back(cur);
  return cm.size() == s.traces.size() && separates(s, cm);
}

// ---------------------------------------------------------------------------
// Bottom-up enumeration with a language cache (the generic listing), and a
// brute-force enumeration of all syntax trees for cross-checking it.
// ---------------------------------------------------------------------------

struct Entry {
  CM cm;
  int op;
  int prop;           // atoms
  int la, ia, lb, ib; // children as (level, index); -1 when absent
};

struct Run {
  std::vector<std::vector<Entry>> levels;   // levels[k] for k >= 1; levels[0] unused
  std::vector<int64_t> candidates;          // candidates built per level
  std::vector<std::vector<std::string>> sorted;  // joined CMs per level, sorted (filled lazily)
  std::vector<std::string> bf_formula;      // brute force: per joined CM, one tree text
  bool brute = false;
  std::map<std::string, std::string> bf_text;
  std::vector<std::vector<std::string>> bf_levels;
  // solve result
  int solved_size = 0;
  std::string solved_formula;
  int64_t constructed = 0;
};

void formula_of(const Run& r, int level, int idx, std::string* out) {
  const Entry& e = r.levels[level][idx];
  if (e.op == ATOM) { *out += "p" + std::to_string(e.prop); return; }
  *out += "(";
  *out += kOpText[e.op];
  *out += " ";
  formula_of(r, e.la, e.ia, out);
  if (e.lb > 0) { *out += " "; formula_of(r, e.lb, e.ib, out); }
  *out += ")";
}

// The level loop. When `stop_at_solution` is set, return as soon as a
// candidate separates the specification (the early return of the listing);
// otherwise every level up to max_level is built completely.
void enumerate(const Spec& s, int max_level, unsigned mask, bool stop_at_solution, Run* r) {
  r->levels.assign(2, {});
  r->candidates.assign(2, 0);
  std::set<std::string> cache;  // every characteristic matrix seen so far, all sizes

  auto consider = [&](int level, Entry&& e) -> bool {
    r->candidates[level] += 1;
    r->constructed += 1;
    const bool sep = separates(s, e.cm);
    std::string key = join(e.cm);
    const bool is_new = cache.insert(key).second;
    if (is_new) r->levels[level].push_back(std::move(e));
    if (sep && stop_at_solution) {
      r->solved_size = level;
      if (is_new) {
        formula_of(*r, level, (int)r->levels[level].size() - 1, &r->solved_formula);
      }
      return true;
    }
    return false;
  };

  // Level 1: the atomic predicates.
  for (int p = 0; p < s.n_props; ++p) {
    Entry e;
    e.op = ATOM; e.prop = p; e.la = e.ia = e.lb = e.ib = -1;
    for (const Trace& tr : s.traces) e.cm.push_back(seq_atom(tr, p));
    if (consider(1, std::move(e))) return;
  }

  const int kOps[7] = {NOT, AND, OR, NEXT, FUTURE, GLOBALLY, UNTIL};
  for (int size = 2; size <= max_level; ++size) {
    r->levels.emplace_back();
    r->candidates.push_back(0);
    for (int op : kOps) {
      if (!enabled(mask, op)) continue;
      if (!is_binary(op)) {
        const int i = size - 1;
        for (int x = 0; x < (int)r->levels[i].size(); ++x) {
          Entry e;
          e.op = op; e.prop = 0; e.la = i; e.ia = x; e.lb = -1; e.ib = -1;
          for (const std::string& seq : r->levels[i][x].cm) e.cm.push_back(seq_unary(op, seq));
          if (consider(size, std::move(e))) return;
        }
        continue;
      }
      for (int i = 1; i <= size - 2; ++i) {
        const int j = size - 1 - i;
        for (int x = 0; x < (int)r->levels[i].size(); ++x) {
          for (int y = 0; y < (int)r->levels[j].size(); ++y) {
            const CM& a = r->levels[i][x].cm;
            const CM& b = r->levels[j][y].cm;
            Entry e;
            e.op = op; e.prop = 0; e.la = i; e.ia = x; e.lb = j; e.ib = y;
            for (size_t k = 0; k < a.size(); ++k) e.cm.push_back(seq_binary(op, a[k], b[k]));
            if (consider(size, std::move(e))) return;
          }
        }
      }
    }
  }
}

// The levels of enumerate() without the early return, with each level's
// candidates shared out among `threads` host threads (the CPU baseline on all
// cores). The candidates are the listing's: every operator, every split,
// every left and right program; item n of a level (an operator, the left
// program's size and index) goes to thread n mod threads. Each thread keeps the
// new characteristic matrices it meets in a set of its own, the cache of the
// levels below is only read meanwhile, and once every thread is done the sets
// are merged in thread order. A level is therefore the same set as in
// enumerate(); only the order of its entries, and so which of several formulas
// with one characteristic matrix is kept, may differ.
void enumerate_threads(const Spec& s, int max_level, unsigned mask, int threads, Run* r) {
  if (threads < 1) threads = 1;
  r->levels.assign(2, {});
  r->candidates.assign(2, 0);
  std::set<std::string> cache;
  for (int p = 0; p < s.n_props; ++p) {
    Entry e;
    e.op = ATOM; e.prop = p; e.la = e.ia = e.lb = e.ib = -1;
    for (const Trace& tr : s.traces) e.cm.push_back(seq_atom(tr, p));
    r->candidates[1] += 1;
    r->constructed += 1;
    if (cache.insert(join(e.cm)).second) r->levels[1].push_back(std::move(e));
  }
  const int kOps[7] = {NOT, AND, OR, NEXT, FUTURE, GLOBALLY, UNTIL};
  struct Item { int op, i, x; };
  for (int size = 2; size <= max_level; ++size) {
    r->levels.emplace_back();
    r->candidates.push_back(0);
    std::vector<Item> items;
    for (int op : kOps) {
      if (!enabled(mask, op)) continue;
      if (!is_binary(op)) {
        for (int x = 0; x < (int)r->levels[size - 1].size(); ++x) items.push_back({op, size - 1, x});
        continue;
      }
      for (int i = 1; i <= size - 2; ++i)
        for (int x = 0; x < (int)r->levels[i].size(); ++x) items.push_back({op, i, x});
    }
    std::vector<std::map<std::string, Entry>> found(threads);
    std::vector<int64_t> built(threads, 0);
    auto work = [&](int t) {
      for (size_t n = t; n < items.size(); n += threads) {
        const Item& it = items[n];
        const CM& a = r->levels[it.i][it.x].cm;
        auto consider = [&](Entry&& e) {
          built[t] += 1;
          std::string key = join(e.cm);
          if (!cache.count(key)) found[t].emplace(std::move(key), std::move(e));  // the first one found stays
        };
        if (!is_binary(it.op)) {
          Entry e;
          e.op = it.op; e.prop = 0; e.la = it.i; e.ia = it.x; e.lb = -1; e.ib = -1;
          for (const std::string& seq : a) e.cm.push_back(seq_unary(it.op, seq));
          consider(std::move(e));
          continue;
        }
        const int j = size - 1 - it.i;
        for (int y = 0; y < (int)r->levels[j].size(); ++y) {
          const CM& b = r->levels[j][y].cm;
          Entry e;
          e.op = it.op; e.prop = 0; e.la = it.i; e.ia = it.x; e.lb = j; e.ib = y;
          for (size_t k = 0; k < a.size(); ++k) e.cm.push_back(seq_binary(it.op, a[k], b[k]));
          consider(std::move(e));
        }
      }
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < threads; ++t) pool.emplace_back(work, t);
    work(0);
    for (std::thread& th : pool) th.join();
    for (int t = 0; t < threads; ++t) {
      r->candidates[size] += built[t];
      r->constructed += built[t];
      for (auto& kv : found[t])
        if (cache.insert(kv.first).second) r->levels[size].push_back(std::move(kv.second));
    }
  }
}

// All syntax trees of an exact size, as texts (no deduplication of any kind).
void trees_of_size(int size, int n_props, unsigned mask, std::vector<std::vector<std::string>>* memo) {
  if ((int)memo->size() > size && !(*memo)[size].empty()) return;
  if ((int)memo->size() <= size) memo->resize(size + 1);
  std::vector<std::string> out;
  if (size == 1) {
    for (int p = 0; p < n_props; ++p) out.push_back("p" + std::to_string(p));
  } else {
    for (int op = NOT; op <= UNTIL; ++op) {
      if (!enabled(mask, op)) continue;
      if (!is_binary(op)) {
        trees_of_size(size - 1, n_props, mask, memo);
        for (const std::string& c : (*memo)[size - 1])
          out.push_back(std::string("(") + kOpText[op] + " " + c + ")");
      } else {
        for (int i = 1; i <= size - 2; ++i) {
          const int j = size - 1 - i;
          trees_of_size(i, n_props, mask, memo);
          trees_of_size(j, n_props, mask, memo);
          for (const std::string& a : (*memo)[i])
            for (const std::string& b : (*memo)[j])
              out.push_back(std::string("(") + kOpText[op] + " " + a + " " + b + ")");
        }
      }
    }
  }
  (*memo)[size] = std::move(out);
}

// Brute force: evaluate every tree of size <= max_size recursively, and keep,
// per size k, the characteristic matrices of size-k trees that no smaller tree
// has. By congruence these sets must equal the enumerator's levels.
void brute_force(const Spec& s, int max_size, unsigned mask, Run* r) {
  r->brute = true;
  r->bf_levels.assign(max_size + 1, {});
  r->candidates.assign(max_size + 1, 0);
  std::vector<std::vector<std::string>> memo;
  std::set<std::string> seen;
  for (int size = 1; size <= max_size; ++size) {
    trees_of_size(size, s.n_props, mask, &memo);
    std::set<std::string> level;
    for (const std::string& text : memo[size]) {
      Tree t;
      parse_formula(text.c_str(), &t);
      std::string cm = cm_by_tree(s, t);
      r->candidates[size] += 1;
      if (seen.count(cm)) continue;
      if (level.insert(cm).second) r->bf_text[cm] = text;
    }
    for (const std::string& cm : level) seen.insert(cm);
    r->bf_levels[size].assign(level.begin(), level.end());
  }
}

int copy_out(const std::string& v, char* buf, size_t cap) {
  if (v.size() + 1 > cap) return -2;
  std::memcpy(buf, v.c_str(), v.size() + 1);
  return (int)v.size();
}

}  // namespace

extern "C" {

// A specification from per-position proposition sets: masks[i * stride + t]
// has bit p set iff proposition p holds at position t of trace i.
void* oracle_spec_new(int n_props, int n_traces, int n_pos, const int32_t* lengths,
                      const int32_t* masks, int stride) {
  if (n_props < 1 || n_props > 31 || n_traces < 0 || n_pos < 0 || n_pos > n_traces) return nullptr;
  Spec* s = new Spec;
  s->n_props = n_props;
  s->n_pos = n_pos;
  for (int i = 0; i < n_traces; ++i) {
    Trace tr;
    for (int t = 0; t < lengths[i]; ++t) {
      std::vector<bool> letter(n_props);
      for (int p = 0; p < n_props; ++p) letter[p] = ((masks[(size_t)i * stride + t] >> p) & 1) != 0;
      tr.holds.push_back(letter);
    }
    s->traces.push_back(tr);
  }
  return s;
}

void oracle_spec_free(void* s) { delete static_cast<Spec*>(s); }

// Characteristic matrix of a formula by the recursive definition. Returns the
// formula's size, -1 on a parse error or an atom out of range, -2 if the
// buffer is too small.
int oracle_eval(const void* spec, const char* formula, char* buf, size_t cap) {
  const Spec& s = *static_cast<const Spec*>(spec);
  Tree t;
  if (!parse_formula(formula, &t)) return -1;
  for (const Node& n : t.nodes) if (n.op == ATOM && n.prop >= s.n_props) return -1;
  if (copy_out(cm_by_tree(s, t), buf, cap) < 0) return -2;
  return (int)t.nodes.size();
}

// The same, computed bottom-up with the characteristic-sequence operators.
int oracle_eval_seq(const void* spec, const char* formula, char* buf, size_t cap) {
  const Spec& s = *static_cast<const Spec*>(spec);
  Tree t;
  if (!parse_formula(formula, &t)) return -1;
  for (const Node& n : t.nodes) if (n.op == ATOM && n.prop >= s.n_props) return -1;
  std::vector<CM> val(t.nodes.size());
  for (size_t n = 0; n < t.nodes.size(); ++n) {  // children precede parents in the node list
    const Node& x = t.nodes[n];
    for (const Trace& tr : s.traces) {
      const size_t k = val[n].size();
      if (x.op == ATOM) val[n].push_back(seq_atom(tr, x.prop));
      else if (!is_binary(x.op)) val[n].push_back(seq_unary(x.op, val[x.a][k]));
      else val[n].push_back(seq_binary(x.op, val[x.a][k], val[x.b][k]));
    }
  }
  if (copy_out(join(val[t.root]), buf, cap) < 0) return -2;
  return (int)t.nodes.size();
}

// 1 if the formula separates the specification, 0 if not, -1 on a parse error.
int oracle_separates(const void* spec, const char* formula) {
  const Spec& s = *static_cast<const Spec*>(spec);
  Tree t;
  if (!parse_formula(formula, &t)) return -1;
  for (const Node& n : t.nodes) if (n.op == ATOM && n.prop >= s.n_props) return -1;
  return separates_joined(s, cm_by_tree(s, t)) ? 1 : 0;
}

// Build levels 1..max_level completely (no early return).
void* oracle_enumerate(const void* spec, int max_level, unsigned op_mask) {
  Run* r = new Run;
  enumerate(*static_cast<const Spec*>(spec), max_level, op_mask, false, r);
  return r;
}

// The same levels, each level's candidates shared out among `threads` threads.
void* oracle_enumerate_threads(const void* spec, int max_level, unsigned op_mask, int threads) {
  Run* r = new Run;
  enumerate_threads(*static_cast<const Spec*>(spec), max_level, op_mask, threads, r);
  return r;
}

// Brute force over all syntax trees of size <= max_size.
void* oracle_bruteforce(const void* spec, int max_size, unsigned op_mask) {
  Run* r = new Run;
  brute_force(*static_cast<const Spec*>(spec), max_size, op_mask, r);
  return r;
}

void oracle_run_free(void* r) { delete static_cast<Run*>(r); }

int oracle_run_levels(const void* run) {
  const Run& r = *static_cast<const Run*>(run);
  return r.brute ? (int)r.bf_levels.size() - 1 : (int)r.levels.size() - 1;
}

int64_t oracle_level_size(const void* run, int k) {
  const Run& r = *static_cast<const Run*>(run);
  if (r.brute) return (k >= 1 && k < (int)r.bf_levels.size()) ? (int64_t)r.bf_levels[k].size() : -1;
  return (k >= 1 && k < (int)r.levels.size()) ? (int64_t)r.levels[k].size() : -1;
}

int64_t oracle_level_candidates(const void* run, int k) {
  const Run& r = *static_cast<const Run*>(run);
  return (k >= 1 && k < (int)r.candidates.size()) ? r.candidates[k] : -1;
}

// The characteristic matrix of entry idx of level k ('0'/'1', traces joined by ',').
int oracle_level_cm(const void* run, int k, int64_t idx, char* buf, size_t cap) {
  const Run& r = *static_cast<const Run*>(run);
  if (oracle_level_size(run, k) <= idx || idx < 0) return -1;
  if (r.brute) return copy_out(r.bf_levels[k][idx], buf, cap);
  return copy_out(join(r.levels[k][idx].cm), buf, cap);
}

// Entries [first, first + count) of level k, each characteristic matrix (as
// oracle_level_cm gives it) in a row of its own of `stride` bytes, padded
// with zero bytes. Returns the rows written, -1 on a bad range, -2 if a
// matrix does not fit a row. A plain copy, for exporting large levels.
int64_t oracle_level_cm_rows(const void* run, int k, int64_t first, int64_t count, char* buf, size_t stride) {
  if (first < 0 || count < 0 || first + count > oracle_level_size(run, k)) return -1;
  for (int64_t r = 0; r < count; ++r) {
    char* row = buf + (size_t)r * stride;
    std::memset(row, 0, stride);
    if (oracle_level_cm(run, k, first + r, row, stride) < 0) return -2;
  }
  return count;
}

// One formula with that characteristic matrix.
int oracle_level_formula(const void* run, int k, int64_t idx, char* buf, size_t cap) {
  const Run& r = *static_cast<const Run*>(run);
  if (oracle_level_size(run, k) <= idx || idx < 0) return -1;
  if (r.brute) return copy_out(r.bf_text.at(r.bf_levels[k][idx]), buf, cap);
  std::string f;
  formula_of(r, k, (int)idx, &f);
  return copy_out(f, buf, cap);
}

// Smallest separating formula (the listing's early return). Returns its size,
// 0 if none up to max_size, -2 if the buffer is too small. `constructed`
// receives the number of candidates built, atoms included.
int oracle_solve(const void* spec, int max_size, unsigned op_mask, char* buf, size_t cap,
                 int64_t* constructed) {
  Run r;
  enumerate(*static_cast<const Spec*>(spec), max_size, op_mask, true, &r);
  if (constructed) *constructed = r.constructed;
  if (r.solved_size == 0) { if (cap) buf[0] = '\0'; return 0; }
  if (copy_out(r.solved_formula, buf, cap) < 0) return -2;
  return r.solved_size;
}

}  // extern "C"
