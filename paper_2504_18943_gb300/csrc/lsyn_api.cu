// Host side of the lsyn C ABI (include/lsyn.h): context and memory layout,
// the level schedule of the bottom-up enumeration, solve, export and eval.
//
// The level loop follows the listing of paragraph "A generic program
// synthesiser" (section "Program synthesis"): level 1 is the distinct atoms;
// level k applies every unary operator to level k-1 and every binary operator
// to every split {i, j} with i + j = k - 1, checks every candidate against the
// specification and caches the new characteristic matrices. All of it runs in
// the kernels of lsyn_device.cuh; the host only plans launches and reads a
// few counters back per level.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lsyn.h"
#include "lsyn_ctx.h"
#include "lsyn_internal.h"

using namespace lsyn;

namespace {

thread_local std::string g_create_error;

uint32_t mix32(uint32_t x) {
  x ^= x >> 16; x *= 0x7FEB352Du; x ^= x >> 15; x *= 0x846CA68Bu; x ^= x >> 16;
  return x;
}


}  // namespace

std::string& lsyn::thread_error() { return g_create_error; }

double lsyn::now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

namespace {

// Clears the large table beside the first levels after a reset: one block
// per SM walking the table in grid strides, so that the level kernels on the
// caller's stream still find room on every SM (a memset's grid holds the SMs
// until it drains, and the first levels would wait behind it); streaming
// stores keep the zeroed lines from evicting the levels' rows from L2.
__global__ void __launch_bounds__(256) k_clear_table(uint4* t, size_t n16) {
  const size_t stride = size_t(gridDim.x) * blockDim.x;
  const uint4 z = make_uint4(0u, 0u, 0u, 0u);
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n16; i += stride) __stcs(t + i, z);
}

__global__ void k_level_begin(DevCounters* c) {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  c->t0 = t;
  c->timed_out = 0;
  c->full = 0;
  c->solved = 0;
  c->error = 0;
  c->defer_n[0] = 0;
  c->defer_n[1] = 0;
  c->defer_overflow = 0;
  c->holes_n = 0;
  for (int i = 0; i < kLaunchKinds; ++i) c->built_k[i] = c->inserted_k[i] = 0;
  for (int i = 0; i < 8; ++i) c->work[i] = 0;
  c->sol = ~0ull;
}

__device__ void reconstruct_one(const unsigned long long* prov, unsigned long long root,
                                const unsigned long long* root_ptr, char* buf, unsigned cap, int* status) {
  const char kOp[8] = {'p', '!', '&', '|', 'X', 'F', 'G', 'U'};
  struct Frame {
    unsigned long long d;
    int stage;
  };
  Frame st[80];
  int sp = 0;
  unsigned n = 0;
  int bad = 0;
  st[sp++] = {root_ptr ? *root_ptr : root, 0};
  auto put = [&](char ch) {
    if (n + 1 < cap) buf[n++] = ch;
    else bad = 1;
  };
  while (sp > 0 && !bad) {
    Frame& f = st[sp - 1];
    const unsigned op = desc_op(f.d);
    if (op == kAtom) {
      put('p');
      char tmp[12];
      int m = 0;
      unsigned v = desc_left(f.d);
      do { tmp[m++] = char('0' + v % 10); v /= 10; } while (v);
      while (m) put(tmp[--m]);
      --sp;
      continue;
    }
    const bool bin = op == kAnd || op == kOr || op == kUntil;
    if (f.stage == 0) {
      put('(');
      put(kOp[op & 7]);
      put(' ');
      f.stage = 1;
      if (sp >= 80) { bad = 2; break; }
      st[sp++] = {prov[desc_left(f.d)], 0};
    } else if (f.stage == 1 && bin) {
      put(' ');
      f.stage = 2;
      if (sp >= 80) { bad = 2; break; }
      st[sp++] = {prov[desc_right(f.d)], 0};
    } else {
      put(')');
      --sp;
    }
  }
  buf[n < cap ? n : cap - 1] = '\0';
  *status = bad;
}

__global__ void k_reconstruct(const unsigned long long* prov, unsigned long long root,
                              const unsigned long long* root_ptr, char* buf, unsigned cap, int* status) {
  reconstruct_one(prov, root, root_ptr, buf, cap, status);
}

// One formula per block (thread 0): item i writes buf + i * cap and status[i].
__global__ void k_reconstruct_many(const lsyn::FormulaItem* items, int n, char* buf, unsigned cap, int* status) {
  const int i = blockIdx.x;
  if (i >= n || threadIdx.x != 0) return;
  reconstruct_one(items[i].prov, 0, items[i].root, buf + size_t(i) * cap, cap, status + i);
}

// Candidates built at level k given the sizes of levels 1..k-1 (sizes[i-1]).
int64_t level_candidates(const int64_t* sizes, int k, uint32_t mask) {
  if (k < 2) return 0;
  const int nu = !!(mask & LSYN_OP_NOT) + !!(mask & LSYN_OP_X) + !!(mask & LSYN_OP_F) + !!(mask & LSYN_OP_G);
  const int nb = !!(mask & LSYN_OP_AND) + !!(mask & LSYN_OP_OR) + 2 * !!(mask & LSYN_OP_U);
  int64_t c = int64_t(nu) * sizes[k - 2];
  for (int i = 1; 2 * i <= k - 1; ++i) {
    const int j = k - 1 - i;
    const int64_t a = sizes[i - 1], b = sizes[j - 1];
    c += nb * (i == j ? a * (a - 1) / 2 : a * b);
  }
  return c;
}

lsyn_status launch_desc(lsyn_ctx* c, const CacheView& cv, const unsigned long long* list, const unsigned* list_n,
                        unsigned n, unsigned atoms, const LaunchCfg& lc) {
  cudaError_t e = c->word_bits == 32 ? Kernels<uint32_t>::desc_list(cv, list, list_n, n, atoms, lc)
                                     : Kernels<uint64_t>::desc_list(cv, list, list_n, n, atoms, lc);
  return e == cudaSuccess ? LSYN_OK : c->cuda_fail(e, "desc kernel");
}

}  // namespace

cudaError_t lsyn::launch_level_begin(DevCounters* c, cudaStream_t stream) {
  k_level_begin<<<1, 1, 0, stream>>>(c);
  return cudaGetLastError();
}

cudaError_t lsyn::reconstruct_many(const FormulaItem* items, int n, char* buf, unsigned cap, int* status,
                                   cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  k_reconstruct_many<<<n, 32, 0, stream>>>(items, n, buf, cap, status);
  return cudaGetLastError();
}

lsyn_status lsyn::ctx_reconstruct(lsyn_ctx* c, const unsigned long long* root_ptr, char* out, size_t cap) {
  k_reconstruct<<<1, 1, 0, c->stream>>>(c->prov, 0, root_ptr, c->fbuf, lsyn_ctx::kFormulaCap, c->fstatus);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return c->cuda_fail(e, "reconstruct");
  e = cudaMemcpyAsync(c->h_fbuf, c->fbuf, lsyn_ctx::kFormulaCap, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->h_fstatus, c->fstatus, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return c->cuda_fail(e, "reconstruct copy");
  if (*c->h_fstatus != 0) return c->fail(LSYN_E_STATE, "formula too deep or too long to print");
  const size_t len = strnlen(c->h_fbuf, lsyn_ctx::kFormulaCap);
  if (!out || len + 1 > cap) return c->fail(LSYN_E_INVAL, "formula buffer too small");
  memcpy(out, c->h_fbuf, len + 1);
  return LSYN_OK;
}

namespace {

// Parse prefix formula text into a postorder node list (children first).
bool parse_formula(const char* s, int n_props, std::vector<int4>* nodes, std::string* err) {
  size_t i = 0;
  const size_t len = strlen(s);
  struct P {
    const char* s;
    size_t len;
    size_t& i;
    int n_props;
    std::vector<int4>* nodes;
    std::string* err;
    int depth = 0;
    void skip() { while (i < len && (s[i] == ' ' || s[i] == '\t' || s[i] == '\n')) ++i; }
    int parse() {
      if (++depth > 4096 || nodes->size() > 4096) { *err = "formula too large"; return -1; }
      skip();
      if (i < len && s[i] == 'p') {
        ++i;
        if (i >= len || s[i] < '0' || s[i] > '9') { *err = "bad atom"; return -1; }
        long v = 0;
        while (i < len && s[i] >= '0' && s[i] <= '9') { v = v * 10 + (s[i] - '0'); if (v > 1000) break; ++i; }
        if (v >= n_props) { *err = "atom out of range"; return -1; }
        nodes->push_back(make_int4(int(kAtom), -1, -1, int(v)));
        --depth;
        return int(nodes->size()) - 1;
      }
      if (i >= len || s[i] != '(') { *err = "expected '(' or atom"; return -1; }
      ++i;
      skip();
      if (i >= len) { *err = "truncated"; return -1; }
      int op = -1;
      switch (s[i]) {
        case '!': op = kNot; break;
        case '&': op = kAnd; break;
        case '|': op = kOr; break;
        case 'X': op = kNext; break;
        case 'F': op = kFuture; break;
        case 'G': op = kGlobally; break;
        case 'U': op = kUntil; break;
        default: *err = "unknown operator"; return -1;
      }
      ++i;
      const int a = parse();
      if (a < 0) return -1;
      int b = -1;
      if (op == kAnd || op == kOr || op == kUntil) {
        b = parse();
        if (b < 0) return -1;
      }
      skip();
      if (i >= len || s[i] != ')') { *err = "expected ')'"; return -1; }
      ++i;
      nodes->push_back(make_int4(op, a, b, 0));
      --depth;
      return int(nodes->size()) - 1;
    }
  } p{s, len, i, n_props, nodes, err};
  if (p.parse() < 0) return false;
  p.skip();
  if (i != len) { *err = "trailing text"; return false; }
  return true;
}

// Words per trace at most (traces up to 16 x word_bits positions).
constexpr int kMaxPlanes = 16;

struct Layout {
  int T = 0, word_bits = 0, max_len = 0, steps = 0;
  int planes = 1;                // words per trace
  unsigned plane_vecs_needed = 0;  // 16-byte vectors of one word per trace
  unsigned vecs_needed = 0;        // all planes
};

lsyn_status validate(const lsyn_problem* p, Layout* L, std::string* err) {
  if (!p) { *err = "problem is NULL"; return LSYN_E_INVAL; }
  if (p->n_props < 1 || p->n_props > 32) { *err = "n_props must be in 1..32"; return LSYN_E_INVAL; }
  if (p->n_pos < 0 || p->n_neg < 0 || p->n_pos + p->n_neg < 1) { *err = "need n_pos, n_neg >= 0 and at least one trace"; return LSYN_E_INVAL; }
  if (p->word_bits != 32 && p->word_bits != 64) { *err = "word_bits must be 32 or 64"; return LSYN_E_INVAL; }
  if (!p->lengths || !p->atom_words) { *err = "lengths and atom_words are required"; return LSYN_E_INVAL; }
  L->T = p->n_pos + p->n_neg;
  if (L->T > (1 << 24)) { *err = "too many traces"; return LSYN_E_INVAL; }
  L->word_bits = p->word_bits;
  L->max_len = 1;
  for (int i = 0; i < L->T; ++i) {
    if (p->lengths[i] < 1 || p->lengths[i] > p->word_bits * kMaxPlanes) {
      *err = "trace " + std::to_string(i) + " has a length outside 1.." + std::to_string(p->word_bits * kMaxPlanes);
      return LSYN_E_INVAL;
    }
    L->max_len = std::max(L->max_len, int(p->lengths[i]));
  }
  L->planes = (L->max_len + p->word_bits - 1) / p->word_bits;
  L->steps = 0;  // log-step shifts within one word
  while ((1 << L->steps) < std::min(L->max_len, p->word_bits)) ++L->steps;
  L->plane_vecs_needed = unsigned((size_t(L->T) * (p->word_bits / 8) + 15) / 16);
  L->vecs_needed = L->plane_vecs_needed * unsigned(L->planes);
  return LSYN_OK;
}

// Pack the padded per-word constants and atom rows on the host: `vecs`
// vectors per CM, plane j (a word of every trace) at vector j * plane_vecs.
void pack_host(const lsyn_problem* p, const Layout& L, unsigned vecs, unsigned plane_vecs,
               std::vector<uint32_t>* consts, std::vector<uint32_t>* atoms) {
  const unsigned n32 = vecs * 4;  // 32-bit words per padded CM
  consts->assign(size_t(5) * n32, 0u);
  atoms->assign(size_t(p->n_props) * n32, 0u);
  uint32_t* lm = consts->data();
  uint32_t* lab = lm + n32;
  uint32_t* care = lab + n32;
  uint32_t* key = care + n32;
  uint32_t* mul = key + n32;
  const int per = p->word_bits / 32;  // 32-bit halves per word
  // Words are stored position 0 first (most significant bit); the 32-bit
  // halves of a 64-bit word are little-endian in memory.
  auto store = [&](uint32_t* dst, int i, uint64_t w_lsb_first) {
    if (per == 1) {
      dst[i] = rev32(uint32_t(w_lsb_first));
    } else {
      const uint64_t r = rev64(w_lsb_first);
      dst[2 * i] = uint32_t(r);
      dst[2 * i + 1] = uint32_t(r >> 32);
    }
  };
  const int wb = p->word_bits;
  const unsigned words_per_plane = plane_vecs * unsigned(4 / per);  // in words of word_bits bits
  for (int i = 0; i < L.T; ++i) {
    const int len = p->lengths[i];
    store(lab, i, i < p->n_pos ? 1ull : 0ull);  // the position-0 bit (plane 0)
    store(care, i, 1ull);
    for (int j = 0; j < L.planes; ++j) {
      // positions j*wb .. j*wb + wb - 1 of the trace, those before its end
      const int n_in = std::max(0, std::min(wb, len - j * wb));
      const uint64_t m = n_in >= 64 ? ~0ull : ((1ull << n_in) - 1ull);
      const int at = int(unsigned(j) * words_per_plane) + i;
      store(lm, at, m);
      for (int q = 0; q < p->n_props; ++q) {
        const size_t src = (size_t(q) * size_t(L.T) + size_t(i)) * size_t(L.planes) + size_t(j);
        uint64_t w;
        if (per == 1) w = static_cast<const uint32_t*>(p->atom_words)[src];
        else w = static_cast<const uint64_t*>(p->atom_words)[src];
        store(atoms->data() + size_t(q) * n32, at, w & m);
      }
    }
  }
  for (unsigned i = 0; i < n32; ++i) {
    key[i] = mix32(i * 2u + 0x51ED270Bu);
    mul[i] = mix32(i * 2u + 0x2545F491u) | 1u;
  }
}

// One internal row (planes x plane_vecs vectors, position 0 in the top bit)
// to the ABI's [trace][plane] words with bit t = position t.
void planes_to_abi(const uint8_t* row, uint8_t* dst, int T, int planes, unsigned plane_vecs, int word_bits) {
  const size_t wbytes = size_t(word_bits / 8);
  const size_t words_per_plane = size_t(plane_vecs) * 16 / wbytes;
  for (int i = 0; i < T; ++i)
    for (int j = 0; j < planes; ++j) {
      uint8_t* d = dst + (size_t(i) * size_t(planes) + size_t(j)) * wbytes;
      memcpy(d, row + (size_t(j) * words_per_plane + size_t(i)) * wbytes, wbytes);
      reverse_words(d, 1, word_bits);
    }
}

}  // namespace


bool lsyn::cache_sizing(unsigned long long cache_bytes, size_t M, double load, unsigned long long* table_cap,
                        unsigned long long* entries) {
  unsigned long long best_cap = 0, best_e = 0;
  for (unsigned long long cap = 1024; cap <= (1ull << 32); cap <<= 1) {
    if (cap * 8 >= cache_bytes) break;
    unsigned long long e = (cache_bytes - cap * 8) / (M + kEntryMetaBytes);
    e = std::min<unsigned long long>(e, (unsigned long long)(double(cap) * load));
    e = std::min<unsigned long long>(e, kMaxEntries);
    if (e > best_e) { best_e = e; best_cap = cap; }
  }
  *table_cap = best_cap;
  *entries = best_e;
  return best_e >= 64;
}

uint32_t lsyn::plan_hole_moves(const uint2* holes, unsigned n, uint32_t start, uint32_t total,
                               std::vector<uint2>* mv) {
  std::vector<std::pair<uint32_t, uint32_t>> rng;
  for (unsigned i = 0; i < n; ++i) {
    const uint32_t lo = std::max(holes[i].x, start), hi = std::min(holes[i].y, total);
    if (lo < hi) rng.push_back({lo, hi});
  }
  std::sort(rng.begin(), rng.end());
  uint64_t H = 0;
  for (auto& r : rng) H += r.second - r.first;
  const uint32_t dense_end = total - uint32_t(H);
  size_t ri = 0;  // range holding or following the next valid candidate id >= dense_end
  uint32_t v = dense_end;
  auto next_valid = [&]() {
    while (ri < rng.size() && rng[ri].second <= v) ++ri;
    while (ri < rng.size() && rng[ri].first <= v && v < rng[ri].second) { v = rng[ri].second; ++ri; }
  };
  for (auto& r : rng) {
    for (uint32_t hole = r.first; hole < r.second && hole < dense_end; ++hole) {
      next_valid();
      mv->push_back(make_uint2(v, hole));
      ++v;
    }
  }
  return dense_end;
}

void lsyn::ctx_level_plan(lsyn_ctx* c, int k, LevelPlan* lp) {
  *lp = LevelPlan();
  memset(&lp->plan, 0, sizeof(lp->plan));
  lp->start = c->level_start.back() + c->level_n.back();
  // Ids a warp reserves at a time: large enough to keep the shared counter
  // cold, small enough that the reservations of every resident warp stay a
  // small part of the free arena.
  {
    const unsigned long long free_ids = c->max_entries > lp->start ? c->max_entries - lp->start : 0;
    const unsigned long long warps = (unsigned long long)c->sms * 24ull;
    c->chunk = unsigned(std::max(1ull, std::min(32ull, free_ids / (8ull * warps))));
    // a small level: chunks no larger than its candidates spread over the
    // warps, so that the ids warps leave unused (holes to close) stay few
    const long long cand = level_candidate_count(c, k);
    if (cand > 0)
      c->chunk = unsigned(std::max(1ull, std::min<unsigned long long>(c->chunk, (unsigned long long)cand / (8ull * warps))));
  }
  const double M = double(c->vecs) * 16.0;
  if (k == 1) {
    lp->op_bytes_unary = double(c->n_props) * M;
    return;
  }
  const uint32_t m = c->op_mask;
  lp->uops = ((m & LSYN_OP_NOT) ? 1u : 0u) | ((m & LSYN_OP_X) ? 2u : 0u) | ((m & LSYN_OP_F) ? 4u : 0u) |
             ((m & LSYN_OP_G) ? 8u : 0u);
  lp->u_first = c->level_start[k - 1];
  lp->u_count = lp->uops ? c->level_n[k - 1] : 0;
  lp->op_bytes_unary = double(lp->u_count) * M;
  lp->cand_unary = double(lp->u_count) * double(__builtin_popcount(lp->uops));
  const uint32_t bops = ((m & LSYN_OP_AND) ? 1u : 0u) | ((m & LSYN_OP_OR) ? 2u : 0u) | ((m & LSYN_OP_U) ? 12u : 0u);
  if (!bops || k < 3) return;
  BinaryPlan& plan = lp->plan;
  plan.ops = bops;
  plan.work_slot = 0;
  plan.tile = c->path == 2 ? std::max(1u, std::min(32u, unsigned((48 * 1024) / (c->vecs * 16)))) : 1u;
  if (c->path == 2 && c->tile_rows) {
    plan.tile = c->tile_rows;
    plan.tile_fixed = 1;
  }
  unsigned long long tiles = 0, pairs = 0;
  for (int i = 1; 2 * i <= k - 1; ++i) {
    const int j = k - 1 - i;
    const uint32_t ni = c->level_n[i], nj = c->level_n[j];
    if (!ni || !nj || (i == j && ni < 2)) continue;
    Split sp;
    memset(&sp, 0, sizeof(sp));
    if (i == j || ni <= nj) {
      sp.left_start = c->level_start[i]; sp.left_n = ni;
      sp.right_start = c->level_start[j]; sp.right_n = nj;
    } else {
      sp.left_start = c->level_start[j]; sp.left_n = nj;
      sp.right_start = c->level_start[i]; sp.right_n = ni;
    }
    sp.tri = i == j ? 1u : 0u;
    sp.lt_tiles = (sp.left_n + plan.tile - 1) / plan.tile;
    sp.rt_tiles = (sp.right_n + plan.tile - 1) / plan.tile;
    sp.tiles_begin = tiles;
    sp.pairs_begin = pairs;
    // a level with itself: the unordered pairs a < b (and, or and both orders of U)
    sp.pairs = sp.tri ? (unsigned long long)sp.left_n * (sp.left_n - 1) / 2 : (unsigned long long)sp.left_n * sp.right_n;
    tiles += (unsigned long long)sp.lt_tiles * sp.rt_tiles;
    pairs += sp.pairs;
    lp->op_bytes_binary += double(sp.left_n + (sp.tri ? 0u : sp.right_n)) * M;
    plan.s[plan.n_splits++] = sp;
  }
  plan.total_tiles = tiles;
  plan.total_pairs = pairs;
}

lsyn_status lsyn::ctx_commit_level(lsyn_ctx* c, int k, const DevCounters& h, uint32_t total,
                                   unsigned long long deferred, const LevelPlan& lp, lsyn_level_stats* out) {
  const uint32_t start = lp.start;
  const uint32_t unique = total - start;
  if (h.inserted() != unique)
    return c->fail(LSYN_E_STATE, "insert count " + std::to_string(h.inserted()) + " differs from the level size " +
                                     std::to_string(unique));
  c->level_start.push_back(start);
  c->level_n.push_back(unique);
  c->levels_done = k;
  std::vector<int64_t> sizes(c->level_n.begin() + 1, c->level_n.end());
  const int64_t planned = k == 1 ? c->n_props : level_candidates(sizes.data(), k, c->op_mask);
  const bool stopped = h.solved && c->full_levels == false && int64_t(h.built()) < planned;
  c->last_incomplete = h.full || stopped;
  c->constructed += h.built();
  c->last_sol = h.solved ? h.sol : ~0ull;
  if (out) {
    memset(out, 0, sizeof(*out));
    out->level = k;
    out->solved = h.solved ? 1 : 0;
    out->cache_full = h.full ? 1 : 0;
    out->early_exit = stopped ? 1 : 0;
    out->candidates = int64_t(h.built());
    out->unique = unique;
    out->total = total;
    out->deferred = int64_t(deferred);
    const double M = double(c->vecs) * 16.0;
    const double C = double(h.built()), U = double(unique);
    // a level that stopped at a solution read only part of its operands
    const double done = planned > 0 ? std::min(1.0, C / double(planned)) : 1.0;
    out->bytes_alg = (lp.op_bytes_unary + lp.op_bytes_binary) * done + C * 32.0 + (C - U) * M + U * (M + 16.0);
  }
  return LSYN_OK;
}

int64_t lsyn::level_candidate_count(const lsyn_ctx* c, int k) {
  if (k == 1) return c->n_props;
  std::vector<int64_t> sizes(c->level_n.begin() + 1, c->level_n.end());
  if (int(sizes.size()) < k - 1) return 0;
  return level_candidates(sizes.data(), k, c->op_mask);
}

extern "C" {

const char* lsyn_version(void) { return "lsyn 0.1 (sm_103a)"; }

int64_t lsyn_level_candidates(const int64_t* level_sizes, int32_t k, uint32_t op_mask) {
  if (!level_sizes || k < 2) return 0;
  return level_candidates(level_sizes, k, op_mask ? op_mask : LSYN_OPS_ALL);
}

const char* lsyn_last_error(const lsyn_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

void lsyn_destroy(lsyn_ctx* c) {
  if (!c || c->borrowed) return;  // a borrowed handle belongs to its batch or server
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  if (c->side) cudaStreamSynchronize(c->side);  // a clear of the big table may still run there
  if (c->events_ready)
    for (auto& e : c->ev) if (e) cudaEventDestroy(e);
  for (auto& e : c->ev_side) if (e) cudaEventDestroy(e);
  if (c->side) cudaStreamDestroy(c->side);
  c->mem.release_all();
  if (c->owns_host) {
    if (c->h_snap) cudaFreeHost(c->h_snap);
    if (c->h_fbuf) cudaFreeHost(c->h_fbuf);
    if (c->h_fstatus) cudaFreeHost(c->h_fstatus);
  }
  if (prev >= 0) cudaSetDevice(prev);
  delete c;
}

lsyn_status lsyn_create(const lsyn_problem* problem, const lsyn_config* config, lsyn_ctx** out) {
  return lsyn::ctx_create(problem, config, false, out);
}

}  // extern "C"

lsyn_status lsyn::ctx_shell(const lsyn_problem* problem, const lsyn_config* config, bool warp_layout,
                            lsyn_ctx** out, std::vector<uint32_t>* consts, std::vector<uint32_t>* atoms) {
  g_create_error.clear();
  if (!out) { g_create_error = "out is NULL"; return LSYN_E_INVAL; }
  *out = nullptr;
  Layout L;
  lsyn_status s = validate(problem, &L, &g_create_error);
  if (s != LSYN_OK) return s;
  lsyn_config cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.device = -1;
  if (config) cfg = *config;
  const uint32_t mask = cfg.op_mask ? cfg.op_mask : LSYN_OPS_ALL;
  if (mask & ~LSYN_OPS_ALL) { g_create_error = "unknown operator bits"; return LSYN_E_INVAL; }
  const double load = cfg.table_load > 0 ? cfg.table_load : 0.5;
  if (!(load > 0 && load <= 0.9)) { g_create_error = "table_load must be in (0, 0.9]"; return LSYN_E_INVAL; }
  const unsigned long long cache_bytes = cfg.cache_bytes ? cfg.cache_bytes : (1ull << 30);
  if (cfg.tile_rows != 0 && cfg.tile_rows != 8 && cfg.tile_rows != 16 && cfg.tile_rows != 32) {
    g_create_error = "tile_rows must be 0, 8, 16 or 32";
    return LSYN_E_INVAL;
  }
  if (!(cfg.time_limit_ms >= 0)) { g_create_error = "time_limit_ms must be >= 0"; return LSYN_E_INVAL; }

  // Paths: A (thread per candidate) up to 128 bytes, padded to a power of two
  // of 16-byte vectors; C (one vector per lane) up to 512 bytes; D (whole
  // warps of vectors, looped per lane) up to 64 KiB.
  // Traces longer than a word (several planes) always take path D, each plane
  // padded to whole warps of vectors so a lane holds the same traces' words in
  // every plane.
  unsigned vecs = 0, plane_vecs = 0;
  if (L.planes == 1 && L.vecs_needed <= 8 && !warp_layout) {
    vecs = 1;
    while (vecs < L.vecs_needed) vecs <<= 1;
    plane_vecs = vecs;
  } else if (L.planes == 1 && L.vecs_needed <= 4096) {
    vecs = (L.vecs_needed + 31u) / 32u * 32u;
    plane_vecs = vecs;
  } else if (L.planes > 1 && (L.plane_vecs_needed + 31u) / 32u * 32u * unsigned(L.planes) <= 4096) {
    plane_vecs = (L.plane_vecs_needed + 31u) / 32u * 32u;
    vecs = plane_vecs * unsigned(L.planes);
  } else {
    g_create_error = "characteristic matrices above 64 KiB (" + std::to_string(L.vecs_needed * 16) +
                     " bytes) are not supported: at most 64 KiB";
    return LSYN_E_UNSUPPORTED;
  }
  const size_t M = size_t(vecs) * 16;
  unsigned long long best_cap = 0, best_e = 0;
  if (!cache_sizing(cache_bytes, M, load, &best_cap, &best_e)) {
    g_create_error = "cache_bytes too small";
    return LSYN_E_INVAL;
  }

  lsyn_ctx* c = new (std::nothrow) lsyn_ctx;
  if (!c) { g_create_error = "out of host memory"; return LSYN_E_NOMEM; }
  c->op_mask = mask;
  c->full_levels = cfg.full_levels != 0;
  c->timing = cfg.timing != 0;
  c->table_load = load;
  c->mem.alloc = cfg.alloc;
  c->mem.free = cfg.free;
  c->mem.user = cfg.alloc_user;
  c->stream = static_cast<cudaStream_t>(cfg.stream);
  c->n_props = problem->n_props;
  c->n_pos = problem->n_pos;
  c->n_neg = problem->n_neg;
  c->T = L.T;
  c->word_bits = L.word_bits;
  c->max_len = L.max_len;
  c->steps = L.steps;
  c->vecs = vecs;
  c->planes = unsigned(L.planes);
  c->plane_vecs = plane_vecs;
  c->path = vecs <= 8 ? 1 : vecs == 32 ? 2 : 3;
  c->table_cap = best_cap;
  c->max_entries = unsigned(best_e);
  c->defer_cap = cfg.defer_cap ? cfg.defer_cap : unsigned(std::max(1ull << 16, std::min(1ull << 23, best_e / 16)));
  c->hole_cap = cfg.hole_cap ? std::min(cfg.hole_cap, 1u << 24) : 1u << 16;
  c->tile_rows = unsigned(cfg.tile_rows);
  c->time_limit_ms = cfg.time_limit_ms;
  c->move_cap = c->hole_cap * 32u;
  cudaError_t e;
  if (cfg.device >= 0 && (e = cudaSetDevice(cfg.device)) != cudaSuccess) {
    delete c;
    g_create_error = cudaGetErrorString(e);
    return LSYN_E_CUDA;
  }
  if ((e = cudaGetDevice(&c->device)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device)) != cudaSuccess) {
    delete c;
    g_create_error = cudaGetErrorString(e);
    return LSYN_E_CUDA;
  }
  if (consts && atoms) pack_host(problem, L, vecs, plane_vecs, consts, atoms);
  c->level_start.assign(1, 0);
  c->level_n.assign(1, 0);
  *out = c;
  return LSYN_OK;
}

lsyn_status lsyn::ctx_create(const lsyn_problem* problem, const lsyn_config* config, bool warp_layout,
                             lsyn_ctx** out) {
  std::vector<uint32_t> consts, atoms;
  lsyn_ctx* c = nullptr;
  lsyn_status s = ctx_shell(problem, config, warp_layout, &c, &consts, &atoms);
  if (s != LSYN_OK) return s;
  const size_t M = size_t(c->vecs) * 16;
  auto bail = [&](lsyn_status st, const std::string& msg) {
    g_create_error = msg;
    lsyn_destroy(c);
    return st;
  };
  cudaError_t e;
  c->arena = static_cast<uint4*>(c->mem.get(size_t(c->max_entries) * M));
  c->prov = static_cast<unsigned long long*>(c->mem.get(size_t(c->max_entries) * 8));
  c->table = static_cast<unsigned long long*>(c->mem.get(size_t(c->table_cap) * 8));
  c->ctr = static_cast<DevCounters*>(c->mem.get(sizeof(DevCounters)));
  c->consts = static_cast<uint4*>(c->mem.get(size_t(5) * M));
  c->atoms = static_cast<uint4*>(c->mem.get(size_t(c->n_props) * M));
  c->defer[0] = static_cast<unsigned long long*>(c->mem.get(size_t(c->defer_cap) * 8));
  c->defer[1] = static_cast<unsigned long long*>(c->mem.get(size_t(c->defer_cap) * 8));
  c->slotpos = static_cast<unsigned*>(c->mem.get(size_t(c->max_entries) * 4));
  c->homes = static_cast<unsigned*>(c->mem.get(size_t(c->max_entries) * 4));
  c->holes = static_cast<uint2*>(c->mem.get(size_t(c->hole_cap) * sizeof(uint2)));
  c->moves = static_cast<uint2*>(c->mem.get(size_t(c->move_cap) * sizeof(uint2)));
  c->hole_bits = static_cast<unsigned*>(c->mem.get((3 * size_t(c->hole_cap) + 32) * sizeof(unsigned)));
  c->fbuf = static_cast<char*>(c->mem.get(lsyn_ctx::kFormulaCap));
  c->fstatus = static_cast<int*>(c->mem.get(sizeof(int)));
  if (!c->arena || !c->prov || !c->table || !c->ctr || !c->consts || !c->atoms || !c->defer[0] || !c->defer[1] ||
      !c->fbuf || !c->fstatus || !c->slotpos || !c->homes || !c->holes || !c->moves || !c->hole_bits)
    return bail(LSYN_E_NOMEM, "device allocation failed");
  c->big_table = c->table;
  c->big_cap = c->table_cap;
  if (c->big_cap >= 8 * lsyn_ctx::kFrontSlots) {
    c->front_table = static_cast<unsigned long long*>(c->mem.get(size_t(lsyn_ctx::kFrontSlots) * 8));
    if (!c->front_table) return bail(LSYN_E_NOMEM, "device allocation failed");
    if ((e = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking)) != cudaSuccess)
      return bail(LSYN_E_CUDA, cudaGetErrorString(e));
    for (auto& ev : c->ev_side)
      if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
        return bail(LSYN_E_CUDA, cudaGetErrorString(e));
    c->front_cap = lsyn_ctx::kFrontSlots;
  }
  if (cudaMallocHost(&c->h_snap, sizeof(Snap) * lsyn_ctx::kSnaps) != cudaSuccess ||
      cudaMallocHost(&c->h_fbuf, lsyn_ctx::kFormulaCap) != cudaSuccess ||
      cudaMallocHost(&c->h_fstatus, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return bail(LSYN_E_NOMEM, "pinned host allocation failed");
  }
  c->owns_host = true;
  for (auto& ev : c->ev)
    if ((e = cudaEventCreate(&ev)) != cudaSuccess) return bail(LSYN_E_CUDA, cudaGetErrorString(e));
  c->events_ready = true;

  e = cudaMemcpyAsync(c->consts, consts.data(), consts.size() * 4, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->atoms, atoms.data(), atoms.size() * 4, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);  // host vectors go out of scope
  if (e != cudaSuccess) return bail(LSYN_E_CUDA, cudaGetErrorString(e));
  s = lsyn_reset(c);
  if (s != LSYN_OK) return bail(s, c->err);
  *out = c;
  return LSYN_OK;
}

extern "C" {

lsyn_status lsyn_reset(lsyn_ctx* c) {
  if (!c) return LSYN_E_INVAL;
  if (c->borrowed) return c->fail(LSYN_E_STATE, "a batch or server problem is driven by its owner");
  cudaSetDevice(c->device);
  cudaError_t e;
  if (c->front_cap) {
    // the front table now; the big one on the side stream, after the work
    // queued so far on the main stream (which may still read it)
    e = cudaMemsetAsync(c->front_table, 0, size_t(c->front_cap) * 8, c->stream);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_side[0], c->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->side, c->ev_side[0], 0);
    // An SM runs blocks of kernels side by side only while its shared-memory
    // carveout suits them all: the clear asks for the largest carveout, which
    // every level and close kernel fits in, so that none waits for the clear.
    static const cudaError_t carve = cudaFuncSetAttribute(
        (const void*)k_clear_table, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess) e = carve;
    if (e == cudaSuccess) {
      k_clear_table<<<c->sms, 256, 0, c->side>>>(reinterpret_cast<uint4*>(c->big_table), size_t(c->big_cap) / 2);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_side[1], c->side);
    c->table = c->front_table;
    c->table_cap = c->front_cap;
    c->front_active = true;
    c->big_clear_pending = true;
  } else {
    e = cudaMemsetAsync(c->table, 0, size_t(c->table_cap) * 8, c->stream);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(c->ctr, 0, sizeof(DevCounters), c->stream);
  if (e != cudaSuccess) return c->cuda_fail(e, "reset");
  c->level_start.assign(1, 0);
  c->level_n.assign(1, 0);
  c->levels_done = 0;
  c->last_incomplete = false;
  c->needs_reset = false;
  c->constructed = 0;
  c->last_sol = ~0ull;
  return LSYN_OK;
}

lsyn_status lsyn_enumerate_level(lsyn_ctx* c, int32_t k, lsyn_level_stats* out) {
  if (!c) return LSYN_E_INVAL;
  if (c->borrowed) return c->fail(LSYN_E_STATE, "a batch or server problem is driven by its owner");
  if (c->needs_reset) return c->fail(LSYN_E_STATE, "a level was interrupted by the time limit: reset the context");
  if (k != c->levels_done + 1) return c->fail(LSYN_E_STATE, "level k must be levels_done + 1");
  if (c->last_incomplete) return c->fail(LSYN_E_STATE, "the previous level is incomplete (cache full or stopped early)");
  if (k > 64) return c->fail(LSYN_E_INVAL, "levels above 64 are not supported");
  cudaSetDevice(c->device);
  const double t0 = now_ms();
  LaunchCfg lc{c->stream, c->sms};
  int snap = 0, evn = 0;
  int ev_kind[lsyn_ctx::kSnaps];
  cudaError_t e;
  auto take_snap = [&]() -> cudaError_t {
    if (snap >= lsyn_ctx::kSnaps) return cudaErrorInvalidValue;
    return cudaMemcpyAsync(&c->h_snap[snap++].c, c->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, c->stream);
  };
  auto ev_begin = [&]() { if (c->timing) cudaEventRecord(c->ev[2 * evn], c->stream); };
  auto ev_end = [&](int kind) {
    if (c->timing) { cudaEventRecord(c->ev[2 * evn + 1], c->stream); ev_kind[evn] = kind; }
    ++evn;
  };

  LevelPlan lp;
  ctx_level_plan(c, k, &lp);
  const uint32_t start = lp.start;
  int launches = 0;
  // inside lsyn_solve with a time limit: what is left of it is this level's budget
  c->level_budget_ns = 0;
  if (c->solve_deadline_ms > 0) {
    const double left_ms = c->solve_deadline_ms - t0;
    c->level_budget_ns = left_ms > 0 ? (unsigned long long)(left_ms * 1e6) + 1ull : 1ull;
  }
  ev_begin();
  k_level_begin<<<1, 1, 0, c->stream>>>(c->ctr);
  ++launches;
  if ((e = cudaGetLastError()) != cudaSuccess) return c->cuda_fail(e, "level begin");
  // Leave the front table before a level whose candidates could load it past
  // table_load: wait for the big table's clear, then re-insert every entry's
  // slot there (by its hash home; levels are closed, so every slot is
  // published). An overflow of the rebuild is reported with the level.
  if (c->front_active) {
    const long long cand = level_candidate_count(c, k);  // negative: overflowed, so unbounded
    if (cand < 0 || double(start) + double(cand) > double(c->front_cap) * c->table_load) {
      if ((e = cudaStreamWaitEvent(c->stream, c->ev_side[1], 0)) != cudaSuccess) return c->cuda_fail(e, "table switch");
      c->big_clear_pending = false;
      e = c->word_bits == 32 ? Kernels<uint32_t>::rehash(c->front_table, c->front_cap, c->big_table, c->big_cap,
                                                         c->homes, c->slotpos, start, &c->ctr->error, lc)
                             : Kernels<uint64_t>::rehash(c->front_table, c->front_cap, c->big_table, c->big_cap,
                                                         c->homes, c->slotpos, start, &c->ctr->error, lc);
      ++launches;
      if (e != cudaSuccess) return c->cuda_fail(e, "table switch");
      c->table = c->big_table;
      c->table_cap = c->big_cap;
      c->front_active = false;
    }
  }
  ev_end(3);

  // Each launch counts into its own kind of the level's counters
  // (DevCounters::built_k / inserted_k), so the one read of the counters when
  // the level closes gives every launch's share: no copy between launches.
  CacheView cv = c->view(c->defer[0], &c->ctr->defer_n[0]);
  bool ran_unary = false, ran_binary = false;
  const double M = double(c->vecs) * 16.0;
  if (k == 1) {
    ev_begin();
    lsyn_status s = launch_desc(c, cv, nullptr, nullptr, 0, unsigned(c->n_props), lc);
    ++launches;
    if (s != LSYN_OK) return s;
    ev_end(3);
  } else {
    if (lp.uops && lp.u_count) {
      CacheView uv = cv;
      uv.kind = kKindUnary;
      // CMs above 512 bytes (path D): a unary batch (one row, four candidates)
      // streams tens of microseconds of rows, so one id reservation per batch
      // is cheap beside it, while every id a warp leaves unused costs a row
      // move (2 M bytes) when the level closes: reserve exactly the batch's
      // inserts (and no prefetched chunk). The binary kernel's shorter
      // batches keep their chunks: a reservation per batch slowed it more
      // than its holes cost.
      if (c->vecs > 32u) uv.chunk = 1;
      ev_begin();
      e = c->word_bits == 32 ? Kernels<uint32_t>::unary(uv, lp.u_first, lp.u_count, lp.uops, lc)
                             : Kernels<uint64_t>::unary(uv, lp.u_first, lp.u_count, lp.uops, lc);
      ++launches;
      if (e != cudaSuccess) return c->cuda_fail(e, "unary kernel");
      ev_end(0);
      ran_unary = true;
    }
    if (lp.plan.n_splits > 0) {
      CacheView bv = cv;
      bv.kind = kKindBinary;
      ev_begin();
      e = c->word_bits == 32 ? Kernels<uint32_t>::binary(bv, lp.plan, lc) : Kernels<uint64_t>::binary(bv, lp.plan, lc);
      ++launches;
      if (e != cudaSuccess) return c->cuda_fail(e, "binary kernel");
      ev_end(1);
      ran_binary = true;
    }
  }
  // Close the level without a host round trip in the common case: one pass
  // over the deferred candidates (its count is read on the device) and the
  // hole plan + moves are queued behind the level's kernels, then read back
  // with one synchronisation. Candidates deferred again by that pass (rare)
  // are settled by host-driven passes, then the holes they left are closed.
  // List 1 is empty when the level begins (k_level_begin), so the first pass
  // needs no clear.
  auto pass = [&](int from, unsigned n, bool clear) -> lsyn_status {  // list `from` into list 1 - from
    if (clear && (e = cudaMemsetAsync(&c->ctr->defer_n[1 - from], 0, sizeof(unsigned), c->stream)) != cudaSuccess)
      return c->cuda_fail(e, "memset");
    CacheView rv = c->view(c->defer[1 - from], &c->ctr->defer_n[1 - from]);
    rv.early_exit = 0;  // a deferred candidate must be settled even after a solution
    if (c->vecs > 32u) rv.chunk = 1;  // as the unary kernel's (path D)
    ev_begin();
    lsyn_status s = launch_desc(c, rv, c->defer[from], &c->ctr->defer_n[from], n, 0, lc);
    ++launches;
    if (s != LSYN_OK) return s;
    ev_end(2);
    return LSYN_OK;
  };
  auto close_holes = [&]() -> lsyn_status {
    ev_begin();
    e = c->word_bits == 32 ? Kernels<uint32_t>::close_holes(cv, start, c->hole_bits, c->moves, c->move_cap, lc)
                           : Kernels<uint64_t>::close_holes(cv, start, c->hole_bits, c->moves, c->move_cap, lc);
    launches += 3;
    if (e != cudaSuccess) return c->cuda_fail(e, "hole fixup kernels");
    ev_end(3);
    if ((e = take_snap()) != cudaSuccess) return c->cuda_fail(e, "snapshot");
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return c->cuda_fail(e, "level sync");
    return LSYN_OK;
  };
  lsyn_status ls = pass(0, c->defer_cap, false);
  if (ls != LSYN_OK) return ls;
  if ((ls = close_holes()) != LSYN_OK) return ls;
  // the pass reads list 0 and leaves its count as the level's kernels wrote it
  unsigned long long deferred = std::min(c->h_snap[snap - 1].c.defer_n[0], c->defer_cap);
  int cur = 1;
  for (int npass = 1;; ++npass) {
    const DevCounters& h = c->h_snap[snap - 1].c;
    if (h.timed_out) break;  // reported below
    if (h.defer_overflow) return c->fail(LSYN_E_STATE, "deferred list overflow: the level is not exact");
    if (h.error == 1) return c->fail(LSYN_E_STATE, "hash table probe overflow");
    if (h.error) break;  // reported below
    const unsigned n = std::min(h.defer_n[cur], c->defer_cap);
    if (n == 0) break;
    if (npass >= 48) return c->fail(LSYN_E_STATE, "deferred candidates did not settle");
    deferred += n;
    if ((ls = pass(cur, n, true)) != LSYN_OK) return ls;
    cur = 1 - cur;
    if ((e = take_snap()) != cudaSuccess) return c->cuda_fail(e, "snapshot");
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return c->cuda_fail(e, "resolve sync");
    if (std::min(c->h_snap[snap - 1].c.defer_n[cur], c->defer_cap) == 0 && (ls = close_holes()) != LSYN_OK) return ls;
  }
  const DevCounters& h = c->h_snap[snap - 1].c;
  if (h.timed_out) {
    c->needs_reset = true;  // the level is partial, and its entries are in the cache
    return c->fail(LSYN_E_TIMEOUT, "time limit passed during level " + std::to_string(k) +
                                       ": the level is incomplete; reset the context before using it again");
  }
  if (h.error) {
    static const char* const what[] = {"", "hash table probe overflow", "hole log overflow",
                                       "hole fixup found an inconsistent slot", "inconsistent hole log",
                                       "hash table rebuild overflow", "an operand row copy did not complete"};
    return c->fail(LSYN_E_STATE, std::string("internal consistency check failed: ") +
                                     (h.error < 7 ? what[h.error] : "unknown code"));
  }
  const uint32_t total = std::min(h.n_entries, c->max_entries);
  lsyn_status st = ctx_commit_level(c, k, c->h_snap[snap - 1].c, total, deferred, lp, out);
  if (st != LSYN_OK) return st;
  if (out) {
    out->launches = launches;
    // Per launch, from its exact built / inserted counters: operands, one table
    // sector per candidate, a compare read per duplicate, CM + provenance +
    // slot per insert.
    // a launch that stopped at a solution read its operands only in part: in
    // proportion to the candidates it built
    auto launch_bytes = [&](unsigned kind, double operands, double planned) {
      const double Cl = double(h.built_k[kind]);
      const double Ul = double(h.inserted_k[kind]);
      const double done = planned > 0 ? std::min(1.0, Cl / planned) : 1.0;
      return operands * done + Cl * 32.0 + (Cl - Ul) * M + Ul * (M + 16.0);
    };
    const double planned = double(level_candidate_count(c, k) > 0 ? level_candidate_count(c, k) : 0);
    if (ran_binary) out->bytes_binary = launch_bytes(kKindBinary, lp.op_bytes_binary, planned - lp.cand_unary);
    if (ran_unary) out->bytes_unary = launch_bytes(kKindUnary, lp.op_bytes_unary, lp.cand_unary);
    if (c->timing) {
      for (int i = 0; i < evn; ++i) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, c->ev[2 * i], c->ev[2 * i + 1]) == cudaSuccess) out->kernel_ms[ev_kind[i]] += ms;
      }
    }
    out->ms = now_ms() - t0;
  }
  return LSYN_OK;
}

lsyn_status lsyn_solve(lsyn_ctx* c, int32_t max_size, lsyn_result* out) {
  if (!c || !out) return LSYN_E_INVAL;
  if (c->borrowed) return c->fail(LSYN_E_STATE, "a batch or server problem is driven by its owner");
  if (max_size < 1 || max_size > 64) return c->fail(LSYN_E_INVAL, "max_size must be in 1..64");
  const double t0 = now_ms();
  out->found = 0;
  out->size = 0;
  out->exact = 0;
  out->launches = 0;
  lsyn_status result = LSYN_NOT_FOUND;
  const int first_k = c->levels_done + 1;
  for (int k = first_k; k <= max_size; ++k) {
    // the first level of the call always runs to its end; the later ones get
    // what is left of the limit as their budget inside the kernels
    c->solve_deadline_ms = c->time_limit_ms > 0 && k > first_k ? t0 + c->time_limit_ms : 0;
    // the deadline is checked between levels: the first level of the call always runs
    if (c->time_limit_ms > 0 && k > first_k && now_ms() - t0 >= c->time_limit_ms) {
      c->err = "time limit of " + std::to_string(c->time_limit_ms) + " ms passed before level " + std::to_string(k);
      result = LSYN_E_TIMEOUT;
      break;
    }
    lsyn_level_stats st;
    lsyn_status s = lsyn_enumerate_level(c, k, &st);
    if (s != LSYN_OK) { result = s; break; }
    out->launches += st.launches;
    if (out->level_stats && k <= out->level_stats_cap) out->level_stats[k - 1] = st;
    if (st.solved) {
      out->launches += 1;
      s = ctx_reconstruct(c, &c->ctr->sol, out->formula, out->formula_cap);
      if (s != LSYN_OK) { result = s; break; }
      out->found = 1;
      out->size = k;
      out->exact = 1;
      result = LSYN_OK;
      break;
    }
    if (st.cache_full) {
      c->err = "language cache full at level " + std::to_string(k);
      result = LSYN_E_CACHE_FULL;
      break;
    }
  }
  c->solve_deadline_ms = 0;
  c->level_budget_ns = 0;
  // a solve that ended on the front table: the big table's clear joins the
  // caller's stream here, so that the solve's stream order covers it
  if (c->big_clear_pending && cudaStreamWaitEvent(c->stream, c->ev_side[1], 0) == cudaSuccess)
    c->big_clear_pending = false;
  out->levels_done = c->levels_done;
  out->constructed = int64_t(c->constructed);
  out->unique = int64_t(c->level_start.back() + c->level_n.back());
  out->ms = now_ms() - t0;
  return result;
}

lsyn_status lsyn_level_count(const lsyn_ctx* c, int32_t k, int64_t* n_out) {
  if (!c || !n_out || k < 1 || k > c->levels_done) return LSYN_E_INVAL;
  *n_out = c->level_n[k];
  return LSYN_OK;
}

lsyn_status lsyn_export_level(lsyn_ctx* c, int32_t k, int64_t first, int64_t count, void* dst, size_t cap) {
  if (!c || k < 1 || k > c->levels_done || first < 0 || count < 0) return LSYN_E_INVAL;
  if (uint64_t(first) + uint64_t(count) > c->level_n[k]) return c->fail(LSYN_E_INVAL, "range outside the level");
  const size_t wbytes = size_t(c->word_bits / 8);
  const size_t row = size_t(c->T) * size_t(c->planes) * wbytes;
  if (count == 0) return LSYN_OK;
  if (!dst || cap < row * size_t(count)) return c->fail(LSYN_E_INVAL, "destination too small");
  cudaSetDevice(c->device);
  const uint4* src = c->arena + (size_t(c->level_start[k]) + size_t(first)) * c->vecs;
  cudaError_t e;
  if (c->planes == 1) {
    e = cudaMemcpy2DAsync(dst, row, src, size_t(c->vecs) * 16, row, size_t(count), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return c->cuda_fail(e, "export");
    reverse_words(dst, size_t(count) * size_t(c->T), c->word_bits);  // back to bit t = position t
    return LSYN_OK;
  }
  // several words per trace: whole rows, then [trace][plane] words per row
  std::vector<uint8_t> tmp(size_t(count) * size_t(c->vecs) * 16);
  e = cudaMemcpyAsync(tmp.data(), src, tmp.size(), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return c->cuda_fail(e, "export");
  for (int64_t r = 0; r < count; ++r)
    planes_to_abi(tmp.data() + size_t(r) * c->vecs * 16, static_cast<uint8_t*>(dst) + size_t(r) * row, c->T,
                  int(c->planes), c->plane_vecs, c->word_bits);
  return LSYN_OK;
}

lsyn_status lsyn_entry_formula(lsyn_ctx* c, int32_t k, int64_t index, char* buf, size_t cap) {
  if (!c || k < 1 || k > c->levels_done || index < 0 || uint64_t(index) >= c->level_n[k]) return LSYN_E_INVAL;
  cudaSetDevice(c->device);
  return ctx_reconstruct(c, c->prov + c->level_start[k] + size_t(index), buf, cap);
}

lsyn_status lsyn_eval(const lsyn_problem* problem, const char* formula, void* dst, const lsyn_config* config) {
  g_create_error.clear();
  Layout L;
  lsyn_status s = validate(problem, &L, &g_create_error);
  if (s != LSYN_OK) return s;
  if (!formula || !dst) { g_create_error = "formula and dst are required"; return LSYN_E_INVAL; }
  std::vector<int4> nodes;
  if (!parse_formula(formula, problem->n_props, &nodes, &g_create_error)) return LSYN_E_INVAL;
  lsyn_config cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.device = -1;
  if (config) cfg = *config;
  if (cfg.device >= 0 && cudaSetDevice(cfg.device) != cudaSuccess) { g_create_error = "bad device"; return LSYN_E_CUDA; }
  cudaStream_t stream = static_cast<cudaStream_t>(cfg.stream);
  const unsigned plane_vecs = std::max(1u, L.plane_vecs_needed);
  const unsigned vecs = plane_vecs * unsigned(L.planes);
  const size_t M = size_t(vecs) * 16;
  std::vector<uint32_t> consts, atoms;
  pack_host(problem, L, vecs, plane_vecs, &consts, &atoms);
  Alloc mem;
  mem.alloc = cfg.alloc;
  mem.free = cfg.free;
  mem.user = cfg.alloc_user;
  uint4* d_lm = static_cast<uint4*>(mem.get(M));
  uint4* d_atoms = static_cast<uint4*>(mem.get(size_t(problem->n_props) * M));
  int4* d_nodes = static_cast<int4*>(mem.get(nodes.size() * sizeof(int4)));
  uint4* d_scratch = static_cast<uint4*>(mem.get(nodes.size() * M));
  uint4* d_out = static_cast<uint4*>(mem.get(M));
  if (!d_lm || !d_atoms || !d_nodes || !d_scratch || !d_out) {
    mem.release_all();
    g_create_error = "device allocation failed";
    return LSYN_E_NOMEM;
  }
  std::vector<uint8_t> host_out(M);
  LaunchCfg lc{stream, 1};
  cudaError_t e = cudaMemcpyAsync(d_lm, consts.data(), M, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_atoms, atoms.data(), atoms.size() * 4, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_nodes, nodes.data(), nodes.size() * sizeof(int4), cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) {
    if (L.word_bits == 32)
      e = Kernels<uint32_t>::eval(d_atoms, d_lm, plane_vecs, unsigned(L.planes), d_nodes, int(nodes.size()), L.steps,
                                  reinterpret_cast<uint32_t*>(d_scratch), reinterpret_cast<uint32_t*>(d_out), lc);
    else
      e = Kernels<uint64_t>::eval(d_atoms, d_lm, plane_vecs, unsigned(L.planes), d_nodes, int(nodes.size()), L.steps,
                                  reinterpret_cast<uint64_t*>(d_scratch), reinterpret_cast<uint64_t*>(d_out), lc);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(host_out.data(), d_out, M, cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  mem.release_all();
  if (e != cudaSuccess) {
    g_create_error = std::string("eval: ") + cudaGetErrorString(e);
    return LSYN_E_CUDA;
  }
  // back to the ABI's [trace][plane] words with bit t = position t
  planes_to_abi(host_out.data(), static_cast<uint8_t*>(dst), L.T, L.planes, plane_vecs, L.word_bits);
  return LSYN_OK;
}

}  // extern "C"
