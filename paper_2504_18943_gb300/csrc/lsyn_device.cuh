// Device code of the LTLf semantic enumerator: bitwise LTLf operators on
// characteristic-matrix words, the candidate hash, the specification check,
// the lock-free dedup-insert into the device-resident language cache, and the
// level kernels. Included once per word type by kernels_w32.cu / kernels_w64.cu
// with LSYN_WORD defined.
//
// Layout. A characteristic matrix (CM) is one word per trace, positives first,
// padded with zero words to `vecs` 16-byte vectors; a word holds a trace's
// characteristic sequence ("Parallel enumeration of LTLf formulae on GPUs"),
// position 0 in the most significant bit. Traces longer than a word take one
// word per "plane": plane j holds positions [j w, (j + 1) w) of every trace and
// occupies `plane_vecs` vectors. Padding bits (positions >= length, padding
// traces) are zero for every formula.
#pragma once

#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>

#include "lsyn_internal.h"

namespace lsyn {

constexpr unsigned kFull = 0xFFFFFFFFu;

template <typename W> struct WordInfo;
template <> struct WordInfo<uint32_t> { static constexpr int kMaxSteps = 5; };
template <> struct WordInfo<uint64_t> { static constexpr int kMaxSteps = 6; };

// ---------------------------------------------------------------------------
// Operators on one trace word ("Logical operations as bitwise operations").
// Inside the library a characteristic sequence is stored most significant bit
// first, as the paper writes it: position 0 is the top bit, position t is bit
// (word_bits - 1 - t), so "position t + 1" is the next lower bit and positions
// at or beyond the trace's end are the low padding bits, always 0.
//
// The enumeration kernels use these forms (w_op):
//   not : ~a & lenmask
//   X   : a << 1                        (position t takes position t + 1)
//   F   : -(a & -a)                     (every bit from the lowest set bit up:
//                                        "holds at t or at some later position")
//   G   : not F not, masked to the trace length
//   U   : B | (A & ((A|B) + B  ^  (A & ~B)))   with A = phi, B = psi.
// F and U are suffix scans computed by the integer adder's carry chain: in
// (A|B) + B a carry is generated where B holds and propagated where A holds, so
// the carry into bit j says "psi at some later position with phi on every
// position in between", and U_j = B_j | (A_j & carry_j).
//
// The formula evaluator (w_op_logstep) uses the paper's log-step forms instead:
//   F: a |= a << s for s = 1, 2, 4, ...; U: R |= A & (R << s); A &= A << s
// (R starts as psi, A as phi; R uses the old A). Both are checked against the
// CPU oracle, so each formulation checks the other.
// ---------------------------------------------------------------------------
template <typename W>
__device__ __forceinline__ W w_future(W a) {
  return W(0) - (a & (W(0) - a));
}

template <typename W>
__device__ __forceinline__ W w_until(W phi, W psi) {
  const W cin = ((phi | psi) + psi) ^ (phi & ~psi);
  return psi | (phi & cin);
}

template <typename W>
__device__ __forceinline__ W w_op(uint32_t op, W a, W b, W lm, int /*steps*/) {
  switch (op) {
    case kNot: return ~a & lm;
    case kAnd: return a & b;
    case kOr: return a | b;
    case kNext: return a << 1;
    case kFuture: return w_future<W>(a);
    case kGlobally: return ~w_future<W>(~a & lm) & lm;
    case kUntil: return w_until<W>(a, b);
    default: return W(0);
  }
}

// ---------------------------------------------------------------------------
// Traces longer than a word (planes). The operators carry one word of
// information from the later planes of the same trace:
//   X: the last position of plane j takes the first position of plane j + 1;
//   F: every position of plane j holds if any later plane has a set bit;
//   U: U at the first position of plane j + 1 enters plane j's adder as a
//      carry-in (a psi just after the word's last position), so U is computed
//      from the last plane to the first.
// Positions past a trace's end are 0 in every plane, so no carry crosses it.
// ---------------------------------------------------------------------------
template <typename W>
__device__ __forceinline__ W w_top(W a) {  // the position-0 bit as 0 / 1
  return a >> (sizeof(W) * 8 - 1);
}

template <typename W>
__device__ __forceinline__ W w_until_cin(W phi, W psi, W cin) {
  const W c = ((phi | psi) + psi + cin) ^ (phi & ~psi);
  return psi | (phi & c);
}

// The words of one 16-byte vector.
template <typename W>
struct Words;
template <>
struct Words<uint32_t> {
  static constexpr int N = 4;
  uint32_t w[4];
  __device__ static Words load(uint4 v) { return Words{{v.x, v.y, v.z, v.w}}; }
  __device__ uint4 store() const { return make_uint4(w[0], w[1], w[2], w[3]); }
};
template <>
struct Words<uint64_t> {
  static constexpr int N = 2;
  uint64_t w[2];
  __device__ static Words load(uint4 v) {
    return Words{{uint64_t(v.x) | (uint64_t(v.y) << 32), uint64_t(v.z) | (uint64_t(v.w) << 32)}};
  }
  __device__ uint4 store() const {
    return make_uint4(uint32_t(w[0]), uint32_t(w[0] >> 32), uint32_t(w[1]), uint32_t(w[1] >> 32));
  }
};

// Vector u of plane j of op(a, b) on multi-plane rows: A(k), B(k), LM(k) give
// vector u of plane k of the operands and of the length masks.
template <typename W, class FA, class FB, class FL>
__device__ uint4 mp_op(uint32_t op, unsigned j, unsigned planes, const FA& A, const FB& B, const FL& LM) {
  using V = Words<W>;
  switch (op) {
    case kNot: {
      V a = V::load(A(j));
      const V m = V::load(LM(j));
#pragma unroll
      for (int i = 0; i < V::N; ++i) a.w[i] = ~a.w[i] & m.w[i];
      return a.store();
    }
    case kAnd: {
      const uint4 a = A(j), b = B(j);
      return make_uint4(a.x & b.x, a.y & b.y, a.z & b.z, a.w & b.w);
    }
    case kOr: {
      const uint4 a = A(j), b = B(j);
      return make_uint4(a.x | b.x, a.y | b.y, a.z | b.z, a.w | b.w);
    }
    case kNext: {
      V a = V::load(A(j));
      const V n = j + 1 < planes ? V::load(A(j + 1)) : V::load(make_uint4(0, 0, 0, 0));
#pragma unroll
      for (int i = 0; i < V::N; ++i) a.w[i] = (a.w[i] << 1) | w_top<W>(n.w[i]);
      return a.store();
    }
    case kFuture:
    case kGlobally: {
      const bool g = op == kGlobally;  // G = not F not, negation masked to the trace
      V later = V::load(make_uint4(0, 0, 0, 0));
      for (int k = int(planes) - 1; k > int(j); --k) {
        V x = V::load(A(unsigned(k)));
        if (g) {
          const V m = V::load(LM(unsigned(k)));
#pragma unroll
          for (int i = 0; i < V::N; ++i) x.w[i] = ~x.w[i] & m.w[i];
        }
#pragma unroll
        for (int i = 0; i < V::N; ++i) later.w[i] |= x.w[i];
      }
      V x = V::load(A(j));
      const V m = V::load(LM(j));
#pragma unroll
      for (int i = 0; i < V::N; ++i) {
        const W xi = g ? (~x.w[i] & m.w[i]) : x.w[i];
        const W f = w_future<W>(xi) | (later.w[i] ? m.w[i] : W(0));
        x.w[i] = g ? (~f & m.w[i]) : f;
      }
      return x.store();
    }
    case kUntil: {
      V c = V::load(make_uint4(0, 0, 0, 0)), r = c;
      for (int k = int(planes) - 1; k >= int(j); --k) {
        const V phi = V::load(A(unsigned(k))), psi = V::load(B(unsigned(k)));
#pragma unroll
        for (int i = 0; i < V::N; ++i) {
          r.w[i] = w_until_cin<W>(phi.w[i], psi.w[i], c.w[i]);
          c.w[i] = w_top<W>(r.w[i]);
        }
      }
      return r.store();
    }
    default:
      return make_uint4(0, 0, 0, 0);
  }
}

// `steps` is the smallest s with 2^s >= the longest trace.
template <typename W>
__device__ __forceinline__ W w_future_logstep(W a, int steps) {
#pragma unroll
  for (int s = 0; s < WordInfo<W>::kMaxSteps; ++s)
    if (s < steps) a |= a << (1u << s);
  return a;
}

template <typename W>
__device__ __forceinline__ W w_until_logstep(W phi, W psi, int steps) {
  W r = psi;
#pragma unroll
  for (int s = 0; s < WordInfo<W>::kMaxSteps; ++s) {
    if (s < steps) {
      const unsigned sh = 1u << s;
      r |= phi & (r << sh);
      phi &= phi << sh;
    }
  }
  return r;
}

template <typename W>
__device__ __forceinline__ W w_op_logstep(uint32_t op, W a, W b, W lm, int steps) {
  switch (op) {
    case kNot: return ~a & lm;
    case kAnd: return a & b;
    case kOr: return a | b;
    case kNext: return a << 1;
    case kFuture: return w_future_logstep<W>(a, steps);
    case kGlobally: return ~w_future_logstep<W>(~a & lm, steps) & lm;
    case kUntil: return w_until_logstep<W>(a, b, steps);
    default: return W(0);
  }
}

__device__ __forceinline__ uint64_t lo64(uint4 v) { return uint64_t(v.x) | (uint64_t(v.y) << 32); }
__device__ __forceinline__ uint64_t hi64(uint4 v) { return uint64_t(v.z) | (uint64_t(v.w) << 32); }
__device__ __forceinline__ uint4 make4(uint64_t a, uint64_t b) {
  return make_uint4(uint32_t(a), uint32_t(a >> 32), uint32_t(b), uint32_t(b >> 32));
}

// The operator applied to every word of a 16-byte vector.
template <typename W>
__device__ __forceinline__ uint4 v_op(uint32_t op, uint4 a, uint4 b, uint4 lm, int steps);

template <>
__device__ __forceinline__ uint4 v_op<uint32_t>(uint32_t op, uint4 a, uint4 b, uint4 lm, int steps) {
  return make_uint4(w_op<uint32_t>(op, a.x, b.x, lm.x, steps), w_op<uint32_t>(op, a.y, b.y, lm.y, steps),
                    w_op<uint32_t>(op, a.z, b.z, lm.z, steps), w_op<uint32_t>(op, a.w, b.w, lm.w, steps));
}

template <>
__device__ __forceinline__ uint4 v_op<uint64_t>(uint32_t op, uint4 a, uint4 b, uint4 lm, int steps) {
  return make4(w_op<uint64_t>(op, lo64(a), lo64(b), lo64(lm), steps),
               w_op<uint64_t>(op, hi64(a), hi64(b), hi64(lm), steps));
}

// Vector v of op(row a, row b) of a CM in global memory, planes or not.
template <typename W>
__device__ __forceinline__ uint4 row_op(const CacheView& cv, uint32_t op, const uint4* a, const uint4* b, unsigned v) {
  if (cv.planes <= 1) return v_op<W>(op, __ldg(a + v), __ldg(b + v), __ldg(cv.lenmask + v), 0);
  const unsigned pv = cv.plane_vecs, j = v / pv, u = v - j * pv;
  if (j >= cv.planes) return make_uint4(0, 0, 0, 0);  // padding vectors after the last plane
  return mp_op<W>(op, j, cv.planes, [&](unsigned k) { return __ldg(a + k * pv + u); },
                  [&](unsigned k) { return __ldg(b + k * pv + u); },
                  [&](unsigned k) { return __ldg(cv.lenmask + k * pv + u); });
}


// ---------------------------------------------------------------------------
// Hash of a CM: over its 32-bit words w_i, H = (sum hi32(p_i), sum lo32(p_i))
// mod 2^32 with p_i = (w_i xor key_i) * mul_i as a 64-bit product, then a
// 64-bit finaliser. The low bits index the table, the high 32 bits are the
// slot tag. Equal CMs always hash equally; collisions only cost a compare.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void h_acc(uint4 v, uint4 key, uint4 mul, uint32_t& lo, uint32_t& hi) {
  uint64_t p;
  p = uint64_t(v.x ^ key.x) * mul.x; lo += uint32_t(p); hi += uint32_t(p >> 32);
  p = uint64_t(v.y ^ key.y) * mul.y; lo += uint32_t(p); hi += uint32_t(p >> 32);
  p = uint64_t(v.z ^ key.z) * mul.z; lo += uint32_t(p); hi += uint32_t(p >> 32);
  p = uint64_t(v.w ^ key.w) * mul.w; lo += uint32_t(p); hi += uint32_t(p >> 32);
}

// Warp-path variant of the hash: acc += w_i * mul_i (64-bit products and sum)
// per 32-bit word, then the two 32-bit halves are summed across the warp and
// finalised with h_fin. Equal CMs hash equally; that is all dedup needs.
__device__ __forceinline__ uint64_t h_mac(uint4 v, uint4 mul, uint64_t acc) {
  acc += uint64_t(v.x) * mul.x;
  acc += uint64_t(v.y) * mul.y;
  acc += uint64_t(v.z) * mul.z;
  acc += uint64_t(v.w) * mul.w;
  return acc;
}

__device__ __forceinline__ uint64_t h_fin(uint32_t hi, uint32_t lo) {
  uint64_t x = (uint64_t(hi) << 32) | lo;
  x ^= x >> 31;
  x *= 0xBF58476D1CE4E5B9ull;
  x ^= x >> 29;
  x *= 0x94D049BB133111EBull;
  x ^= x >> 32;
  return x;
}

// Specification check (section "Synthesising linear temporal logic formulae
// from examples", separation): the position-0 bit of every real trace word must
// equal its label (1 for P, 0 for N); `lab` and `care` hold that bit only.
// Returns nonzero on a mismatch in this vector.
__device__ __forceinline__ uint32_t spec_bad(uint4 c, uint4 lab, uint4 care) {
  return ((c.x ^ lab.x) & care.x) | ((c.y ^ lab.y) & care.y) | ((c.z ^ lab.z) & care.z) |
         ((c.w ^ lab.w) & care.w);
}

__device__ __forceinline__ uint32_t v_ne(uint4 a, uint4 b) {
  return (a.x ^ b.x) | (a.y ^ b.y) | (a.z ^ b.z) | (a.w ^ b.w);
}

__device__ __forceinline__ void st_release(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long cas_acquire(unsigned long long* p, unsigned long long cmp,
                                                          unsigned long long val) {
  unsigned long long old;
  asm volatile("atom.acquire.gpu.global.cas.b64 %0, [%1], %2, %3;" : "=l"(old) : "l"(p), "l"(cmp), "l"(val) : "memory");
  return old;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// One probe of a table slot: returns what is there, after claiming the slot
// with `val` if it was empty (then 0). The slot is read first and claimed with
// a compare-and-swap only when it reads empty: most probes meet an occupied
// slot (an equal CM, or another tag), and on this GPU a random load costs far
// less than a random atomic (whole solves 1.45x faster than one CAS per probe).
// A claim that loses a race returns the winner's value, as the CAS alone
// would. Acquire semantics (load and CAS): when the value is a published id,
// the writer's release (fence.acq_rel.gpu, then a relaxed store of the slot)
// synchronises with this read, so the entry's CM row, stored before the
// release, is visible to this thread's later reads, and, after a warp
// barrier, to its warp's.
__device__ __forceinline__ unsigned long long probe_slot(unsigned long long* p, unsigned long long val) {
  const unsigned long long sv = ld_acquire_u64(p);
  return sv != 0ull ? sv : cas_acquire(p, 0ull, val);
}

__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Polled by the level kernels every few batches (once per tile): a solution
// was found (with early exit), or the level's time budget is spent.
__device__ __forceinline__ bool stop_requested(const CacheView& cv) {
  if (cv.early_exit && ld_relaxed_u32(&cv.ctr->solved) != 0u) return true;
  if (cv.time_budget_ns && global_ns() - cv.ctr->t0 > cv.time_budget_ns) {
    cv.ctr->timed_out = 1u;
    return true;
  }
  return false;
}

__device__ __forceinline__ void record_solution(const CacheView& cv, uint64_t desc) {
  atomicMin(&cv.ctr->sol, (unsigned long long)desc);
  atomicExch(&cv.ctr->solved, 1u);
}

// A candidate that met a claimed but unpublished slot with its own tag cannot
// be compared yet: it is re-examined by a later pass over the deferred list.
__device__ __forceinline__ void defer(const CacheView& cv, uint64_t desc) {
  const unsigned idx = atomicAdd(cv.defer_out_n, 1u);
  if (idx < cv.defer_cap) cv.defer_out[idx] = desc;
  else atomicExch(&cv.ctr->defer_overflow, 1u);
}

__device__ __forceinline__ const uint4* row_ptr(const CacheView& cv, uint32_t id) {
  return cv.arena + size_t(id) * cv.vecs;
}

// Pair `local` of a split, as row offsets (left, right). For a level paired
// with itself: the pairs a < b in order of b (b = 1, 2, ...; a = 0 .. b-1), so
// that no pair index is wasted. Otherwise, with large_outer, the right
// (larger) side's rows in order, each with every row of the left (smaller)
// side: each large row is read once while the small side stays in L2, which
// made 16 KiB CMs (path D) 15 % faster at the large workload's level 8 than
// the left-major order; without it, row-major over left x right, which
// measured faster for CMs of up to 128 bytes (path A), whose levels L2 holds
// anyway.
__device__ __forceinline__ uint2 split_pair(const Split& S, unsigned long long local, bool large_outer) {
  if (!S.tri) {
    if (large_outer) {
      const uint32_t ib = uint32_t(local / S.left_n);
      return make_uint2(uint32_t(local - (unsigned long long)ib * S.left_n), ib);
    }
    const uint32_t ia = uint32_t(local / S.right_n);
    return make_uint2(ia, uint32_t(local - (unsigned long long)ia * S.right_n));
  }
  unsigned long long b = (unsigned long long)((1.0 + sqrt(1.0 + 8.0 * double(local))) * 0.5);
  while (b > 1 && b * (b - 1) / 2 > local) --b;
  while ((b + 1) * b / 2 <= local) ++b;
  return make_uint2(uint32_t(local - b * (b - 1) / 2), uint32_t(b));
}

// ===========================================================================
// Path A: one thread holds a whole CM (V vectors, at most 128 bytes).
// ===========================================================================
template <typename W, int V>
struct PathA {
  struct Consts {
    uint4 lm[V], lab[V], care[V], key[V], mul[V];
  };

  __device__ static void load_consts(const CacheView& cv, Consts* s) {
    for (int i = threadIdx.x; i < V; i += blockDim.x) {
      s->lm[i] = cv.lenmask[i];
      s->lab[i] = cv.label[i];
      s->care[i] = cv.care[i];
      s->key[i] = cv.hkey[i];
      s->mul[i] = cv.hmul[i];
    }
  }

  __device__ static void load_row(const uint4* p, uint4 (&x)[V]) {
#pragma unroll
    for (int v = 0; v < V; ++v) x[v] = __ldg(p + v);
  }

  // Spec check, then probe / compare / insert one candidate.
  // `full`: the arena is full, so only the spec check is done (see path C).
  __device__ static unsigned process(const CacheView& cv, const Consts& s, const uint4 (&c)[V], uint64_t desc,
                                     bool full) {
    uint32_t lo = 0, hi = 0, bad = 0;
#pragma unroll
    for (int v = 0; v < V; ++v) {
      h_acc(c[v], s.key[v], s.mul[v], lo, hi);
      bad |= spec_bad(c[v], s.lab[v], s.care[v]);
    }
    if (bad == 0) record_solution(cv, desc);
    if (full) return 0;
    const uint64_t h = h_fin(hi, lo);
    const unsigned long long tag = (h >> 32) << 32;
    unsigned long long pos = h & cv.table_mask;
    for (unsigned long long it = 0; it <= cv.table_mask; ++it, pos = (pos + 1) & cv.table_mask) {
      unsigned long long* slot = cv.table + pos;
      // Claims an empty slot, or returns what is there.
      const unsigned long long sv = probe_slot(slot, tag | kSlotPending);
      if (sv == 0ull) {
        const unsigned id = atomicAdd(&cv.ctr->n_entries, 1u);
        if (id >= cv.max_entries) {
          st_release(slot, tag | kSlotTomb);
          atomicExch(&cv.ctr->full, 1u);
          return 0;
        }
        uint4* dst = cv.arena + size_t(id) * cv.vecs;
#pragma unroll
        for (int v = 0; v < V; ++v) dst[v] = c[v];
        cv.prov[id] = desc;
        cv.slotpos[id] = unsigned(pos);
        cv.homes[id] = uint32_t(h);
        st_release(slot, tag | (unsigned long long)(id + 1u));  // orders this thread's CM and provenance first
        return 1;
      }
      // A tombstone is left only by a claim past a full arena, and such a
      // level is incomplete: the candidate could not be inserted any more,
      // so probing stops (a small table full of tombstones would otherwise
      // leave it nowhere to stop).
      if (uint32_t(sv) == kSlotTomb) return 0;
      if ((sv & 0xFFFFFFFF00000000ull) != tag) continue;
      const uint32_t low = uint32_t(sv);
      if (low == kSlotPending) { defer(cv, desc); return 0; }
      const uint4* src = row_ptr(cv, low - 1u);
      uint32_t ne = 0;
#pragma unroll
      for (int v = 0; v < V; ++v) ne |= v_ne(__ldcg(src + v), c[v]);
      if (ne == 0) return 0;  // duplicate: an equal CM is already cached
    }
    atomicExch(&cv.ctr->error, 1u);
    return 0;
  }

  __device__ static unsigned candidate(const CacheView& cv, const Consts& s, uint32_t op, const uint4 (&a)[V],
                                       const uint4 (&b)[V], uint64_t desc, bool full) {
    uint4 c[V];
#pragma unroll
    for (int v = 0; v < V; ++v) c[v] = v_op<W>(op, a[v], b[v], s.lm[v], cv.steps);
    return process(cv, s, c, desc, full);
  }
};

template <typename W, int V>
__global__ void __launch_bounds__(256) k_unary_a(CacheView cv, uint32_t first, uint32_t count, uint32_t ops) {
  using P = PathA<W, V>;
  __shared__ typename P::Consts s;
  P::load_consts(cv, &s);
  __syncthreads();
  unsigned long long built = 0, ins = 0;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
    if (stop_requested(cv)) break;
    const bool full = ld_relaxed_u32(&cv.ctr->full) != 0u;
    const uint32_t id = first + i;
    uint4 a[V];
    P::load_row(row_ptr(cv, id), a);
    const uint32_t opc[4] = {kNot, kNext, kFuture, kGlobally};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (!((ops >> q) & 1u)) continue;
      ins += P::candidate(cv, s, opc[q], a, a, pack_desc(opc[q], id, 0), full);
      ++built;
    }
  }
  if (built) atomicAdd(&cv.ctr->built_k[cv.kind], built);
  if (ins) atomicAdd(&cv.ctr->inserted_k[cv.kind], ins);
}

template <typename W, int V>
__global__ void __launch_bounds__(256) k_binary_a(CacheView cv, BinaryPlan plan) {
  using P = PathA<W, V>;
  __shared__ typename P::Consts s;
  P::load_consts(cv, &s);
  __syncthreads();
  unsigned long long built = 0, ins = 0;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long p = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; p < plan.total_pairs;
       p += stride) {
    if (stop_requested(cv)) break;
    int sp = 0;
    while (sp + 1 < plan.n_splits && plan.s[sp + 1].pairs_begin <= p) ++sp;
    const Split& S = plan.s[sp];
    const uint2 ab = split_pair(S, p - S.pairs_begin, false);
    const uint32_t a_id = S.left_start + ab.x, b_id = S.right_start + ab.y;
    const bool full = ld_relaxed_u32(&cv.ctr->full) != 0u;
    uint4 a[V], b[V];
    P::load_row(row_ptr(cv, a_id), a);
    P::load_row(row_ptr(cv, b_id), b);
    if (plan.ops & 1u) { ins += P::candidate(cv, s, kAnd, a, b, pack_desc(kAnd, a_id, b_id), full); ++built; }
    if (plan.ops & 2u) { ins += P::candidate(cv, s, kOr, a, b, pack_desc(kOr, a_id, b_id), full); ++built; }
    if (plan.ops & 4u) { ins += P::candidate(cv, s, kUntil, a, b, pack_desc(kUntil, a_id, b_id), full); ++built; }
    if (plan.ops & 8u) { ins += P::candidate(cv, s, kUntil, b, a, pack_desc(kUntil, b_id, a_id), full); ++built; }
  }
  if (built) atomicAdd(&cv.ctr->built_k[cv.kind], built);
  if (ins) atomicAdd(&cv.ctr->inserted_k[cv.kind], ins);
}

// Rebuild a candidate from its descriptor (operands are complete levels).
template <typename W, int V>
__device__ void rebuild_a(const CacheView& cv, const typename PathA<W, V>::Consts& s, uint64_t d, uint4 (&c)[V]) {
  const uint32_t op = desc_op(d);
  uint4 a[V], b[V];
  if (op == kAtom) {
    PathA<W, V>::load_row(cv.atoms + size_t(desc_left(d)) * cv.vecs, c);
    return;
  }
  PathA<W, V>::load_row(row_ptr(cv, desc_left(d)), a);
  if (op == kAnd || op == kOr || op == kUntil) PathA<W, V>::load_row(row_ptr(cv, desc_right(d)), b);
  else {
#pragma unroll
    for (int v = 0; v < V; ++v) b[v] = a[v];
  }
#pragma unroll
  for (int v = 0; v < V; ++v) c[v] = v_op<W>(op, a[v], b[v], s.lm[v], cv.steps);
}

template <typename W, int V>
__global__ void __launch_bounds__(256) k_desc_a(CacheView cv, const unsigned long long* list,
                                                const unsigned int* list_n, unsigned int list_cap,
                                                unsigned int implicit_atoms) {
  using P = PathA<W, V>;
  __shared__ typename P::Consts s;
  P::load_consts(cv, &s);
  __syncthreads();
  unsigned n = implicit_atoms;
  if (list) n = min(*list_n, list_cap);
  const uint32_t stride = gridDim.x * blockDim.x;
  unsigned long long ins = 0;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    if (stop_requested(cv)) break;
    const uint64_t d = list ? list[i] : pack_desc(kAtom, i, 0);
    uint4 c[V];
    rebuild_a<W, V>(cv, s, d, c);
    ins += P::process(cv, s, c, d, ld_relaxed_u32(&cv.ctr->full) != 0u);
  }
  if (ins) atomicAdd(&cv.ctr->inserted_k[cv.kind], ins);
  if (implicit_atoms && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&cv.ctr->built_k[cv.kind], (unsigned long long)n);
}

// ===========================================================================
// Warp paths (C and D): a warp holds a CM, lane l holds vectors l, l + 32, ...
// ===========================================================================
__device__ __forceinline__ void cp_async16(uint4* smem, const uint4* gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Bulk copies of whole rows into shared memory (the TMA unit's non-tensor
// form), completed on a per-warp mbarrier: lane 0 arms the barrier with the
// bytes to expect and issues the copies; every lane then waits on the
// barrier's phase. Addresses are 16-byte aligned and sizes multiples of 16.
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0u;
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
// Orders this thread's earlier shared-memory accesses (and, after a warp
// barrier, its warp's) before later accesses of the async proxy (bulk copies).
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Waits for phase `parity` of the barrier, at most `limit` polls per lane;
// warp-uniform result (false: some lane gave up).
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity, unsigned limit) {
  bool done = false;
  for (unsigned i = 0; i < limit && !done; ++i) done = mbar_try_wait(bar, parity);
  return __all_sync(0xFFFFFFFFu, done);
}

__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

__device__ __forceinline__ void st_relaxed(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint32_t comp(const uint4& v, int i) {
  return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}

// The position-0 bit (the top bit) of every trace word of a vector, packed
// (word j -> bit j).
template <typename W> __device__ __forceinline__ uint32_t bit0s(uint4 c);
template <> __device__ __forceinline__ uint32_t bit0s<uint32_t>(uint4 c) {
  return (c.x >> 31) | ((c.y >> 31) << 1) | ((c.z >> 31) << 2) | ((c.w >> 31) << 3);
}
template <> __device__ __forceinline__ uint32_t bit0s<uint64_t>(uint4 c) { return (c.y >> 31) | ((c.w >> 31) << 1); }

// Warp-batch bookkeeping shared by paths C and D: probe states, pending
// publication of claimed slots, and per-warp id reservations.
struct WarpDedup {
  enum { kProbing = 0, kDone = 1, kClaimed = 2, kDeferred = 3 };

  // Ids this warp reserved from the shared counter and has not used yet:
  // [next, end). Reserving `chunk` ids per counter update keeps the counter
  // cold; what a warp leaves unused when it exits is logged as a hole and
  // filled after the level (Kernels::fixup). With full chunks (32 ids) the
  // next chunk is reserved at the start of a batch whose inserts may need it
  // (`pre`, in lane 0; `pre_ok` is warp-uniform): an atomic round trip is long
  // under load, and this one then overlaps the batch's hashing and probing
  // instead of delaying its inserts.
  struct Ids {
    unsigned next = 0, end = 0;
    unsigned pre = 0;
    bool pre_ok = false;
    unsigned long long inserted = 0;
  };

  // The arena-full flag, polled by every batch: once the arena is full each
  // further claim leaves a tombstone in the table, so warps must stop
  // claiming at once (a flag polled every few batches let the tombstones of
  // a small table fill it). The flag has a cache line of its own.
  __device__ static bool arena_full(const CacheView& cv) {
    return __any_sync(kFull, (threadIdx.x & 31) == 0 && ld_relaxed_u32(&cv.ctr->full) != 0u);
  }

  __device__ static void prefetch(const CacheView& cv, Ids& ids) {
    if (!ids.pre_ok && ids.end - ids.next < 32u && cv.chunk >= 32u) {
      if ((threadIdx.x & 31) == 0) ids.pre = atomicAdd(&cv.ctr->n_entries, cv.chunk);
      ids.pre_ok = true;
    }
  }

  // Ids for a batch's n_claim inserts when the current chunk holds `have`:
  // the first fresh id (warp-uniform) once the chunk runs out; advances `ids`.
  // Claim rank r takes ids.next + r while r < have, then fresh + (r - have).
  __device__ static unsigned take(const Ids& ids, unsigned n_claim, unsigned have, unsigned base, bool use_pre) {
    return n_claim > have ? __shfl_sync(kFull, use_pre ? ids.pre : base, 0) : 0u;
  }
  // Ids reserved on demand for a batch that needs n_claim - have more: a full
  // chunk, or exactly those in a warp's last batch (nothing is left to hole).
  __device__ static unsigned demand(const CacheView& cv, unsigned n_claim, unsigned have, bool last) {
    return last ? n_claim - have : max(cv.chunk, n_claim - have);
  }
  __device__ static void advance(const CacheView& cv, Ids& ids, unsigned n_claim, unsigned have, unsigned fresh,
                                 bool use_pre, bool last = false) {
    if (n_claim > have) {
      ids.next = fresh + (n_claim - have);
      ids.end = fresh + (use_pre ? cv.chunk : demand(cv, n_claim, have, last));
      if (use_pre) ids.pre_ok = false;
    } else {
      ids.next += n_claim;
    }
  }

  __device__ static void log_hole(const CacheView& cv, unsigned lo, unsigned hi) {
    if (lo < hi && lo < cv.max_entries) {
      const unsigned h = atomicAdd(&cv.ctr->holes_n, 1u);
      if (h < cv.hole_cap) cv.holes[h] = make_uint2(lo, min(hi, cv.max_entries));
      else atomicExch(&cv.ctr->error, 2u);
    }
  }

  __device__ static void retire(const CacheView& cv, Ids& ids) {
    const int lane = threadIdx.x & 31;
    if (lane == 0) {
      log_hole(cv, ids.next, ids.end);
      if (ids.pre_ok) log_hole(cv, ids.pre, ids.pre + cv.chunk);
      if (ids.inserted) atomicAdd(&cv.ctr->inserted_k[cv.kind], ids.inserted);
    }
    ids.next = ids.end = 0;
    ids.pre_ok = false;
    ids.inserted = 0;
  }

  // A slot this lane claimed whose CM words were stored but not yet
  // published. It is published by a later batch (or by flush()) after a fence;
  // meanwhile the slot reads as pending and an equal candidate is deferred.
  struct Pending {
    unsigned long long* slot = nullptr;
    unsigned long long val = 0;
  };

  // Publish this warp's pending slots (all lanes call it together). Every
  // lane stored part of each claimed row; the warp barrier orders those
  // stores before the fence, and the fence before the relaxed slot stores,
  // so each slot store is a release of its whole row (and of the owner's
  // provenance words).
  __device__ static void flush(Pending& pend) {
    if (__any_sync(kFull, pend.slot != nullptr)) {
      __syncwarp();
      fence_acq_rel_gpu();
      if (pend.slot) st_relaxed(pend.slot, pend.val);
      pend.slot = nullptr;
    }
  }
};

// Unary operator code of position o in the batch order (not, X, F, G).
__device__ __forceinline__ uint32_t unary_code(int o) { return o == 0 ? kNot : uint32_t(3 + o); }

// ===========================================================================
// Path C (CMs of exactly one 16-byte vector per lane: 32 vectors, 512 bytes for
// 32-bit words): "hash first". A warp batch covers up to 32 candidates, one per
// lane for probing. Candidates are not held while their probes are in flight:
// the generator recomputes candidate q from operands kept in shared memory or
// registers whenever it is needed (hashing, comparing, writing). Registers stay
// few, so more warps fit, and each warp has up to 32 probes and 8 compare
// reads in flight.
// ===========================================================================
template <typename W>
struct PathC {
  static constexpr int WPV = int(16 / sizeof(W));
  static constexpr int kGroup = 8;             // compare reads staged together
  static constexpr int kStage = kGroup * 32;   // uint4 of staging per warp

  using Pending = WarpDedup::Pending;
  using Ids = WarpDedup::Ids;

  struct Consts {
    uint4 mul;     // hash multipliers of this lane's 32-bit words
    uint32_t lab;  // bit j: 1 iff word j of this lane's vector belongs to a positive trace
  };

  __device__ static void load_consts(const CacheView& cv, Consts& k) {
    const int lane = threadIdx.x & 31;
    k.mul = cv.hmul[lane];
    k.lab = bit0s<W>(cv.label[lane]);
  }

  // The first (at most) kGroup set bits of m.
  __device__ static uint32_t first_bits(uint32_t m) {
    uint32_t g = 0;
#pragma unroll
    for (int i = 0; i < kGroup; ++i) {
      const uint32_t b = m & (0u - m);
      g |= b;
      m ^= b;
    }
    return g;
  }

  // gen.compute(q): this lane's vector of candidate q (q warp-uniform);
  // gen.desc(q): descriptor of candidate q. Candidates 0..n-1, bit q of `en`
  // (warp-uniform) says candidate q is real.
  // kEarlyPublish: publish the previous batch's slots before probing (for
  // generators whose consecutive batches share an operand, so that a warp never
  // defers on its own inserts); otherwise after probing, when the fence no
  // longer waits for those stores.
  // last (warp-uniform): the warp's final batch of the launch; it reserves no
  // chunk ahead and takes exactly the ids its inserts need, so that its
  // unused ids (holes, moved at the level's close) stay few.
  template <bool kEarlyPublish, class Gen>
  __device__ static void batch(const CacheView& cv, const Consts& k, const Gen& gen, int n, uint32_t en,
                               uint4* stage, Pending& pend, Ids& ids, bool last = false) {
    const int lane = threadIdx.x & 31;
    if (!last) WarpDedup::prefetch(cv, ids);
    uint32_t my_lo = 0, my_hi = 0, bad = 0;
    for (int q0 = 0; q0 < n; q0 += 4) {  // n is a multiple of 4: four operators per operand group
      uint4 c4[4];
      gen.compute4(q0, c4);
#pragma unroll
      for (int o = 0; o < 4; ++o) {
        const int q = q0 + o;
        const uint64_t acc = h_mac(c4[o], k.mul, 0ull);
        const uint32_t lo = __reduce_add_sync(kFull, uint32_t(acc));
        const uint32_t hi = __reduce_add_sync(kFull, uint32_t(acc >> 32));
        my_lo = lane == q ? lo : my_lo;
        my_hi = lane == q ? hi : my_hi;
        bad |= ((bit0s<W>(c4[o]) ^ k.lab) != 0u ? 1u : 0u) << q;
      }
    }
    // Separation (section "Synthesising ... from examples"): the position-0 bit
    // of every trace word equals the trace's label. Padding words are 0 with
    // label 0.
    bad = __reduce_or_sync(kFull, bad);
    const bool mine = lane < n && ((en >> lane) & 1u);
    const uint64_t my_desc = gen.desc(lane < n ? lane : 0);
    if (mine && !((bad >> lane) & 1u)) record_solution(cv, my_desc);

    // Once the arena is full this level can never be extended: only the spec
    // check (above) matters, so the rest of the batch skips the dedup instead
    // of filling the table with tombstones.
    const bool full = WarpDedup::arena_full(cv);
    int state = (mine && !full) ? WarpDedup::kProbing : WarpDedup::kDone;
    constexpr int kProbing = WarpDedup::kProbing, kDone = WarpDedup::kDone,
                  kClaimed = WarpDedup::kClaimed, kDeferred = WarpDedup::kDeferred;
    const uint64_t h = h_fin(my_hi, my_lo);
    const unsigned long long tag = (h >> 32) << 32;
    unsigned long long pos = h & cv.table_mask;

    // Twins inside the batch (equal hashes; common, since the batch's
    // candidates share an operand): compare each with its lowest-lane twin in
    // registers; an equal one is a duplicate and does not probe.
    const uint32_t mine_mask = __ballot_sync(kFull, mine);
    const uint32_t peers = __match_any_sync(kFull, (unsigned long long)h) & mine_mask;
    const bool has_twin = mine && (peers & ((1u << lane) - 1u)) != 0u;
    const int twin = __ffs(peers) - 1;
    for (uint32_t m = __ballot_sync(kFull, has_twin); m; m &= m - 1u) {
      const int q = __ffs(m) - 1;
      const int p = __shfl_sync(kFull, twin, q);
      const bool eq = !__any_sync(kFull, v_ne(gen.compute(q), gen.compute(p)) != 0u);
      if (lane == q && eq) state = kDone;
    }

    if (kEarlyPublish) WarpDedup::flush(pend);
    uint32_t cmp_id = 0;
    unsigned long long guard = 0;
    while (true) {
      bool need = false;
      if (state == kProbing) {
        // Claims an empty slot, or returns what is there.
        const unsigned long long sv = probe_slot(cv.table + pos, tag | kSlotPending);
        if (sv == 0ull) {
          state = kClaimed;
        } else {
          const uint32_t low = uint32_t(sv);
          if (low == kSlotTomb) state = kDone;  // the arena is full: this level is incomplete (see path A)
          else if ((sv & 0xFFFFFFFF00000000ull) != tag) pos = (pos + 1) & cv.table_mask;
          else if (low == kSlotPending) state = kDeferred;
          else {
            need = true;
            cmp_id = low - 1u;
          }
        }
      }
      uint32_t cm = __ballot_sync(kFull, need);
      if (cm) __syncwarp();  // the probing lanes' acquires, before every lane's row reads
      while (cm) {
        const uint32_t grp = first_bits(cm);
        cm ^= grp;
        // Stage the stored rows (published before their slots; cp.async.cg
        // reads them from L2), then recompute and compare.
        int slot = 0;
        for (uint32_t m = grp; m; m &= m - 1u, ++slot) {
          const int q = __ffs(m) - 1;
          const uint32_t id = __shfl_sync(kFull, cmp_id, q);
          cp_async16(stage + slot * 32 + lane, row_ptr(cv, id) + lane);
        }
        cp_async_wait_all();
        uint32_t ne = 0;
        slot = 0;
        for (uint32_t m = grp; m; m &= m - 1u, ++slot) {
          const int q = __ffs(m) - 1;
          ne |= (v_ne(stage[slot * 32 + lane], gen.compute(q)) != 0u ? 1u : 0u) << q;
        }
        ne = __reduce_or_sync(kFull, ne);
        if ((grp >> lane) & 1u) {
          if (!((ne >> lane) & 1u)) state = kDone;  // equal CM already cached
          else pos = (pos + 1) & cv.table_mask;
        }
      }
      if (!__any_sync(kFull, state == kProbing)) break;
      if (++guard > cv.table_mask) {  // every slot seen: cannot happen at load <= 0.9
        if (lane == 0) atomicExch(&cv.ctr->error, 1u);
        if (state == kProbing) state = kDone;
      }
    }

    const uint32_t claim = __ballot_sync(kFull, state == kClaimed);
    const unsigned n_claim = unsigned(__popc(claim));
    const unsigned have = ids.end - ids.next;  // warp-uniform
    const bool use_pre = n_claim > have && ids.pre_ok;
    unsigned base = 0;
    if (n_claim > have && !use_pre && lane == 0)
      base = atomicAdd(&cv.ctr->n_entries, WarpDedup::demand(cv, n_claim, have, last));
    if (!kEarlyPublish) WarpDedup::flush(pend);  // overlaps the id reservation above
    if (claim) {
      const unsigned fresh = WarpDedup::take(ids, n_claim, have, base, use_pre);
      unsigned rank = 0;
      for (uint32_t m = claim; m; m &= m - 1u, ++rank) {
        const int q = __ffs(m) - 1;
        const unsigned id = rank < have ? ids.next + rank : fresh + (rank - have);
        if (id < cv.max_entries) cv.arena[size_t(id) * cv.vecs + lane] = gen.compute(q);
      }
      const unsigned my_rank = unsigned(__popc(claim & ((1u << lane) - 1u)));
      const unsigned my_id = my_rank < have ? ids.next + my_rank : fresh + (my_rank - have);
      WarpDedup::advance(cv, ids, n_claim, have, fresh, use_pre, last);
      ids.inserted += __popc(__ballot_sync(kFull, state == kClaimed && my_id < cv.max_entries));
      if (state == kClaimed) {
        unsigned long long* slot = cv.table + pos;
        if (my_id < cv.max_entries) {
          cv.prov[my_id] = my_desc;
          cv.slotpos[my_id] = unsigned(pos);
          cv.homes[my_id] = uint32_t(h);
          pend.slot = slot;
          pend.val = tag | (unsigned long long)(my_id + 1u);
        } else {
          st_relaxed(slot, tag | kSlotTomb);  // nothing to order: no CM behind it
          atomicExch(&cv.ctr->full, 1u);
        }
      }
    }
    if (state == kDeferred) defer(cv, my_desc);
  }
};

// Candidate generators of path C.
template <typename W>
struct BinaryGen {
  const uint4* a_rows;  // shared memory: row p of the group at a_rows[p * 32]
  uint4 b;              // this lane's vector of the streamed operand
  uint32_t a0, b_id;    // cache id of row 0 of the group, and of b
  int steps, lane;
  __device__ void compute4(int q0, uint4 (&c)[4]) const {
    const uint4 a = a_rows[(q0 >> 2) * 32 + lane];
    c[0] = v_op<W>(kAnd, a, b, b, steps);
    c[1] = v_op<W>(kOr, a, b, b, steps);
    c[2] = v_op<W>(kUntil, a, b, b, steps);
    c[3] = v_op<W>(kUntil, b, a, b, steps);
  }
  __device__ uint4 compute(int q) const {
    const uint4 a = a_rows[(q >> 2) * 32 + lane];
    switch (q & 3) {
      case 0: return v_op<W>(kAnd, a, b, b, steps);
      case 1: return v_op<W>(kOr, a, b, b, steps);
      case 2: return v_op<W>(kUntil, a, b, b, steps);
      default: return v_op<W>(kUntil, b, a, b, steps);
    }
  }
  __device__ uint64_t desc(int q) const {
    const uint32_t ai = a0 + uint32_t(q >> 2);
    switch (q & 3) {
      case 0: return pack_desc(kAnd, ai, b_id);
      case 1: return pack_desc(kOr, ai, b_id);
      case 2: return pack_desc(kUntil, ai, b_id);
      default: return pack_desc(kUntil, b_id, ai);
    }
  }
};

template <typename W>
struct UnaryGen {
  const uint4* rows;  // shared memory: row p at rows[p * 32]
  uint4 lm;
  uint32_t id0;       // cache id of row 0
  int steps, lane;
  __device__ void compute4(int q0, uint4 (&c)[4]) const {
    const uint4 a = rows[(q0 >> 2) * 32 + lane];
    c[0] = v_op<W>(kNot, a, a, lm, steps);
    c[1] = v_op<W>(kNext, a, a, lm, steps);
    c[2] = v_op<W>(kFuture, a, a, lm, steps);
    c[3] = v_op<W>(kGlobally, a, a, lm, steps);
  }
  __device__ uint4 compute(int q) const {
    return v_op<W>(unary_code(q & 3), rows[(q >> 2) * 32 + lane], make_uint4(0, 0, 0, 0), lm, steps);
  }
  __device__ uint64_t desc(int q) const { return pack_desc(unary_code(q & 3), id0 + uint32_t(q >> 2), 0); }
};

template <typename W>
struct ListGen {
  const CacheView* cv;
  const uint64_t* d;  // shared memory: the batch's descriptors
  uint4* keep;        // shared memory: this lane's vector of candidate q at keep[q * 32 + lane]
  uint4 lm;
  int lane;
  // The batch's hash pass computes every candidate (in groups of four, in
  // order) before any compute(q): each candidate's operands are read once and
  // its vector kept for the compare and write passes.
  __device__ void compute4(int q0, uint4 (&c)[4]) const {
#pragma unroll
    for (int o = 0; o < 4; ++o) c[o] = build(q0 + o);
#pragma unroll
    for (int o = 0; o < 4; ++o) keep[(q0 + o) * 32 + lane] = c[o];
  }
  __device__ uint4 compute(int q) const { return keep[q * 32 + lane]; }
  __device__ uint4 build(int q) const {
    const uint64_t dd = d[q];
    const uint32_t op = desc_op(dd);
    if (op == kAtom) return __ldg(cv->atoms + size_t(desc_left(dd)) * cv->vecs + lane);
    const uint4 a = __ldg(row_ptr(*cv, desc_left(dd)) + lane);
    const uint4 b = (op == kAnd || op == kOr || op == kUntil) ? __ldg(row_ptr(*cv, desc_right(dd)) + lane) : a;
    return v_op<W>(op, a, b, lm, cv->steps);
  }
  __device__ uint64_t desc(int q) const { return d[q]; }
};

// Rows of level k-1 per warp batch of k_unary_c (4 operators each: 32
// candidates, every lane probes): fewer warps fit than with 4-row batches
// (the rows take shared memory), but each batch's round trips serve twice the
// candidates, which measured faster.
constexpr int kUnaryRowsC = 8;

template <typename W>
__global__ void __launch_bounds__(256, 3) k_unary_c(CacheView cv, uint32_t first, uint32_t count, uint32_t ops) {
  using P = PathC<W>;
  constexpr int ROWS = kUnaryRowsC;
  extern __shared__ uint4 smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  uint4* rows = smem + wib * (ROWS * 32 + P::kStage);
  uint4* stage = rows + ROWS * 32;
  typename P::Consts k;
  P::load_consts(cv, k);
  UnaryGen<W> gen;
  gen.rows = rows;
  gen.lm = cv.lenmask[lane];
  gen.steps = cv.steps;
  gen.lane = lane;
  uint32_t en_ops = 0;  // candidate q is real iff its operator is enabled
#pragma unroll
  for (int q = 0; q < 4 * ROWS; ++q) en_ops |= ((ops >> (q & 3)) & 1u) << q;
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  unsigned long long built = 0;
  typename P::Pending pend;
  typename P::Ids idr;
  uint32_t iter = 0;
  for (uint32_t base = warp * ROWS; base < count; base += nwarps * ROWS, ++iter) {
    if ((iter & 3u) == 0 && __any_sync(kFull, stop_requested(cv))) break;
    const uint32_t nrows = min(uint32_t(ROWS), count - base);
#pragma unroll
    for (int p = 0; p < ROWS; ++p)
      if (p < int(nrows)) rows[p * 32 + lane] = __ldg(row_ptr(cv, first + base + p) + lane);
    __syncwarp();
    gen.id0 = first + base;
    const uint32_t en = en_ops & ((nrows >= 8u ? 0xFFFFFFFFu : ((1u << (4 * nrows)) - 1u)));
    const bool last = base + nwarps * ROWS >= count;
    P::template batch<false>(cv, k, gen, int(4 * nrows), en, stage, pend, idr, last);
    built += __popc(en);
    __syncwarp();
  }
  WarpDedup::flush(pend);
  WarpDedup::retire(cv, idr);
  if (lane == 0 && built) atomicAdd(&cv.ctr->built_k[cv.kind], built);
}

template <typename W>
__global__ void __launch_bounds__(256, 4) k_binary_c(CacheView cv, BinaryPlan plan) {
  using P = PathC<W>;
  constexpr int PAIRS = 8;  // 32 candidates per batch
  extern __shared__ uint4 smem[];
  __shared__ unsigned long long s_tile;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint4* s_left = smem;  // plan.tile rows x 32 vectors
  uint4* stage = smem + size_t(plan.tile) * 32 + warp * P::kStage;
  typename P::Consts k;
  P::load_consts(cv, k);
  uint32_t en_ops = 0;
#pragma unroll
  for (int q = 0; q < 4 * PAIRS; ++q) en_ops |= ((plan.ops >> (q & 3)) & 1u) << q;
  __shared__ unsigned s_row;
  BinaryGen<W> gen;
  gen.steps = cv.steps;
  gen.lane = lane;
  unsigned long long built = 0;
  typename P::Pending pend;
  typename P::Ids idr;
  while (true) {
    if (threadIdx.x == 0) {
      unsigned long long t = atomicAdd(&cv.ctr->work[plan.work_slot], 1ull);
      if (stop_requested(cv)) t = plan.total_tiles;  // early exit is polled once per tile
      s_tile = t;
      s_row = 0;
    }
    __syncthreads();
    const unsigned long long tile = s_tile;
    if (tile >= plan.total_tiles) break;
    int sp = 0;
    while (sp + 1 < plan.n_splits && plan.s[sp + 1].tiles_begin <= tile) ++sp;
    const Split& S = plan.s[sp];
    const unsigned long long t = tile - S.tiles_begin;
    const uint32_t lt = uint32_t(t / S.rt_tiles);
    const uint32_t rt = uint32_t(t - (unsigned long long)lt * S.rt_tiles);
    const bool skip = S.tri && rt < lt;
    const uint32_t l0 = lt * plan.tile, r0 = rt * plan.tile;
    const uint32_t ln = skip ? 0u : min(plan.tile, S.left_n - l0);
    const uint32_t rn = skip ? 0u : min(plan.tile, S.right_n - r0);
    {
      const uint4* src = row_ptr(cv, S.left_start + l0);
      const uint32_t total = ln * 32u;
      for (uint32_t i = threadIdx.x; i < total; i += blockDim.x) s_left[i] = __ldg(src + i);
    }
    __syncthreads();
    while (true) {
      // streamed rows are handed out one at a time: warps that meet more
      // duplicates (or more inserts) do not hold the others at the barrier
      unsigned rr = 0;
      if (lane == 0) rr = atomicAdd(&s_row, 1u);
      rr = __shfl_sync(kFull, rr, 0);
      if (rr >= rn) break;
      gen.b_id = S.right_start + r0 + rr;
      gen.b = __ldg(row_ptr(cv, gen.b_id) + lane);
      for (uint32_t li = 0; li < ln; li += PAIRS) {
        // pairs li .. li + np - 1 of the staged rows; same level: only a < b
        uint32_t np = min(uint32_t(PAIRS), ln - li);
        gen.a0 = S.left_start + l0 + li;
        if (S.tri) np = gen.b_id > gen.a0 ? min(np, gen.b_id - gen.a0) : 0u;
        if (np == 0) break;  // rows ascend: no later row pairs with b either
        gen.a_rows = s_left + li * 32;
        const uint32_t en = en_ops & (np >= 8u ? 0xFFFFFFFFu : ((1u << (4 * np)) - 1u));
        P::template batch<true>(cv, k, gen, int(4 * np), en, stage, pend, idr);
        built += __popc(en);
      }
    }
    __syncthreads();
  }
  WarpDedup::flush(pend);
  WarpDedup::retire(cv, idr);
  if (lane == 0 && built) atomicAdd(&cv.ctr->built_k[cv.kind], built);
}

// Splits whose smaller level has fewer than kSmallSplitRows rows (the atoms
// against a large level): a block tile of the small level would give batches
// of fewer than 8 pairs. (Up to 16 rows measured the same as 8; at 32 and
// above the block tiles of k_binary_c were faster, the row reuse of a shared
// tile outweighing partly filled batches.) Here each warp stages 8 rows
// of the larger level (`left`, in chunks of 8: lt_tiles chunks per split) in
// shared memory and pairs them with every row of the smaller level (`right`,
// read from L2), one full batch of 8 pairs x 4 operators per small row. The
// candidate set is the split's; only the operand roles differ (and and or
// commute, and both orders of U are built). A work item is one chunk against
// `group` rows of the small side (all of them unless the level is too small
// to give every warp a few chunks: lt_tiles chunks x rt_tiles row groups);
// items are dealt to warps in grid-stride order; no block barrier.
constexpr uint32_t kSmallSplitRows = 16;

template <typename W>
__global__ void __launch_bounds__(256, 3) k_binary_small_c(CacheView cv, BinaryPlan plan) {
  using P = PathC<W>;
  constexpr int ROWS = 8;
  extern __shared__ uint4 smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  uint4* rows = smem + wib * (ROWS * 32 + P::kStage);
  uint4* stage = rows + ROWS * 32;
  typename P::Consts k;
  P::load_consts(cv, k);
  uint32_t en_ops = 0;
#pragma unroll
  for (int q = 0; q < 4 * ROWS; ++q) en_ops |= ((plan.ops >> (q & 3)) & 1u) << q;
  BinaryGen<W> gen;
  gen.a_rows = rows;
  gen.steps = cv.steps;
  gen.lane = lane;
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  unsigned long long built = 0;
  typename P::Pending pend;
  typename P::Ids idr;
  for (unsigned long long c = warp; c < plan.total_tiles; c += nwarps) {
    if (__any_sync(kFull, stop_requested(cv))) break;
    int sp = 0;
    while (sp + 1 < plan.n_splits && plan.s[sp + 1].tiles_begin <= c) ++sp;
    const Split& S = plan.s[sp];
    const unsigned long long local = c - S.tiles_begin;
    const uint32_t chunk = uint32_t(local / S.rt_tiles);
    const uint32_t r0 = uint32_t(local - (unsigned long long)chunk * S.rt_tiles) * S.group;
    const uint32_t r1 = min(r0 + S.group, S.right_n);
    const uint32_t l0 = chunk * uint32_t(ROWS);
    const uint32_t np = min(uint32_t(ROWS), S.left_n - l0);
#pragma unroll
    for (int p = 0; p < ROWS; ++p)
      if (p < int(np)) rows[p * 32 + lane] = __ldg(row_ptr(cv, S.left_start + l0 + p) + lane);
    __syncwarp();
    gen.a0 = S.left_start + l0;
    const uint32_t en = en_ops & (np >= 8u ? 0xFFFFFFFFu : ((1u << (4 * np)) - 1u));
    const bool last_item = c + nwarps >= plan.total_tiles;
    for (uint32_t r = r0; r < r1; ++r) {
      gen.b_id = S.right_start + r;
      gen.b = __ldg(row_ptr(cv, gen.b_id) + lane);
      P::template batch<true>(cv, k, gen, int(4 * np), en, stage, pend, idr, last_item && r + 1u == r1);
      built += __popc(en);
    }
    __syncwarp();
  }
  WarpDedup::flush(pend);
  WarpDedup::retire(cv, idr);
  if (lane == 0 && built) atomicAdd(&cv.ctr->built_k[cv.kind], built);
}

// Candidates per warp batch of k_desc_c. A deferred candidate is built from
// its descriptor's operand rows in global memory, one round trip per group of
// four; small batches keep that chain short and spread a short list (the
// usual case) over many warps.
constexpr int kDescBatch = 8;

template <typename W>
__global__ void __launch_bounds__(256, 3) k_desc_c(CacheView cv, const unsigned long long* list,
                                                   const unsigned int* list_n, unsigned int list_cap,
                                                   unsigned int implicit_atoms) {
  using P = PathC<W>;
  constexpr int N = kDescBatch;
  extern __shared__ uint4 smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  uint4* stage = smem + wib * (P::kStage + N * 32 + N / 2);
  uint4* keep = stage + P::kStage;
  uint64_t* dbuf = reinterpret_cast<uint64_t*>(keep + N * 32);  // N descriptors
  typename P::Consts k;
  P::load_consts(cv, k);
  ListGen<W> gen;
  gen.cv = &cv;
  gen.d = dbuf;
  gen.keep = keep;
  gen.lm = cv.lenmask[lane];
  gen.lane = lane;
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  unsigned n = implicit_atoms;
  if (list) n = min(*list_n, list_cap);
  typename P::Pending pend;
  typename P::Ids idr;
  for (uint32_t base = warp * N; base < n; base += nwarps * N) {
    if (__any_sync(kFull, stop_requested(cv))) break;
    const uint32_t cnt = min(uint32_t(N), n - base);
    // descriptors past cnt (up to a multiple of 4) are harmless atoms, disabled by `en`
    if (lane < int(cnt)) dbuf[lane] = list ? list[base + lane] : pack_desc(kAtom, base + lane, 0);
    else if (lane < N) dbuf[lane] = pack_desc(kAtom, 0, 0);
    __syncwarp();
    P::template batch<false>(cv, k, gen, int((cnt + 3u) & ~3u), (1u << cnt) - 1u, stage, pend, idr);
    __syncwarp();
  }
  WarpDedup::flush(pend);
  WarpDedup::retire(cv, idr);
  if (implicit_atoms && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&cv.ctr->built_k[cv.kind], (unsigned long long)n);
}

// ===========================================================================
// Path D (CMs above 512 bytes, e.g. 2048 traces of 64-bit words = 16 KiB): the
// hash-first scheme of path C with rv = vecs / 32 vectors per lane, walked in
// loops, VPT vectors at a time (their operand loads in flight together).
// Operand rows are read through L1/L2 whenever a candidate is (re)computed;
// compares read the stored row directly.
// ===========================================================================
template <typename W, int VPT = 1, int CU = 1>
struct PathD {
  using Pending = WarpDedup::Pending;
  using Ids = WarpDedup::Ids;

  // f(v, c) for this lane's vectors v of candidate q, VPT computed together.
  template <class Gen, class F>
  __device__ static void each_vec(const Gen& gen, int q, unsigned rv, F&& f) {
    const unsigned lane = threadIdx.x & 31u;
    for (unsigned r = 0; r < rv; r += VPT) {
      uint4 c[VPT];
#pragma unroll
      for (int u = 0; u < VPT; ++u)
        c[u] = r + u < rv ? gen.compute(q, lane + 32u * (r + u)) : make_uint4(0, 0, 0, 0);
#pragma unroll
      for (int u = 0; u < VPT; ++u)
        if (r + u < rv) f(lane + 32u * (r + u), c[u]);
    }
  }

  template <bool kEarlyPublish, class Gen>
  __device__ static void batch(const CacheView& cv, const Gen& gen, int n, uint32_t en, Pending& pend, Ids& ids) {
    WarpDedup::prefetch(cv, ids);
    const int lane = threadIdx.x & 31;
    const unsigned rv = cv.vecs >> 5;
    uint32_t my_lo = 0, my_hi = 0, bad = 0;
    // Four candidates at a time (one operand group and its four operators, or
    // four descriptors): one pass over this lane's vectors, VPT at a time.
    for (int q0 = 0; q0 < n; q0 += 4) {
      uint64_t acc[4] = {0, 0, 0, 0};
      uint32_t diff[4] = {0, 0, 0, 0};
      for (unsigned r = 0; r < rv; r += VPT) {
#pragma unroll
        for (int u = 0; u < VPT; ++u) {
          if (r + u >= rv) break;
          const unsigned v = lane + 32u * (r + u);
          uint4 c[4];
          gen.compute4(q0, v, c);
          const uint4 mul = __ldg(cv.hmul + v);
          const uint32_t lab = v < cv.plane_vecs ? bit0s<W>(__ldg(cv.label + v)) : 0u;
#pragma unroll
          for (int o = 0; o < 4; ++o) {
            acc[o] = h_mac(c[o], mul, acc[o]);
            if (v < cv.plane_vecs) diff[o] |= bit0s<W>(c[o]) ^ lab;  // position 0: plane 0
          }
        }
      }
#pragma unroll
      for (int o = 0; o < 4; ++o) {
        const int q = q0 + o;
        const uint32_t lo = __reduce_add_sync(kFull, uint32_t(acc[o]));
        const uint32_t hi = __reduce_add_sync(kFull, uint32_t(acc[o] >> 32));
        my_lo = lane == q ? lo : my_lo;
        my_hi = lane == q ? hi : my_hi;
        if (q < 32) bad |= (diff[o] != 0u ? 1u : 0u) << q;
      }
    }
    bad = __reduce_or_sync(kFull, bad);
    const bool mine = lane < n && ((en >> lane) & 1u);
    const uint64_t my_desc = gen.desc(lane < n ? lane : 0);
    if (mine && !((bad >> lane) & 1u)) record_solution(cv, my_desc);

    constexpr int kProbing = WarpDedup::kProbing, kDone = WarpDedup::kDone,
                  kClaimed = WarpDedup::kClaimed, kDeferred = WarpDedup::kDeferred;
    const bool full = WarpDedup::arena_full(cv);
    int state = (mine && !full) ? kProbing : kDone;  // a full arena: spec check only
    const uint64_t h = h_fin(my_hi, my_lo);
    const unsigned long long tag = (h >> 32) << 32;
    unsigned long long pos = h & cv.table_mask;
    // in-batch twins (equal hashes): settle them by comparing the candidates
    const uint32_t mine_mask = __ballot_sync(kFull, mine);
    const uint32_t peers = __match_any_sync(kFull, (unsigned long long)h) & mine_mask;
    const bool has_twin = mine && (peers & ((1u << lane) - 1u)) != 0u;
    const int twin = __ffs(peers) - 1;
    for (uint32_t m = __ballot_sync(kFull, has_twin); m; m &= m - 1u) {
      const int q = __ffs(m) - 1;
      const int p = __shfl_sync(kFull, twin, q);
      uint32_t ne = 0;
      each_vec(gen, q, rv, [&](unsigned v, const uint4& c) { ne |= v_ne(c, gen.compute(p, v)); });
      const bool eq = !__any_sync(kFull, ne != 0u);
      if (lane == q && eq) state = kDone;
    }
    if (kEarlyPublish) WarpDedup::flush(pend);
    uint32_t cmp_id = 0;
    unsigned long long guard = 0;
    while (true) {
      bool need = false;
      if (state == kProbing) {
        const unsigned long long sv = probe_slot(cv.table + pos, tag | kSlotPending);
        if (sv == 0ull) {
          state = kClaimed;
        } else {
          const uint32_t low = uint32_t(sv);
          if (low == kSlotTomb) state = kDone;  // the arena is full: this level is incomplete (see path A)
          else if ((sv & 0xFFFFFFFF00000000ull) != tag) pos = (pos + 1) & cv.table_mask;
          else if (low == kSlotPending) state = kDeferred;
          else {
            need = true;
            cmp_id = low - 1u;
          }
        }
      }
      const uint32_t need_m = __ballot_sync(kFull, need);
      if (need_m) __syncwarp();  // the probing lanes' acquires, before every lane's row reads
      // The tag matches of one operand group (four candidates) are compared in
      // one pass over its vectors, so the operands are read once per group.
      uint32_t ne_m = 0;  // bit q: candidate q differs from the row its probe found
      for (uint32_t gm = need_m; gm;) {
        const int g = (__ffs(gm) - 1) >> 2;
        const uint32_t sub = (need_m >> (4 * g)) & 0xFu;  // warp-uniform
        gm &= ~(0xFu << (4 * g));
        const uint4* src[4];
#pragma unroll
        for (int o = 0; o < 4; ++o) src[o] = row_ptr(cv, __shfl_sync(kFull, cmp_id, 4 * g + o));  // published rows, read past L1
        uint32_t ne[4] = {0u, 0u, 0u, 0u};
        if constexpr (CU == 1) {
          for (unsigned r = 0; r < rv; ++r) {
            const unsigned v = lane + 32u * r;
            uint4 c[4];
            gen.compute4(4 * g, v, c, sub);
#pragma unroll
            for (int o = 0; o < 4; ++o)
              if ((sub >> o) & 1u) ne[o] |= v_ne(__ldcg(src[o] + v), c[o]);
          }
        } else {
        // CU vectors per lane of each stored row read together (their loads in
        // flight at once), then compared
        for (unsigned r = 0; r < rv; r += CU) {
          uint4 st[CU][4];
#pragma unroll
          for (int u = 0; u < CU; ++u)
#pragma unroll
            for (int o = 0; o < 4; ++o)
              st[u][o] = ((sub >> o) & 1u) && r + u < rv ? __ldcg(src[o] + lane + 32u * (r + u))
                                                          : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
          for (int u = 0; u < CU; ++u) {
            if (r + u >= rv) break;
            uint4 c[4];
            gen.compute4(4 * g, lane + 32u * (r + u), c, sub);
#pragma unroll
            for (int o = 0; o < 4; ++o)
              if ((sub >> o) & 1u) ne[o] |= v_ne(st[u][o], c[o]);
          }
        }
        }
#pragma unroll
        for (int o = 0; o < 4; ++o)
          if (((sub >> o) & 1u) && __any_sync(kFull, ne[o] != 0u)) ne_m |= 1u << (4 * g + o);
      }
      if ((need_m >> lane) & 1u) {
        if (!((ne_m >> lane) & 1u)) state = kDone;  // equal CM already cached
        else pos = (pos + 1) & cv.table_mask;
      }
      if (!__any_sync(kFull, state == kProbing)) break;
      if (++guard > cv.table_mask) {
        if (lane == 0) atomicExch(&cv.ctr->error, 1u);
        if (state == kProbing) state = kDone;
      }
    }
    const uint32_t claim = __ballot_sync(kFull, state == kClaimed);
    const unsigned n_claim = unsigned(__popc(claim));
    const unsigned have = ids.end - ids.next;
    const bool use_pre = n_claim > have && ids.pre_ok;
    unsigned base = 0;
    if (n_claim > have && !use_pre && lane == 0)
      base = atomicAdd(&cv.ctr->n_entries, max(cv.chunk, n_claim - have));
    if (!kEarlyPublish) WarpDedup::flush(pend);
    if (claim) {
      const unsigned fresh = WarpDedup::take(ids, n_claim, have, base, use_pre);
      // the rows of one operand group's claims in one pass over its vectors
      for (uint32_t gm = claim; gm;) {
        const int g = (__ffs(gm) - 1) >> 2;
        const uint32_t sub = (claim >> (4 * g)) & 0xFu;  // warp-uniform
        gm &= ~(0xFu << (4 * g));
        uint4* dst[4];
#pragma unroll
        for (int o = 0; o < 4; ++o) {
          const int q = 4 * g + o;
          const unsigned rank = unsigned(__popc(claim & ((1u << q) - 1u)));  // ids go by rank among the claims
          const unsigned id = rank < have ? ids.next + rank : fresh + (rank - have);
          dst[o] = ((sub >> o) & 1u) && id < cv.max_entries ? cv.arena + size_t(id) * cv.vecs : nullptr;
        }
        for (unsigned r = 0; r < rv; ++r) {
          const unsigned v = lane + 32u * r;
          uint4 c[4];
          gen.compute4(4 * g, v, c, sub);
#pragma unroll
          for (int o = 0; o < 4; ++o)
            if (dst[o]) dst[o][v] = c[o];
        }
      }
      const unsigned my_rank = unsigned(__popc(claim & ((1u << lane) - 1u)));
      const unsigned my_id = my_rank < have ? ids.next + my_rank : fresh + (my_rank - have);
      WarpDedup::advance(cv, ids, n_claim, have, fresh, use_pre);
      ids.inserted += __popc(__ballot_sync(kFull, state == kClaimed && my_id < cv.max_entries));
      if (state == kClaimed) {
        unsigned long long* slot = cv.table + pos;
        if (my_id < cv.max_entries) {
          cv.prov[my_id] = my_desc;
          cv.slotpos[my_id] = unsigned(pos);
          cv.homes[my_id] = uint32_t(h);
          pend.slot = slot;
          pend.val = tag | (unsigned long long)(my_id + 1u);
        } else {
          st_relaxed(slot, tag | kSlotTomb);
          atomicExch(&cv.ctr->full, 1u);
        }
      }
    }
    if (state == kDeferred) defer(cv, my_desc);
  }
};

// Generators of path D: candidate q (0..31) from operand ids held in shared
// memory (8 groups of 4 operators), vector v of this lane.
template <typename W>
struct PairGenD {
  const CacheView* cv;
  const uint2* pairs;  // shared memory: (a id, b id) of pair p
  __device__ uint4 compute(int q, unsigned v) const {
    const uint2 pr = pairs[q >> 2];
    const uint4* a = row_ptr(*cv, pr.x);
    const uint4* b = row_ptr(*cv, pr.y);
    switch (q & 3) {
      case 0: return row_op<W>(*cv, kAnd, a, b, v);
      case 1: return row_op<W>(*cv, kOr, a, b, v);
      case 2: return row_op<W>(*cv, kUntil, a, b, v);
      default: return row_op<W>(*cv, kUntil, b, a, v);
    }
  }
  // vector v of candidates q0 .. q0 + 3 (one pair, its four operators): the
  // operands' vectors are read once (all four are computed whatever `sub` asks)
  __device__ void compute4(int q0, unsigned v, uint4 (&c)[4], uint32_t /*sub*/ = 0xFu) const {
    const uint2 pr = pairs[q0 >> 2];
    const uint4* a = row_ptr(*cv, pr.x);
    const uint4* b = row_ptr(*cv, pr.y);
    if (cv->planes > 1) {
      c[0] = row_op<W>(*cv, kAnd, a, b, v);
      c[1] = row_op<W>(*cv, kOr, a, b, v);
      c[2] = row_op<W>(*cv, kUntil, a, b, v);
      c[3] = row_op<W>(*cv, kUntil, b, a, v);
      return;
    }
    const uint4 x = __ldg(a + v), y = __ldg(b + v);
    c[0] = v_op<W>(kAnd, x, y, y, 0);
    c[1] = v_op<W>(kOr, x, y, y, 0);
    c[2] = v_op<W>(kUntil, x, y, y, 0);
    c[3] = v_op<W>(kUntil, y, x, y, 0);
  }
  __device__ uint64_t desc(int q) const {
    const uint2 pr = pairs[q >> 2];
    switch (q & 3) {
      case 0: return pack_desc(kAnd, pr.x, pr.y);
      case 1: return pack_desc(kOr, pr.x, pr.y);
      case 2: return pack_desc(kUntil, pr.x, pr.y);
      default: return pack_desc(kUntil, pr.y, pr.x);
    }
  }
};

template <typename W>
struct RowGenD {
  const CacheView* cv;
  uint32_t id0;
  __device__ uint4 compute(int q, unsigned v) const {
    const uint4* a = row_ptr(*cv, id0 + uint32_t(q >> 2));
    return row_op<W>(*cv, unary_code(q & 3), a, a, v);
  }
  // vector v of candidates q0 .. q0 + 3 (one row, its four operators)
  __device__ void compute4(int q0, unsigned v, uint4 (&c)[4], uint32_t /*sub*/ = 0xFu) const {
    const uint4* a = row_ptr(*cv, id0 + uint32_t(q0 >> 2));
    if (cv->planes > 1) {
#pragma unroll
      for (int o = 0; o < 4; ++o) c[o] = row_op<W>(*cv, unary_code(o), a, a, v);
      return;
    }
    const uint4 x = __ldg(a + v), lm = __ldg(cv->lenmask + v);
#pragma unroll
    for (int o = 0; o < 4; ++o) c[o] = v_op<W>(unary_code(o), x, x, lm, 0);
  }
  __device__ uint64_t desc(int q) const { return pack_desc(unary_code(q & 3), id0 + uint32_t(q >> 2), 0); }
};

template <typename W>
struct ListGenD {
  const CacheView* cv;
  const uint64_t* d;  // shared memory: the batch's descriptors
  __device__ uint4 compute(int q, unsigned v) const {
    const uint64_t dd = d[q];
    const uint32_t op = desc_op(dd);
    if (op == kAtom) return __ldg(cv->atoms + size_t(desc_left(dd)) * cv->vecs + v);
    const uint4* a = row_ptr(*cv, desc_left(dd));
    const uint4* b = (op == kAnd || op == kOr || op == kUntil) ? row_ptr(*cv, desc_right(dd)) : a;
    return row_op<W>(*cv, op, a, b, v);
  }
  // four independent descriptors (the batch is padded with harmless atoms):
  // only those in `sub` are computed
  __device__ void compute4(int q0, unsigned v, uint4 (&c)[4], uint32_t sub = 0xFu) const {
#pragma unroll
    for (int o = 0; o < 4; ++o) c[o] = ((sub >> o) & 1u) ? compute(q0 + o, v) : make_uint4(0, 0, 0, 0);
  }
  __device__ uint64_t desc(int q) const { return d[q]; }
};

// Rows of level k-1 per warp batch of k_unary_d (4 operators each). A batch
// reads its rows once to hash them and again to compare or write its
// candidates; one 16 KiB row per warp keeps the rows of all resident warps
// in L2 between the passes (8 rows per warp did not fit, and the second reads
// went to DRAM), and a batch's round trips stay short beside its streaming.
constexpr int kRowsD = 1;
// Vectors per lane computed together in the hash pass of path D: of k_unary_d
// (one row read, four loads in flight per lane), and of k_binary_d and
// k_desc_d. Measured at 16 KiB CMs: 4 against 1, 2 or 8 for the unary
// kernel, 2 against 1 or 4 for the binary one.
constexpr int kVptUnaryD = 4;
constexpr int kVptD = 2;

template <typename W>
__global__ void __launch_bounds__(256) k_unary_d(CacheView cv, uint32_t first, uint32_t count, uint32_t ops) {
  using P = PathD<W, kVptUnaryD>;
  constexpr int ROWS = kRowsD;
  const int lane = threadIdx.x & 31;
  RowGenD<W> gen;
  gen.cv = &cv;
  uint32_t en_ops = 0;
#pragma unroll
  for (int q = 0; q < 4 * ROWS; ++q) en_ops |= ((ops >> (q & 3)) & 1u) << q;
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  unsigned long long built = 0;
  typename P::Pending pend;
  typename P::Ids idr;
  for (uint32_t base = warp * ROWS; base < count; base += nwarps * ROWS) {
    if (__any_sync(kFull, stop_requested(cv))) break;
    const uint32_t nrows = min(uint32_t(ROWS), count - base);
    gen.id0 = first + base;
    const uint32_t en = en_ops & (nrows >= 8u ? 0xFFFFFFFFu : ((1u << (4 * nrows)) - 1u));
    P::template batch<false>(cv, gen, int(4 * nrows), en, pend, idr);
    built += __popc(en);
  }
  WarpDedup::flush(pend);
  WarpDedup::retire(cv, idr);
  if (lane == 0 && built) atomicAdd(&cv.ctr->built_k[cv.kind], built);
}

// Staged form of k_unary_d for one-plane CMs of 8-16 KiB. Each warp copies
// its operand row into shared memory with one bulk copy (the TMA unit moves the
// whole row while the warp waits on an mbarrier) and every pass of the batch
// (hash and specification check, in-batch twins, compares, writes) computes
// the four operators from that copy: the row is read from HBM once, where
// k_unary_d reads it again after its probes and, with 16 KiB rows, finds it
// evicted from L2 about a quarter of the time. Shared memory bounds the block
// to as many warps as rows of M bytes fit its shared memory: 14 with 16 KiB
// rows.
constexpr unsigned kStagedMinBytes = 8192, kStagedMaxBytes = 16384;
constexpr int kStagedMaxWarps = 16;
constexpr unsigned kBulkChunk = 4096;        // bytes per bulk copy instruction
constexpr unsigned kRowWaitPolls = 1u << 22; // polls of the row's barrier before the warp gives up
// Vectors per lane of each stored row that the compare pass of k_unary_ds
// loads together: with few warps per SM, a compare read one vector at a time
// was a chain of 32 round trips per 16 KiB row.
constexpr int kCmpVecsDS = 4;

template <typename W>
struct RowGenDS {
  const CacheView* cv;
  const uint4* row;  // shared memory: the operand row
  uint32_t id0;
  __device__ uint4 compute(int q, unsigned v) const {
    const uint4 x = row[v];
    return v_op<W>(unary_code(q & 3), x, x, __ldg(cv->lenmask + v), 0);
  }
  __device__ void compute4(int /*q0*/, unsigned v, uint4 (&c)[4], uint32_t /*sub*/ = 0xFu) const {
    const uint4 x = row[v], lm = __ldg(cv->lenmask + v);
#pragma unroll
    for (int o = 0; o < 4; ++o) c[o] = v_op<W>(unary_code(o), x, x, lm, 0);
  }
  __device__ uint64_t desc(int q) const { return pack_desc(unary_code(q & 3), id0, 0); }
};

template <typename W>
__global__ void __launch_bounds__(32 * kStagedMaxWarps) k_unary_ds(CacheView cv, uint32_t first, uint32_t count,
                                                                   uint32_t ops) {
  using P = PathD<W, kVptUnaryD, kCmpVecsDS>;
  extern __shared__ __align__(128) uint4 smem_rows[];
  __shared__ unsigned long long s_bar[kStagedMaxWarps];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const unsigned row_bytes = cv.vecs * 16u;
  uint4* row = smem_rows + size_t(wib) * cv.vecs;
  unsigned long long* bar = s_bar + wib;
  if (lane == 0) mbar_init(bar, 1u);
  __syncwarp();
  RowGenDS<W> gen;
  gen.cv = &cv;
  gen.row = row;
  const uint32_t en = ops & 0xFu;  // the four operators of the row, as enabled
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  unsigned long long built = 0;
  typename P::Pending pend;
  typename P::Ids idr;
  unsigned parity = 0;
  for (uint32_t base = warp; base < count; base += nwarps) {
    if (__any_sync(kFull, stop_requested(cv))) break;
    // every lane's reads of the previous row are done before the copy overwrites it
    __syncwarp();
    if (lane == 0) {
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(bar, row_bytes);
      const char* src = reinterpret_cast<const char*>(row_ptr(cv, first + base));
      char* dst = reinterpret_cast<char*>(row);
      for (unsigned off = 0; off < row_bytes; off += kBulkChunk)
        bulk_load(dst + off, src + off, min(kBulkChunk, row_bytes - off), bar);
    }
    if (!mbar_wait_bounded(bar, parity, kRowWaitPolls)) {
      // cannot happen while the copy engine works: record it, give the copy a
      // second bounded wait (it writes this block's shared memory) and stop
      if (lane == 0) atomicExch(&cv.ctr->error, 6u);
      mbar_wait_bounded(bar, parity, kRowWaitPolls);
      break;
    }
    parity ^= 1u;
    gen.id0 = first + base;
    P::template batch<false>(cv, gen, 4, en, pend, idr);
    built += __popc(en);
  }
  WarpDedup::flush(pend);
  WarpDedup::retire(cv, idr);
  if (lane == 0 && built) atomicAdd(&cv.ctr->built_k[cv.kind], built);
}

// Pairs of every split in one flat index space (as path A), kPairsD per warp
// batch (4 measured faster than 8, 2 or 1 at 16 KiB CMs).
constexpr int kPairsD = 4;

template <typename W>
__global__ void __launch_bounds__(256) k_binary_d(CacheView cv, BinaryPlan plan) {
  using P = PathD<W, kVptD>;
  constexpr int PAIRS = kPairsD;
  __shared__ uint2 s_pairs[8][PAIRS];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  PairGenD<W> gen;
  gen.cv = &cv;
  gen.pairs = s_pairs[wib];
  const unsigned long long warp = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) >> 5;
  const unsigned long long nwarps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
  unsigned long long built = 0;
  typename P::Pending pend;
  typename P::Ids idr;
  for (unsigned long long g0 = warp * PAIRS; g0 < plan.total_pairs; g0 += nwarps * PAIRS) {
    if (__any_sync(kFull, stop_requested(cv))) break;
    // lane p < PAIRS maps pair g0 + p to its operands
    uint32_t ok = 0;
    if (lane < PAIRS) {
      const unsigned long long pidx = g0 + lane;
      bool valid = pidx < plan.total_pairs;
      uint2 pr = make_uint2(0, 0);
      if (valid) {
        int sp = 0;
        while (sp + 1 < plan.n_splits && plan.s[sp + 1].pairs_begin <= pidx) ++sp;
        const Split& S = plan.s[sp];
        const uint2 ab = split_pair(S, pidx - S.pairs_begin, true);
        pr = make_uint2(S.left_start + ab.x, S.right_start + ab.y);
      }
      s_pairs[wib][lane] = pr;
      ok = valid ? 1u : 0u;
    }
    const uint32_t pv = __ballot_sync(kFull, ok != 0u) & ((1u << PAIRS) - 1u);
    __syncwarp();
    uint32_t en = 0;
#pragma unroll
    for (int q = 0; q < 4 * PAIRS; ++q) en |= (((pv >> (q >> 2)) & 1u) & ((plan.ops >> (q & 3)) & 1u)) << q;
    if (en) {
      P::template batch<true>(cv, gen, 4 * PAIRS, en, pend, idr);
      built += __popc(en);
    }
    __syncwarp();
  }
  WarpDedup::flush(pend);
  WarpDedup::retire(cv, idr);
  if (lane == 0 && built) atomicAdd(&cv.ctr->built_k[cv.kind], built);
}

// Descriptors per warp batch of k_desc_d: one group of four. A path-D batch
// walks its groups one after another, each a chain of passes over the
// candidates' vectors, so a short deferred list (the usual case) spreads over
// many warps instead of queueing in a few.
constexpr int kDescBatchD = 4;

template <typename W>
__global__ void __launch_bounds__(256) k_desc_d(CacheView cv, const unsigned long long* list,
                                                const unsigned int* list_n, unsigned int list_cap,
                                                unsigned int implicit_atoms) {
  using P = PathD<W, kVptD>;
  constexpr int N = kDescBatchD;
  __shared__ uint64_t s_d[8][N];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  ListGenD<W> gen;
  gen.cv = &cv;
  gen.d = s_d[wib];
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  unsigned n = implicit_atoms;
  if (list) n = min(*list_n, list_cap);
  typename P::Pending pend;
  typename P::Ids idr;
  for (uint32_t base = warp * N; base < n; base += nwarps * N) {
    if (__any_sync(kFull, stop_requested(cv))) break;
    const uint32_t cnt = min(uint32_t(N), n - base);
    if (lane < N)
      s_d[wib][lane] = lane < int(cnt) ? (list ? list[base + lane] : pack_desc(kAtom, base + lane, 0))
                                       : pack_desc(kAtom, 0, 0);
    __syncwarp();
    P::template batch<false>(cv, gen, int(cnt), (1u << cnt) - 1u, pend, idr);
    __syncwarp();
  }
  WarpDedup::flush(pend);
  WarpDedup::retire(cv, idr);
  if (implicit_atoms && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&cv.ctr->built_k[cv.kind], (unsigned long long)n);
}

// ===========================================================================
// Batch kernels: the path-D engine over many problems at once. Work items of
// every problem in the step form one index space (per-problem prefix sums in
// StepProblem); warps pull items from a counter, so uneven problems share the
// GPU. When a warp moves to another problem it publishes its pending slots,
// returns its unused ids to that problem's hole log and adds its built count.
// ===========================================================================
__device__ __forceinline__ int find_problem(const StepProblem* steps, int n, unsigned long long item, int which) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {  // last problem whose begin <= item
    const int mid = (lo + hi + 1) >> 1;
    const unsigned long long b = which == 0 ? steps[mid].d_items_begin
                               : which == 1 ? steps[mid].u_items_begin : steps[mid].b_items_begin;
    if (b <= item) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <typename W>
struct BatchWarp {
  int cur = -1;
  unsigned long long built = 0;
  WarpDedup::Pending pend;
  WarpDedup::Ids ids;

  // Make problem p current; its CacheView is copied to this warp's shared slot.
  __device__ void enter(const StepProblem* steps, int p, CacheView* s_cv) {
    if (p == cur) return;
    leave(s_cv);
    const uint32_t* src = reinterpret_cast<const uint32_t*>(&steps[p].cv);
    uint32_t* dst = reinterpret_cast<uint32_t*>(s_cv);
    for (int i = threadIdx.x & 31; i < int(sizeof(CacheView) / 4); i += 32) dst[i] = src[i];
    __syncwarp();
    cur = p;
  }
  __device__ void leave(CacheView* s_cv) {
    if (cur < 0) return;
    WarpDedup::flush(pend);
    WarpDedup::retire(*s_cv, ids);
    if ((threadIdx.x & 31) == 0 && built) atomicAdd(&s_cv->ctr->built_k[s_cv->kind], built);
    built = 0;
    __syncwarp();
    cur = -1;
  }
};

__device__ __forceinline__ unsigned long long grab(unsigned long long* counter) {
  unsigned long long it = 0;
  if ((threadIdx.x & 31) == 0) it = atomicAdd(counter, 1ull);
  return __shfl_sync(kFull, it, 0);
}

// Path A inside the batch runner (CMs of at most 8 vectors): every lane holds
// one candidate, named by its descriptor, rebuilds it from its operands and
// probes / inserts it alone, exactly as k_unary_a / k_binary_a / k_desc_a do.
// The problem's constants sit in this warp's shared slot `ca`, laid out as
// PathA<W, V>::Consts.
template <typename W, int V>
__device__ __forceinline__ unsigned batch_a_one(const CacheView& cv, const uint4* ca, uint64_t d) {
  const auto& s = *reinterpret_cast<const typename PathA<W, V>::Consts*>(ca);
  uint4 c[V];
  rebuild_a<W, V>(cv, s, d, c);
  return PathA<W, V>::process(cv, s, c, d, ld_relaxed_u32(&cv.ctr->full) != 0u);
}

template <typename W>
__device__ __forceinline__ void batch_a_load(const CacheView& cv, uint4* ca) {
  const unsigned V = cv.vecs;
  for (unsigned i = threadIdx.x & 31; i < V; i += 32) {
    ca[i] = cv.lenmask[i];
    ca[V + i] = cv.label[i];
    ca[2 * V + i] = cv.care[i];
    ca[3 * V + i] = cv.hkey[i];
    ca[4 * V + i] = cv.hmul[i];
  }
  __syncwarp();
}

// Every lane with `on` set settles descriptor d; returns the warp's inserts.
template <typename W>
__device__ unsigned batch_a(const CacheView& cv, const uint4* ca, uint64_t d, bool on) {
  unsigned ins = 0;
  if (on) {
    switch (cv.vecs) {
      case 1: ins = batch_a_one<W, 1>(cv, ca, d); break;
      case 2: ins = batch_a_one<W, 2>(cv, ca, d); break;
      case 4: ins = batch_a_one<W, 4>(cv, ca, d); break;
      default: ins = batch_a_one<W, 8>(cv, ca, d); break;
    }
  }
  return __reduce_add_sync(kFull, ins);
}

template <typename W, int VPT>
__global__ void __launch_bounds__(256) k_batch_run(StepHeader* hdr, const StepProblem* steps) {
  using PD = PathD<W, VPT>;
  __shared__ CacheView s_cv[8];
  __shared__ uint2 s_pairs[8][8];
  __shared__ uint64_t s_d[8][32];
  __shared__ uint4 s_ca[8][40];  // path-A constants of the warp's problem (5 x up to 8 vectors)
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  CacheView* cv = &s_cv[wib];
  uint4* ca = s_ca[wib];
  const int n = hdr->n;
  const uint32_t R = uint32_t(hdr->rows);  // unary rows / binary pairs per work item (2, 4 or 8)
  BatchWarp<W> bw;
  auto enter = [&](int p) {
    const bool fresh = p != bw.cur;
    bw.enter(steps, p, cv);
    if (fresh && cv->vecs <= 8u) batch_a_load<W>(*cv, ca);
  };
  // 1. descriptors: atoms of problems at level 1, deferred re-examination
  for (unsigned long long it = grab(&hdr->work[0].v); it < hdr->total_d; it = grab(&hdr->work[0].v)) {
    const int p = find_problem(steps, n, it, 0);
    enter(p);
    const StepProblem& sp = steps[p];
    const uint32_t base = uint32_t(it - sp.d_items_begin) * 32u;
    const uint32_t cnt = min(32u, sp.d_n - base);
    const uint64_t d = lane < int(cnt) ? (sp.d_list ? sp.d_list[base + lane] : pack_desc(kAtom, base + lane, 0))
                                       : pack_desc(kAtom, 0, 0);
    if (cv->vecs <= 8u) {
      bw.ids.inserted += batch_a<W>(*cv, ca, d, lane < int(cnt));
    } else {
      s_d[wib][lane] = d;
      __syncwarp();
      ListGenD<W> gen;
      gen.cv = cv;
      gen.d = s_d[wib];
      PD::template batch<false>(*cv, gen, int(cnt), cnt >= 32u ? 0xFFFFFFFFu : ((1u << cnt) - 1u), bw.pend,
                                bw.ids);
    }
    if (!sp.d_list) bw.built += cnt;  // atoms count as built; deferred ones were counted when first built
    __syncwarp();
  }
  // 2. unary operators, R rows (4R candidates) per item
  for (unsigned long long it = grab(&hdr->work[1].v); it < hdr->total_u; it = grab(&hdr->work[1].v)) {
    const int p = find_problem(steps, n, it, 1);
    enter(p);
    if (__any_sync(kFull, stop_requested(*cv))) continue;
    const StepProblem& sp = steps[p];
    const uint32_t base = uint32_t(it - sp.u_items_begin) * R;
    const uint32_t nrows = min(R, sp.u_count - base);
    uint32_t en = 0;
#pragma unroll
    for (int q = 0; q < 32; ++q) en |= ((sp.u_ops >> (q & 3)) & 1u & (uint32_t(q >> 2) < nrows ? 1u : 0u)) << q;
    if (cv->vecs <= 8u) {
      const uint32_t opc[4] = {kNot, kNext, kFuture, kGlobally};
      const uint64_t d = pack_desc(opc[lane & 3], sp.u_first + base + uint32_t(lane >> 2), 0);
      bw.ids.inserted += batch_a<W>(*cv, ca, d, (en >> lane) & 1u);
    } else {
      RowGenD<W> gen;
      gen.cv = cv;
      gen.id0 = sp.u_first + base;
      PD::template batch<false>(*cv, gen, int(4 * nrows), en, bw.pend, bw.ids);
    }
    bw.built += __popc(en);
  }
  // 3. binary operators, R pairs (4R candidates) per item
  for (unsigned long long it = grab(&hdr->work[2].v); it < hdr->total_b; it = grab(&hdr->work[2].v)) {
    const int p = find_problem(steps, n, it, 2);
    enter(p);
    if (__any_sync(kFull, stop_requested(*cv))) continue;
    const StepProblem& sp = steps[p];
    const unsigned long long g0 = (it - sp.b_items_begin) * (unsigned long long)R;
    uint32_t ok = 0;
    if (lane < int(R)) {
      unsigned long long pidx = g0 + lane;
      int si = 0;
      while (si + 1 < int(sp.n_splits) && sp.s[si + 1].pairs_begin <= pidx) ++si;
      const Split& S = sp.s[si];
      const unsigned long long end = S.pairs_begin + S.pairs;
      bool valid = pidx < end;
      uint2 pr = make_uint2(0, 0);
      if (valid) {
        const uint2 ab = split_pair(S, pidx - S.pairs_begin, cv->vecs > 8u);  // path D jobs: large side outer
        pr = make_uint2(S.left_start + ab.x, S.right_start + ab.y);
      }
      s_pairs[wib][lane] = pr;
      ok = valid ? 1u : 0u;
    }
    const uint32_t pv = __ballot_sync(kFull, ok != 0u) & 0xFFu;
    __syncwarp();
    uint32_t en = 0;
#pragma unroll
    for (int q = 0; q < 32; ++q) en |= (((pv >> (q >> 2)) & 1u) & ((sp.b_ops >> (q & 3)) & 1u)) << q;
    if (en) {
      if (cv->vecs <= 8u) {
        const uint2 pr = s_pairs[wib][lane >> 2];
        const int o = lane & 3;  // and, or, U(a, b), U(b, a)
        const uint64_t d = o == 0 ? pack_desc(kAnd, pr.x, pr.y)
                         : o == 1 ? pack_desc(kOr, pr.x, pr.y)
                         : o == 2 ? pack_desc(kUntil, pr.x, pr.y) : pack_desc(kUntil, pr.y, pr.x);
        bw.ids.inserted += batch_a<W>(*cv, ca, d, (en >> lane) & 1u);
      } else {
        PairGenD<W> gen;
        gen.cv = cv;
        gen.pairs = s_pairs[wib];
        PD::template batch<true>(*cv, gen, int(4 * R), en, bw.pend, bw.ids);
      }
      bw.built += __popc(en);
    }
    __syncwarp();
  }
  bw.leave(cv);
}

// Reset the counters of every problem of a step (thread per problem) and the
// step's work counters.
static __global__ void k_batch_begin(StepHeader* hdr, const StepProblem* steps, int n_max) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p == 0) hdr->work[0].v = hdr->work[1].v = hdr->work[2].v = 0;
  if (p >= n_max || p >= hdr->n) return;  // only the step's problems (slots past n are stale)
  DevCounters* c = steps[p].cv.ctr;
  c->full = 0;
  c->solved = 0;
  c->error = 0;
  c->defer_n[0] = 0;
  c->defer_n[1] = 0;
  c->defer_overflow = 0;
  c->holes_n = 0;
  for (int i = 0; i < kLaunchKinds; ++i) c->built_k[i] = c->inserted_k[i] = 0;
  c->sol = ~0ull;
  c->timed_out = 0;
  for (int i = 0; i < 8; ++i) c->work[i] = 0;  // tile counters of one-problem launches in the step
}

// Hole fixup of a batch step: warp per (problem, src, dst) move, then each
// problem's entry count (dense end) is set.
static __global__ void __launch_bounds__(256) k_batch_fixup(const StepProblem* steps, const uint4* moves, unsigned n,
                                                            const unsigned* dense_end, int n_problems) {
  const int lane = threadIdx.x & 31;
  const unsigned warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned nwarps = (gridDim.x * blockDim.x) >> 5;
  for (unsigned m = warp; m < n; m += nwarps) {
    const CacheView& cv = steps[moves[m].x].cv;
    const unsigned src = moves[m].y, dst = moves[m].z;
    const uint4* a = cv.arena + size_t(src) * cv.vecs;
    uint4* b = cv.arena + size_t(dst) * cv.vecs;
    for (unsigned v = lane; v < cv.vecs; v += 32) b[v] = a[v];
    if (lane == 0) {
      cv.prov[dst] = cv.prov[src];
      cv.homes[dst] = cv.homes[src];
      const unsigned sp = cv.slotpos[src];
      cv.slotpos[dst] = sp;
      const unsigned long long old = cv.table[sp];
      if (uint32_t(old) == src + 1u) cv.table[sp] = (old & 0xFFFFFFFF00000000ull) | (unsigned long long)(dst + 1u);
      else atomicExch(&cv.ctr->error, 3u);
    }
  }
}

static __global__ void k_batch_set_entries(const StepProblem* steps, const unsigned* dense_end, int n) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n || dense_end[p] == 0xFFFFFFFFu) return;
  steps[p].cv.ctr->n_entries = dense_end[p];
  steps[p].cv.ctr->holes_n = 0;
}

// ===========================================================================
// Hole fixup: after a level, move the entries that lie above the level's dense
// end into the holes below it: copy the CM row, its provenance and slot index,
// and repoint the table slot to the new id. A warp takes kFixupMoves moves at
// a time with their loads in flight together (a move is a chain of dependent
// loads: the move, the row or the slot index, the slot). Sources lie at or
// above the dense end and destinations below it, so the moves are disjoint.
// ===========================================================================
constexpr int kFixupMoves = 4;

static __global__ void __launch_bounds__(256) k_fixup(CacheView cv, const uint2* moves, unsigned n,
                                                      const unsigned* n_dev) {
  constexpr int G = kFixupMoves;
  const int lane = threadIdx.x & 31;
  const unsigned warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned nwarps = (gridDim.x * blockDim.x) >> 5;
  if (n_dev) n = *n_dev;  // planned on the device (k_hole_plan)
  for (unsigned m0 = warp * G; m0 < n; m0 += nwarps * G) {
    const unsigned g = min(unsigned(G), n - m0);
    uint2 mv[G];
#pragma unroll
    for (int j = 0; j < G; ++j) mv[j] = j < int(g) ? moves[m0 + j] : make_uint2(0u, 0u);
    for (unsigned v0 = 0; v0 < cv.vecs; v0 += 32) {
      const unsigned v = v0 + unsigned(lane);
      uint4 t[G];
#pragma unroll
      for (int j = 0; j < G; ++j)
        if (j < int(g) && v < cv.vecs) t[j] = cv.arena[size_t(mv[j].x) * cv.vecs + v];
#pragma unroll
      for (int j = 0; j < G; ++j)
        if (j < int(g) && v < cv.vecs) cv.arena[size_t(mv[j].y) * cv.vecs + v] = t[j];
    }
    // lane j: provenance, lane G + j: hash home, lane 2G + j: slot of move j
    const int j = lane % G, role = lane / G;
    if (j < int(g)) {
      unsigned src = 0, dst = 0;  // mv[j], selected in registers
#pragma unroll
      for (int q = 0; q < G; ++q)
        if (q == j) {
          src = mv[q].x;
          dst = mv[q].y;
        }
      if (role == 0) cv.prov[dst] = cv.prov[src];
      else if (role == 1) cv.homes[dst] = cv.homes[src];
      else if (role == 2) {
        const unsigned sp = cv.slotpos[src];
        cv.slotpos[dst] = sp;
        const unsigned long long old = cv.table[sp];
        if (uint32_t(old) == src + 1u) cv.table[sp] = (old & 0xFFFFFFFF00000000ull) | (unsigned long long)(dst + 1u);
        else atomicExch(&cv.ctr->error, 3u);
      }
    }
  }
}

// Exclusive prefix sum over a block of exactly 1024 threads, one value per
// thread; *total receives the block's sum (the same in every thread).
__device__ __forceinline__ unsigned block_scan_1024(unsigned v, unsigned* total) {
  __shared__ unsigned s_w[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_w[w] = x;
  __syncthreads();
  if (w == 0) {
    unsigned t = s_w[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(kFull, t, o);
      if (lane >= o) t += y;
    }
    s_w[lane] = t;
  }
  __syncthreads();
  const unsigned before = w ? s_w[w - 1] : 0u;
  *total = s_w[31];
  __syncthreads();  // s_w is reused by the next call
  return before + x - v;
}

// Hole plan of a level on the device, in two launches (no host round trip).
// The hole log holds the id ranges [x, y) that warps reserved but left unused;
// clipped to the level's range [start, total) they cover H ids, so the level's
// dense end is total - H. The entries in [dense_end, total) (ids in no hole,
// in id order) are the sources and the hole ids below dense_end (in log order)
// the destinations of the moves, paired by rank: both lists have the same
// length. Each logged range is at most 32 ids (a warp reserves at most 32 ids
// at a time), so H <= 32 x hole_cap and the bitmap of [dense_end, total) fits
// hole_cap words.
//
// Scratch layout (3 x hole_cap + 32 words): header [16] = {H, dense_end,
// words, n}, bits [hole_cap] (holes in [dense_end, total)), word_pref
// [hole_cap + 1] (live entries before each bitmap word), range_pref
// [hole_cap + 1] (destinations before each logged range).
struct HoleScratch {
  unsigned* base;
  unsigned cap;
  __device__ unsigned* hdr() const { return base; }
  __device__ unsigned* bits() const { return base + 16; }
  __device__ unsigned* word_pref() const { return base + 16 + cap; }
  __device__ unsigned* range_pref() const { return base + 16 + 2 * cap + 1; }
};

__device__ __forceinline__ unsigned hole_live_word(const unsigned* bits, unsigned w, unsigned words, unsigned H) {
  unsigned m = ~__ldcg(bits + w);
  if (w == words - 1u && (H & 31u)) m &= (1u << (H & 31u)) - 1u;
  return m;
}

// Plan: one block of exactly 1024 threads. Sets ctr->moves_n (0 on an
// inconsistent log, with ctr->error = 4), ctr->n_entries = dense_end and
// ctr->holes_n = 0.
static __global__ void __launch_bounds__(1024) k_hole_plan(DevCounters* ctr, const uint2* holes, unsigned hole_cap,
                                                           unsigned start, unsigned max_entries, HoleScratch sc,
                                                           unsigned move_cap) {
  const unsigned t = threadIdx.x, T = blockDim.x;
  const unsigned n = ctr->holes_n;
  const unsigned total = min(ctr->n_entries, max_entries);
  if (n > hole_cap || total < start) {  // an overflowed log (its warp set error 2) or no level range
    if (t == 0) {
      ctr->moves_n = 0;
      atomicExch(&ctr->error, 4u);
    }
    return;
  }
  // 1. H and the dense end
  unsigned h = 0;
#pragma unroll 8
  for (unsigned i = t; i < n; i += T) {
    const uint2 r = holes[i];
    const unsigned lo = max(r.x, start), hi = min(r.y, total);
    if (lo < hi) h += hi - lo;
  }
  unsigned H;
  block_scan_1024(h, &H);
  const unsigned words = (H + 31u) >> 5;
  if (H > total - start || words > hole_cap) {
    if (t == 0) {
      ctr->moves_n = 0;
      atomicExch(&ctr->error, 4u);
    }
    return;
  }
  const unsigned dense_end = total - H;
  unsigned* bits = sc.bits();
  for (unsigned w = t; w < words; w += T) bits[w] = 0u;
  __syncthreads();
  // 2. the holes at or above the dense end, as a bitmap of [dense_end, total):
  // one masked OR per bitmap word a range touches (two at most), not one per
  // id (the top of a level's range is mostly holes, and the ORs of one block
  // are served one after another)
#pragma unroll 8
  for (unsigned i = t; i < n; i += T) {
    const uint2 r = holes[i];
    const unsigned lo = max(max(r.x, start), dense_end), hi = min(r.y, total);
    if (lo >= hi) continue;
    unsigned a = lo - dense_end;
    const unsigned b = hi - dense_end;
    while (a < b) {
      const unsigned o = a & 31u, nb = min(32u - o, b - a);
      atomicOr(&bits[a >> 5], (nb == 32u ? 0xFFFFFFFFu : ((1u << nb) - 1u)) << o);
      a += nb;
    }
  }
  __syncthreads();
  // 3. live entries before each bitmap word (contiguous words per thread)
  const unsigned per_w = (words + T - 1u) / T;
  const unsigned w0 = min(t * per_w, words), w1 = min(w0 + per_w, words);
  unsigned c = 0;
#pragma unroll 8
  for (unsigned w = w0; w < w1; ++w) c += unsigned(__popc(hole_live_word(bits, w, words, H)));
  unsigned n_src;
  unsigned o = block_scan_1024(c, &n_src);
  unsigned* wp = sc.word_pref();
#pragma unroll 8
  for (unsigned w = w0; w < w1; ++w) {
    wp[w] = o;
    o += unsigned(__popc(hole_live_word(bits, w, words, H)));
  }
  // 4. destinations before each logged range (contiguous ranges per thread)
  const unsigned per_r = (n + T - 1u) / T;
  const unsigned r0 = min(t * per_r, n), r1 = min(r0 + per_r, n);
  unsigned d = 0;
#pragma unroll 8
  for (unsigned i = r0; i < r1; ++i) {
    const uint2 r = holes[i];
    const unsigned lo = max(r.x, start), hi = min(min(r.y, total), dense_end);
    if (lo < hi) d += hi - lo;
  }
  unsigned n_dst;
  unsigned od = block_scan_1024(d, &n_dst);
  unsigned* rp = sc.range_pref();
#pragma unroll 8
  for (unsigned i = r0; i < r1; ++i) {
    rp[i] = od;
    const uint2 r = holes[i];
    const unsigned lo = max(r.x, start), hi = min(min(r.y, total), dense_end);
    if (lo < hi) od += hi - lo;
  }
  if (t == 0) {
    if (n_src != n_dst || n_src > move_cap) {
      ctr->moves_n = 0;
      atomicExch(&ctr->error, 4u);
      return;
    }
    wp[words] = n_src;
    rp[n] = n_dst;
    unsigned* hd = sc.hdr();
    hd[0] = H;
    hd[1] = dense_end;
    hd[2] = words;
    hd[3] = n;
    ctr->moves_n = n_src;
    ctr->n_entries = dense_end;
    ctr->holes_n = 0;
  }
}

// Moves, by scatter: the r-th live entry of [dense_end, total) is the source
// and the r-th hole id below dense_end the destination of move r. Items
// 0 .. words-1 are the bitmap words (each writes the sources of its live
// entries from the word's prefix), items words .. words+n-1 the logged ranges
// (each writes the destinations of its ids below dense_end from the range's
// prefix). Sources fill moves[r].x and destinations moves[r].y.
static __global__ void __launch_bounds__(256) k_hole_moves(const DevCounters* ctr, const uint2* holes,
                                                           unsigned start, HoleScratch sc, uint2* moves) {
  const unsigned m = ctr->moves_n;
  if (m == 0) return;
  const unsigned* hd = sc.hdr();
  const unsigned H = hd[0], dense_end = hd[1], words = hd[2], n = hd[3];
  const unsigned* bits = sc.bits();
  const unsigned* wp = sc.word_pref();
  const unsigned* rp = sc.range_pref();
  unsigned* out = reinterpret_cast<unsigned*>(moves);
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < words + n; i += gridDim.x * blockDim.x) {
    if (i < words) {
      unsigned live = hole_live_word(bits, i, words, H);
      unsigned r = __ldcg(wp + i);
      for (; live && r < m; live &= live - 1u, ++r) out[2 * size_t(r)] = dense_end + i * 32u + unsigned(__ffs(live) - 1);
    } else {
      const unsigned h = i - words;
      const uint2 rg = holes[h];
      const unsigned lo = max(rg.x, start), hi = min(min(rg.y, dense_end + H), dense_end);
      unsigned r = __ldcg(rp + h);
      for (unsigned id = lo; id < hi && r < m; ++id, ++r) out[2 * size_t(r) + 1] = id;
    }
  }
}

// ===========================================================================
// Table rebuild: re-insert the published slots of entries below live_end into
// a cleared table of any capacity. An entry's home slot comes from the low
// word of its hash (homes[]), so no CM is read; tags move unchanged. Slots of
// entries at or above live_end (a level being undone), tombstones and pending
// claims are dropped.
// ===========================================================================
static __global__ void __launch_bounds__(256) k_rehash(const unsigned long long* old_t, unsigned long long old_cap,
                                                       unsigned long long* new_t, unsigned long long new_mask,
                                                       const unsigned* homes, unsigned* slotpos, unsigned live_end,
                                                       unsigned* error) {
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < old_cap; i += stride) {
    const unsigned long long v = old_t[i];
    const uint32_t low = uint32_t(v);
    if (v == 0ull || low >= kSlotTomb) continue;
    const uint32_t id = low - 1u;
    if (id >= live_end) continue;
    unsigned long long pos = homes[id] & new_mask;
    unsigned long long it = 0;
    for (; it <= new_mask; ++it, pos = (pos + 1) & new_mask)
      if (atomicCAS(new_t + pos, 0ull, v) == 0ull) break;
    if (it > new_mask) {
      atomicExch(error, 5u);
      continue;
    }
    slotpos[id] = unsigned(pos);
  }
}

// ===========================================================================
// Formula evaluation with the paper's log-step operators: one thread per trace
// word walks a postorder node list (x = op, y = left node, z = right node,
// w = proposition); scratch holds one row of words per node.
// ===========================================================================
template <typename W>
__global__ void k_eval(const W* atoms, const W* lenmask, unsigned words, unsigned planes, const int4* nodes,
                       int n_nodes, int steps, W* scratch, W* out) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;  // word slot of a plane (a trace)
  if (t >= words) return;
  const size_t row = size_t(words) * planes;  // one CM: planes x words
  constexpr int kBits = int(sizeof(W) * 8);
  for (int i = 0; i < n_nodes; ++i) {
    const int4 nd = nodes[i];
    const uint32_t op = uint32_t(nd.x);
    W* dst = scratch + size_t(i) * row;
    if (op == kAtom) {
      for (unsigned j = 0; j < planes; ++j) dst[j * words + t] = atoms[size_t(nd.w) * row + j * words + t];
      continue;
    }
    const W* a = scratch + size_t(nd.y) * row;
    const W* b = nd.z >= 0 ? scratch + size_t(nd.z) * row : a;
    // planes from the last: later positions carry into earlier words
    W later = 0, cin = 0;
    for (int j = int(planes) - 1; j >= 0; --j) {
      const size_t o = size_t(j) * words + t;
      const W lm = lenmask[o];
      W v;
      switch (op) {
        case kNext:
          v = (a[o] << 1) | (size_t(j) + 1 < planes ? (a[o + words] >> (kBits - 1)) : W(0));
          break;
        case kFuture:
          v = w_future_logstep<W>(a[o], steps) | (later ? lm : W(0));
          later |= a[o];
          break;
        case kGlobally: {
          const W na = ~a[o] & lm;
          v = ~(w_future_logstep<W>(na, steps) | (later ? lm : W(0))) & lm;
          later |= na;
          break;
        }
        case kUntil: {
          // within the word, or phi to the word's end and U where the next word starts
          const W phi_to_end = ~w_future_logstep<W>(~a[o], steps);
          v = w_until_logstep<W>(a[o], b[o], steps) | (cin ? phi_to_end : W(0));
          cin = v >> (kBits - 1);
          break;
        }
        default:
          v = w_op_logstep<W>(op, a[o], b[o], lm, steps);
      }
      dst[o] = v;
    }
  }
  for (unsigned j = 0; j < planes; ++j) out[j * words + t] = scratch[size_t(n_nodes - 1) * row + j * words + t];
}

// ===========================================================================
// Launchers
// ===========================================================================
inline int occupancy_blocks(const void* fn, int threads, size_t smem) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, smem) != cudaSuccess || n < 1) n = 1;
  return n;
}

template <typename W, int V>
struct LaunchA {
  static cudaError_t desc_list(const CacheView& cv, const unsigned long long* list, const unsigned int* list_n,
                               unsigned int cap, unsigned int atoms, const LaunchCfg& lc) {
    const unsigned n = list ? cap : atoms;
    const unsigned blocks = std::max(1u, std::min((n + 255u) / 256u, unsigned(lc.sms * 8)));
    k_desc_a<W, V><<<blocks, 256, 0, lc.stream>>>(cv, list, list_n, cap, atoms);
    return cudaGetLastError();
  }
  static cudaError_t unary(const CacheView& cv, uint32_t first, uint32_t count, uint32_t ops, const LaunchCfg& lc) {
    static int occ = occupancy_blocks((const void*)k_unary_a<W, V>, 256, 0);
    const unsigned blocks = std::max(1u, std::min((count + 255u) / 256u, unsigned(lc.sms * occ)));
    k_unary_a<W, V><<<blocks, 256, 0, lc.stream>>>(cv, first, count, ops);
    return cudaGetLastError();
  }
  static cudaError_t binary(const CacheView& cv, const BinaryPlan& plan, const LaunchCfg& lc) {
    static int occ = occupancy_blocks((const void*)k_binary_a<W, V>, 256, 0);
    const unsigned long long want = (plan.total_pairs + 255ull) / 256ull;
    const unsigned blocks = unsigned(std::max(1ull, std::min(want, (unsigned long long)lc.sms * occ)));
    k_binary_a<W, V><<<blocks, 256, 0, lc.stream>>>(cv, plan);
    return cudaGetLastError();
  }
};

template <typename W>
struct LaunchC {
  static constexpr size_t kUnarySmem = size_t(8) * (kUnaryRowsC * 32 + PathC<W>::kStage) * sizeof(uint4);
  static constexpr size_t kDescSmem =
      size_t(8) * (PathC<W>::kStage + kDescBatch * 32 + kDescBatch / 2) * sizeof(uint4);
  static constexpr size_t kStageSmem = size_t(8) * PathC<W>::kStage * sizeof(uint4);
  static cudaError_t desc_list(const CacheView& cv, const unsigned long long* list, const unsigned int* list_n,
                               unsigned int cap, unsigned int atoms, const LaunchCfg& lc) {
    static bool once = (cudaFuncSetAttribute((const void*)k_desc_c<W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(kDescSmem)), true);
    (void)once;
    static int occ = occupancy_blocks((const void*)k_desc_c<W>, 256, kDescSmem);
    const unsigned n = list ? cap : atoms;
    const unsigned per_block = 8u * unsigned(kDescBatch);
    const unsigned blocks = std::max(1u, std::min((n + per_block - 1u) / per_block, unsigned(lc.sms * occ)));
    k_desc_c<W><<<blocks, 256, kDescSmem, lc.stream>>>(cv, list, list_n, cap, atoms);
    return cudaGetLastError();
  }
  static cudaError_t unary(const CacheView& cv, uint32_t first, uint32_t count, uint32_t ops, const LaunchCfg& lc) {
    static bool once = (cudaFuncSetAttribute((const void*)k_unary_c<W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(kUnarySmem)), true);
    (void)once;
    static int occ = occupancy_blocks((const void*)k_unary_c<W>, 256, kUnarySmem);
    const unsigned blocks = std::max(1u, std::min((count + 63u) / 64u, unsigned(lc.sms * occ)));
    k_unary_c<W><<<blocks, 256, kUnarySmem, lc.stream>>>(cv, first, count, ops);
    return cudaGetLastError();
  }
  static cudaError_t binary(const CacheView& cv, const BinaryPlan& plan, const LaunchCfg& lc) {
    static bool once = (cudaFuncSetAttribute((const void*)k_binary_c<W>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024), true);
    static bool once_s = (cudaFuncSetAttribute((const void*)k_binary_small_c<W>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, int(kUnarySmem)), true);
    (void)once;
    (void)once_s;
    // Splits with a small side go to k_binary_small_c (larger level as the
    // per-warp staged operand, in chunks of 8 rows); the others keep the
    // block tiles of k_binary_c. Both plans keep the splits' order.
    BinaryPlan big = plan, small = plan;
    big.n_splits = small.n_splits = 0;
    big.total_tiles = small.total_tiles = 0;
    static int occ_b = occupancy_blocks((const void*)k_binary_c<W>, 256, size_t(32) * 32 * sizeof(uint4) + kStageSmem);
    static int occ_s = occupancy_blocks((const void*)k_binary_small_c<W>, 256, kUnarySmem);
    unsigned long long chunks = 0;
    for (int i = 0; i < plan.n_splits; ++i) {
      const Split& sp = plan.s[i];
      if (!sp.tri && sp.left_n < kSmallSplitRows) chunks += (std::max(sp.left_n, sp.right_n) + 7u) / 8u;
    }
    // a few work items per warp even at small levels: row groups of the small
    // side when there are fewer chunks than that
    const unsigned long long want_s = 4ull * lc.sms * occ_s * 8ull;
    const unsigned long long per_chunk = chunks >= want_s || chunks == 0 ? 1ull : (want_s + chunks - 1) / chunks;
    // block tiles of 32 rows, or 16 / 8 when 32 gives too few tiles to fill the
    // GPU; a tile the caller fixed (lsyn_config.tile_rows) is kept as it is
    auto tiles_of = [&](uint32_t t) {
      unsigned long long n = 0;
      for (int i = 0; i < plan.n_splits; ++i) {
        const Split& sp = plan.s[i];
        if (sp.tri || sp.left_n >= kSmallSplitRows)
          n += (unsigned long long)((sp.left_n + t - 1) / t) * ((sp.right_n + t - 1) / t);
      }
      return n;
    };
    uint32_t tile = plan.tile;
    while (!plan.tile_fixed && tile > 8u && tiles_of(tile) < 2ull * lc.sms * occ_b) tile /= 2u;
    big.tile = tile;
    for (int i = 0; i < plan.n_splits; ++i) {
      Split sp = plan.s[i];
      if (!sp.tri && sp.left_n < kSmallSplitRows) {
        if (sp.right_n > sp.left_n) {
          std::swap(sp.left_start, sp.right_start);
          std::swap(sp.left_n, sp.right_n);
        }
        sp.lt_tiles = (sp.left_n + 7u) / 8u;
        sp.group = std::max(1u, unsigned((sp.right_n + per_chunk - 1) / per_chunk));
        sp.rt_tiles = (sp.right_n + sp.group - 1) / sp.group;
        sp.tiles_begin = small.total_tiles;
        small.total_tiles += (unsigned long long)sp.lt_tiles * sp.rt_tiles;
        small.s[small.n_splits++] = sp;
      } else {
        sp.lt_tiles = (sp.left_n + tile - 1) / tile;
        sp.rt_tiles = (sp.right_n + tile - 1) / tile;
        sp.tiles_begin = big.total_tiles;
        big.total_tiles += (unsigned long long)sp.lt_tiles * sp.rt_tiles;
        big.s[big.n_splits++] = sp;
      }
    }
    if (big.n_splits > 0) {
      const size_t smem = size_t(big.tile) * 32 * sizeof(uint4) + kStageSmem;
      const int occ = occupancy_blocks((const void*)k_binary_c<W>, 256, smem);
      const unsigned long long blocks = std::max(1ull, std::min(big.total_tiles, (unsigned long long)lc.sms * occ));
      k_binary_c<W><<<unsigned(blocks), 256, smem, lc.stream>>>(cv, big);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    if (small.n_splits > 0) {
      const unsigned long long blocks =
          std::max(1ull, std::min((small.total_tiles + 7ull) / 8ull, (unsigned long long)lc.sms * occ_s));
      k_binary_small_c<W><<<unsigned(blocks), 256, kUnarySmem, lc.stream>>>(cv, small);
      return cudaGetLastError();
    }
    return cudaSuccess;
  }
};

template <typename W>
struct LaunchD {
  static cudaError_t desc_list(const CacheView& cv, const unsigned long long* list, const unsigned int* list_n,
                               unsigned int cap, unsigned int atoms, const LaunchCfg& lc) {
    static int occ = occupancy_blocks((const void*)k_desc_d<W>, 256, 0);
    const unsigned n = list ? cap : atoms;
    const unsigned per_block = 8u * unsigned(kDescBatchD);
    const unsigned blocks = std::max(1u, std::min((n + per_block - 1u) / per_block, unsigned(lc.sms * occ)));
    k_desc_d<W><<<blocks, 256, 0, lc.stream>>>(cv, list, list_n, cap, atoms);
    return cudaGetLastError();
  }
  static cudaError_t unary(const CacheView& cv, uint32_t first, uint32_t count, uint32_t ops, const LaunchCfg& lc) {
    const unsigned M = cv.vecs * 16u;
    if (cv.planes <= 1 && M >= kStagedMinBytes && M <= kStagedMaxBytes) {
      // one block per SM holding as many warps as rows fit its shared memory
      static int optin = [] {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
          v = 0;
        return v;
      }();
      const int dyn_cap = optin - 1024;  // room for the kernel's static shared memory
      const unsigned warps = dyn_cap > 0 ? std::min(unsigned(kStagedMaxWarps), unsigned(dyn_cap) / M) : 0u;
      if (warps >= 4u) {
        static const cudaError_t attr = cudaFuncSetAttribute((const void*)k_unary_ds<W>,
                                                             cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_cap);
        if (attr != cudaSuccess) return attr;
        const unsigned blocks = std::max(1u, std::min((count + warps - 1u) / warps, unsigned(lc.sms)));
        k_unary_ds<W><<<blocks, 32u * warps, size_t(warps) * M, lc.stream>>>(cv, first, count, ops);
        return cudaGetLastError();
      }
    }
    static int occ = occupancy_blocks((const void*)k_unary_d<W>, 256, 0);
    const unsigned blocks = std::max(1u, std::min((count + 63u) / 64u, unsigned(lc.sms * occ)));
    k_unary_d<W><<<blocks, 256, 0, lc.stream>>>(cv, first, count, ops);
    return cudaGetLastError();
  }
  static cudaError_t binary(const CacheView& cv, const BinaryPlan& plan, const LaunchCfg& lc) {
    static int occ = occupancy_blocks((const void*)k_binary_d<W>, 256, 0);
    const unsigned long long want = (plan.total_pairs + 63ull) / 64ull;
    const unsigned blocks = unsigned(std::max(1ull, std::min(want, (unsigned long long)lc.sms * occ)));
    k_binary_d<W><<<blocks, 256, 0, lc.stream>>>(cv, plan);
    return cudaGetLastError();
  }
};

template <typename W>
int Kernels<W>::path_for(unsigned vecs) {
  if (vecs == 1 || vecs == 2 || vecs == 4 || vecs == 8) return 1;
  if (vecs == 32) return 2;
  if (vecs > 32 && vecs % 32 == 0 && vecs <= 4096) return 3;
  return 0;
}

#define LSYN_DISPATCH(vecs, CALL)                       \
  switch (vecs) {                                       \
    case 1: return LaunchA<W, 1>::CALL;                 \
    case 2: return LaunchA<W, 2>::CALL;                 \
    case 4: return LaunchA<W, 4>::CALL;                 \
    case 8: return LaunchA<W, 8>::CALL;                 \
    case 32: return LaunchC<W>::CALL;                   \
    default:                                            \
      if (vecs > 32 && vecs % 32 == 0) return LaunchD<W>::CALL; \
      return cudaErrorInvalidValue;                     \
  }

template <typename W>
cudaError_t Kernels<W>::desc_list(const CacheView& cv, const unsigned long long* list, const unsigned int* list_n,
                                  unsigned int cap, unsigned int atoms, const LaunchCfg& lc) {
  LSYN_DISPATCH(cv.vecs, desc_list(cv, list, list_n, cap, atoms, lc))
}

template <typename W>
cudaError_t Kernels<W>::unary(const CacheView& cv, uint32_t first, uint32_t count, uint32_t ops,
                              const LaunchCfg& lc) {
  LSYN_DISPATCH(cv.vecs, unary(cv, first, count, ops, lc))
}

template <typename W>
cudaError_t Kernels<W>::binary(const CacheView& cv, const BinaryPlan& plan, const LaunchCfg& lc) {
  LSYN_DISPATCH(cv.vecs, binary(cv, plan, lc))
}

template <typename W>
cudaError_t Kernels<W>::batch_begin(StepHeader* hdr, const StepProblem* steps, int n, const LaunchCfg& lc) {
  k_batch_begin<<<(std::max(n, 1) + 255) / 256, 256, 0, lc.stream>>>(hdr, steps, n);
  return cudaGetLastError();
}

template <typename W>
cudaError_t Kernels<W>::batch_run(StepHeader* hdr, const StepProblem* steps, const LaunchCfg& lc, int blocks_per_sm,
                                  int vpt) {
  const unsigned grid = unsigned(lc.sms * std::max(1, blocks_per_sm));
  if (vpt >= 2) k_batch_run<W, 2><<<grid, 256, 0, lc.stream>>>(hdr, steps);
  else k_batch_run<W, 1><<<grid, 256, 0, lc.stream>>>(hdr, steps);
  return cudaGetLastError();
}

template <typename W>
cudaError_t Kernels<W>::batch_fixup(const StepProblem* steps, const uint4* moves, unsigned n, const unsigned* dense_end,
                                    int n_problems, const LaunchCfg& lc) {
  if (n) {
    const unsigned blocks = std::max(1u, std::min((n + 7u) / 8u, unsigned(lc.sms * 8)));
    k_batch_fixup<<<blocks, 256, 0, lc.stream>>>(steps, moves, n, dense_end, n_problems);
  }
  k_batch_set_entries<<<(std::max(n_problems, 1) + 255) / 256, 256, 0, lc.stream>>>(steps, dense_end, n_problems);
  return cudaGetLastError();
}

template <typename W>
cudaError_t Kernels<W>::rehash(const unsigned long long* old_t, unsigned long long old_cap, unsigned long long* new_t,
                               unsigned long long new_cap, const unsigned* homes, unsigned* slotpos,
                               unsigned live_end, unsigned* error, const LaunchCfg& lc) {
  if (old_cap == 0) return cudaSuccess;
  const unsigned blocks = unsigned(std::min<unsigned long long>((old_cap + 255) / 256, (unsigned long long)lc.sms * 8));
  k_rehash<<<blocks, 256, 0, lc.stream>>>(old_t, old_cap, new_t, new_cap - 1, homes, slotpos, live_end, error);
  return cudaGetLastError();
}

template <typename W>
cudaError_t Kernels<W>::fixup(const CacheView& cv, const uint2* moves, unsigned n, const LaunchCfg& lc) {
  if (n == 0) return cudaSuccess;
  const unsigned per_block = 8u * unsigned(kFixupMoves);
  const unsigned blocks = std::max(1u, std::min((n + per_block - 1u) / per_block, unsigned(lc.sms * 8)));
  k_fixup<<<blocks, 256, 0, lc.stream>>>(cv, moves, n, nullptr);
  return cudaGetLastError();
}

template <typename W>
cudaError_t Kernels<W>::close_holes(const CacheView& cv, unsigned start, unsigned* bits, uint2* moves,
                                    unsigned move_cap, const LaunchCfg& lc) {
  const HoleScratch sc{bits, cv.hole_cap};
  k_hole_plan<<<1, 1024, 0, lc.stream>>>(cv.ctr, cv.holes, cv.hole_cap, start, cv.max_entries, sc, move_cap);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_hole_moves<<<unsigned(lc.sms * 4), 256, 0, lc.stream>>>(cv.ctr, cv.holes, start, sc, moves);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // The move count is known on the device only: a full grid (warps past it exit at once).
  k_fixup<<<unsigned(lc.sms * 8), 256, 0, lc.stream>>>(cv, moves, 0u, &cv.ctr->moves_n);
  return cudaGetLastError();
}

template <typename W>
cudaError_t Kernels<W>::eval(const uint4* atoms, const uint4* lenmask, unsigned plane_vecs, unsigned planes,
                             const int4* nodes, int n_nodes, int steps, W* scratch, W* out, const LaunchCfg& lc) {
  const unsigned words = plane_vecs * unsigned(sizeof(uint4) / sizeof(W));
  k_eval<W><<<(words + 127u) / 128u, 128, 0, lc.stream>>>(reinterpret_cast<const W*>(atoms),
                                                          reinterpret_cast<const W*>(lenmask), words, planes,
                                                          nodes, n_nodes, steps, scratch, out);
  return cudaGetLastError();
}

}  // namespace lsyn
