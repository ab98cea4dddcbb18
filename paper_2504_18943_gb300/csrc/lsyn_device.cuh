// Device code of the LTLf semantic enumerator: bitwise LTLf operators on
// characteristic-matrix words, the candidate hash, the specification check,
// the lock-free dedup-insert into the device-resident language cache, and the
// level kernels. Included once per word type by kernels_w32.cu / kernels_w64.cu
// with LSYN_WORD defined.
//
// Layout. A characteristic matrix (CM) is one word per trace, positives first,
// padded with zero words to `vecs` 16-byte vectors. Bit t of a trace word says
// whether the formula holds at position t ("Parallel enumeration of LTLf
// formulae on GPUs": characteristic sequence, least significant bit = position
// 0). Padding bits (positions >= length, padding traces) are zero for every
// formula.
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
//   not  : complement, masked to the trace length (nothing holds past the end)
//   X    : shift toward position 0 by one (the last position becomes false)
//   F    : suffix-OR by doubling shifts: after the step with shift s every bit
//          t holds the OR of positions [t, t + 2s)
//   G    : not F not (suffix-AND), masked to the trace length
//   U    : log-step doubling. R starts as psi and A as phi; the step with
//          shift s sets R(t) |= A(t) & R(t + s) and then A(t) &= A(t + s), so
//          afterwards R(t) says "psi at some j in [t, t + 2s) and phi on
//          [t, j)" and A(t) says "phi on [t, t + 2s)".
// `steps` is the smallest s with 2^s >= the longest trace.
// ---------------------------------------------------------------------------
template <typename W>
__device__ __forceinline__ W w_future(W a, int steps) {
#pragma unroll
  for (int s = 0; s < WordInfo<W>::kMaxSteps; ++s)
    if (s < steps) a |= a >> (1u << s);
  return a;
}

template <typename W>
__device__ __forceinline__ W w_until(W phi, W psi, int steps) {
  W r = psi;
#pragma unroll
  for (int s = 0; s < WordInfo<W>::kMaxSteps; ++s) {
    if (s < steps) {
      const unsigned sh = 1u << s;
      r |= phi & (r >> sh);
      phi &= phi >> sh;
    }
  }
  return r;
}

template <typename W>
__device__ __forceinline__ W w_op(uint32_t op, W a, W b, W lm, int steps) {
  switch (op) {
    case kNot: return ~a & lm;
    case kAnd: return a & b;
    case kOr: return a | b;
    case kNext: return a >> 1;
    case kFuture: return w_future<W>(a, steps);
    case kGlobally: return ~w_future<W>(~a & lm, steps) & lm;
    case kUntil: return w_until<W>(a, b, steps);
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
// from examples", separation): bit 0 of every real trace word must equal its
// label (1 for P, 0 for N). Returns nonzero on a mismatch in this vector.
__device__ __forceinline__ uint32_t spec_bad(uint4 c, uint4 lab, uint4 care) {
  return ((c.x ^ lab.x) & care.x) | ((c.y ^ lab.y) & care.y) | ((c.z ^ lab.z) & care.z) |
         ((c.w ^ lab.w) & care.w);
}

__device__ __forceinline__ uint32_t v_ne(uint4 a, uint4 b) {
  return (a.x ^ b.x) | (a.y ^ b.y) | (a.z ^ b.z) | (a.w ^ b.w);
}

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ bool stop_requested(const CacheView& cv) {
  return cv.early_exit && ld_relaxed_u32(&cv.ctr->solved) != 0u;
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
  __device__ static void process(const CacheView& cv, const Consts& s, const uint4 (&c)[V], uint64_t desc) {
    uint32_t lo = 0, hi = 0, bad = 0;
#pragma unroll
    for (int v = 0; v < V; ++v) {
      h_acc(c[v], s.key[v], s.mul[v], lo, hi);
      bad |= spec_bad(c[v], s.lab[v], s.care[v]);
    }
    if (bad == 0) record_solution(cv, desc);
    const uint64_t h = h_fin(hi, lo);
    const unsigned long long tag = (h >> 32) << 32;
    unsigned long long pos = h & cv.table_mask;
    for (unsigned long long it = 0; it <= cv.table_mask; ++it, pos = (pos + 1) & cv.table_mask) {
      unsigned long long* slot = cv.table + pos;
      unsigned long long sv = ld_acquire(slot);
      if (sv == 0ull) {
        sv = atomicCAS(slot, 0ull, tag | kSlotPending);
        if (sv == 0ull) {
          const unsigned id = atomicAdd(&cv.ctr->n_entries, 1u);
          if (id >= cv.max_entries) {
            st_release(slot, tag | kSlotTomb);
            atomicExch(&cv.ctr->full, 1u);
            return;
          }
          uint4* dst = cv.arena + size_t(id) * cv.vecs;
#pragma unroll
          for (int v = 0; v < V; ++v) dst[v] = c[v];
          cv.prov[id] = desc;
          __threadfence();
          st_release(slot, tag | (unsigned long long)(id + 1u));
          return;
        }
      }
      if ((sv & 0xFFFFFFFF00000000ull) != tag) continue;
      const uint32_t low = uint32_t(sv);
      if (low == kSlotPending) { defer(cv, desc); return; }
      if (low == kSlotTomb) continue;
      const uint4* src = row_ptr(cv, low - 1u);
      uint32_t ne = 0;
#pragma unroll
      for (int v = 0; v < V; ++v) ne |= v_ne(__ldcg(src + v), c[v]);
      if (ne == 0) return;  // duplicate: an equal CM is already cached
    }
    atomicExch(&cv.ctr->error, 1u);
  }

  __device__ static void candidate(const CacheView& cv, const Consts& s, uint32_t op, const uint4 (&a)[V],
                                   const uint4 (&b)[V], uint64_t desc) {
    uint4 c[V];
#pragma unroll
    for (int v = 0; v < V; ++v) c[v] = v_op<W>(op, a[v], b[v], s.lm[v], cv.steps);
    process(cv, s, c, desc);
  }
};

template <typename W, int V>
__global__ void __launch_bounds__(256) k_unary_a(CacheView cv, uint32_t first, uint32_t count, uint32_t ops) {
  using P = PathA<W, V>;
  __shared__ typename P::Consts s;
  P::load_consts(cv, &s);
  __syncthreads();
  unsigned long long built = 0;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
    if (stop_requested(cv)) break;
    const uint32_t id = first + i;
    uint4 a[V];
    P::load_row(row_ptr(cv, id), a);
    const uint32_t opc[4] = {kNot, kNext, kFuture, kGlobally};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (!((ops >> q) & 1u)) continue;
      P::candidate(cv, s, opc[q], a, a, pack_desc(opc[q], id, 0));
      ++built;
    }
  }
  if (built) atomicAdd(&cv.ctr->built, built);
}

template <typename W, int V>
__global__ void __launch_bounds__(256) k_binary_a(CacheView cv, BinaryPlan plan) {
  using P = PathA<W, V>;
  __shared__ typename P::Consts s;
  P::load_consts(cv, &s);
  __syncthreads();
  unsigned long long built = 0;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long p = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; p < plan.total_pairs;
       p += stride) {
    if (stop_requested(cv)) break;
    int sp = 0;
    while (sp + 1 < plan.n_splits && plan.s[sp + 1].pairs_begin <= p) ++sp;
    const Split& S = plan.s[sp];
    const unsigned long long local = p - S.pairs_begin;
    const uint32_t ia = uint32_t(local / S.right_n);
    const uint32_t ib = uint32_t(local - (unsigned long long)ia * S.right_n);
    if (S.tri && ia >= ib) continue;  // same level: unordered pairs a < b only
    const uint32_t a_id = S.left_start + ia, b_id = S.right_start + ib;
    uint4 a[V], b[V];
    P::load_row(row_ptr(cv, a_id), a);
    P::load_row(row_ptr(cv, b_id), b);
    if (plan.ops & 1u) { P::candidate(cv, s, kAnd, a, b, pack_desc(kAnd, a_id, b_id)); ++built; }
    if (plan.ops & 2u) { P::candidate(cv, s, kOr, a, b, pack_desc(kOr, a_id, b_id)); ++built; }
    if (plan.ops & 4u) { P::candidate(cv, s, kUntil, a, b, pack_desc(kUntil, a_id, b_id)); ++built; }
    if (plan.ops & 8u) { P::candidate(cv, s, kUntil, b, a, pack_desc(kUntil, b_id, a_id)); ++built; }
  }
  if (built) atomicAdd(&cv.ctr->built, built);
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
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    if (stop_requested(cv)) break;
    const uint64_t d = list ? list[i] : pack_desc(kAtom, i, 0);
    uint4 c[V];
    rebuild_a<W, V>(cv, s, d, c);
    P::process(cv, s, c, d);
  }
  if (implicit_atoms && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&cv.ctr->built, (unsigned long long)n);
}

// ===========================================================================
// Path B: a warp holds a CM; lane l holds vectors l, l + 32, ... (RV of them).
// Candidates are processed in batches of up to NB so that their table probes
// and compare reads are in flight together.
// ===========================================================================
template <typename W, int RV>
struct PathB {
  struct LaneConsts {
    uint4 lm[RV], lab[RV], care[RV], key[RV], mul[RV];
  };

  __device__ static void load_consts(const CacheView& cv, LaneConsts& k) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int r = 0; r < RV; ++r) {
      const int v = lane + 32 * r;
      k.lm[r] = cv.lenmask[v];
      k.lab[r] = cv.label[v];
      k.care[r] = cv.care[v];
      k.key[r] = cv.hkey[v];
      k.mul[r] = cv.hmul[v];
    }
  }

  __device__ static void load_row(const uint4* p, uint4 (&x)[RV]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int r = 0; r < RV; ++r) x[r] = __ldg(p + lane + 32 * r);
  }

  enum { kProbing = 0, kDone = 1, kClaimed = 2, kDeferred = 3 };

  // Spec check, probe, compare and insert a batch of NB candidates; bit q of
  // `en` says candidate q is real. c and desc are warp-uniform in meaning.
  template <int NB>
  __device__ static void batch(const CacheView& cv, const LaneConsts& k, const uint4 (&c)[NB][RV],
                               const uint64_t (&desc)[NB], uint32_t en) {
    const int lane = threadIdx.x & 31;
    int my_state = kDone;
    unsigned long long my_tag = 0, my_pos = 0;
    uint64_t my_desc = 0;
    uint32_t sol_mask = 0;
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      if (!((en >> q) & 1u)) continue;
      uint32_t lo = 0, hi = 0, bad = 0;
#pragma unroll
      for (int r = 0; r < RV; ++r) {
        h_acc(c[q][r], k.key[r], k.mul[r], lo, hi);
        bad |= spec_bad(c[q][r], k.lab[r], k.care[r]);
      }
      lo = __reduce_add_sync(kFull, lo);
      hi = __reduce_add_sync(kFull, hi);
      if (!__any_sync(kFull, bad != 0)) sol_mask |= 1u << q;
      if (lane == q) {
        const uint64_t h = h_fin(hi, lo);
        my_tag = (h >> 32) << 32;
        my_pos = h & cv.table_mask;
        my_state = kProbing;
        my_desc = desc[q];
      }
    }
    if (sol_mask && lane < NB && ((sol_mask >> lane) & 1u)) record_solution(cv, my_desc);

    uint32_t my_cmp = 0;
    unsigned long long guard = 0;
    while (true) {
      bool need_cmp = false;
      if (my_state == kProbing) {
        unsigned long long* slot = cv.table + my_pos;
        unsigned long long sv = ld_acquire(slot);
        if (sv == 0ull) {
          sv = atomicCAS(slot, 0ull, my_tag | kSlotPending);
          if (sv == 0ull) my_state = kClaimed;
        }
        if (my_state == kProbing) {
          const uint32_t low = uint32_t(sv);
          if ((sv & 0xFFFFFFFF00000000ull) != my_tag || low == kSlotTomb) {
            my_pos = (my_pos + 1) & cv.table_mask;
          } else if (low == kSlotPending) {
            my_state = kDeferred;
          } else {
            need_cmp = true;
            my_cmp = low - 1u;
          }
        }
      }
      const uint32_t cmp_mask = __ballot_sync(kFull, need_cmp);
      if (cmp_mask) {
        uint4 st[NB][RV];
#pragma unroll
        for (int q = 0; q < NB; ++q) {
          const uint32_t id = __shfl_sync(kFull, my_cmp, q);
          if ((cmp_mask >> q) & 1u) {
            const uint4* src = row_ptr(cv, id);
#pragma unroll
            for (int r = 0; r < RV; ++r) st[q][r] = __ldcg(src + lane + 32 * r);
          }
        }
#pragma unroll
        for (int q = 0; q < NB; ++q) {
          if (!((cmp_mask >> q) & 1u)) continue;
          uint32_t ne = 0;
#pragma unroll
          for (int r = 0; r < RV; ++r) ne |= v_ne(st[q][r], c[q][r]);
          const bool eq = !__any_sync(kFull, ne != 0);
          if (lane == q) {
            if (eq) my_state = kDone;
            else my_pos = (my_pos + 1) & cv.table_mask;
          }
        }
      }
      if (!__any_sync(kFull, my_state == kProbing)) break;
      if (++guard > cv.table_mask + 1) {  // every slot seen: cannot happen at load <= 0.9
        if (lane == 0) atomicExch(&cv.ctr->error, 1u);
        if (my_state == kProbing) my_state = kDone;
      }
    }

    const uint32_t claim = __ballot_sync(kFull, my_state == kClaimed);
    if (claim) {
      unsigned base = 0;
      if (lane == 0) base = atomicAdd(&cv.ctr->n_entries, (unsigned)__popc(claim));
      base = __shfl_sync(kFull, base, 0);
#pragma unroll
      for (int q = 0; q < NB; ++q) {
        if (!((claim >> q) & 1u)) continue;
        const unsigned id = base + __popc(claim & ((1u << q) - 1u));
        if (id < cv.max_entries) {
          uint4* dst = cv.arena + size_t(id) * cv.vecs;
#pragma unroll
          for (int r = 0; r < RV; ++r) dst[lane + 32 * r] = c[q][r];
          if (lane == 0) cv.prov[id] = desc[q];
        }
      }
      __threadfence();
      __syncwarp();
      if (my_state == kClaimed) {
        const unsigned id = base + __popc(claim & ((1u << lane) - 1u));
        unsigned long long* slot = cv.table + my_pos;
        if (id < cv.max_entries) {
          st_release(slot, my_tag | (unsigned long long)(id + 1u));
        } else {
          st_release(slot, my_tag | kSlotTomb);
          atomicExch(&cv.ctr->full, 1u);
        }
      }
    }
    if (my_state == kDeferred) defer(cv, my_desc);
  }
};

template <typename W, int RV>
__global__ void __launch_bounds__(256) k_unary_b(CacheView cv, uint32_t first, uint32_t count, uint32_t ops) {
  using P = PathB<W, RV>;
  typename P::LaneConsts k;
  P::load_consts(cv, k);
  const int lane = threadIdx.x & 31;
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  unsigned long long built = 0;
  for (uint32_t i = warp; i < count; i += nwarps) {
    if (__any_sync(kFull, stop_requested(cv))) break;
    const uint32_t id = first + i;
    uint4 a[RV];
    P::load_row(row_ptr(cv, id), a);
    uint4 c[4][RV];
#pragma unroll
    for (int r = 0; r < RV; ++r) {
      c[0][r] = v_op<W>(kNot, a[r], a[r], k.lm[r], cv.steps);
      c[1][r] = v_op<W>(kNext, a[r], a[r], k.lm[r], cv.steps);
      c[2][r] = v_op<W>(kFuture, a[r], a[r], k.lm[r], cv.steps);
      c[3][r] = v_op<W>(kGlobally, a[r], a[r], k.lm[r], cv.steps);
    }
    const uint64_t d[4] = {pack_desc(kNot, id, 0), pack_desc(kNext, id, 0), pack_desc(kFuture, id, 0),
                           pack_desc(kGlobally, id, 0)};
    P::template batch<4>(cv, k, c, d, ops & 0xFu);
    built += __popc(ops & 0xFu);
  }
  if (lane == 0 && built) atomicAdd(&cv.ctr->built, built);
}

// Binary operators over tiles of a split: the CTA stages `tile` rows of the
// smaller level in shared memory (amortising their loads over every row of the
// other level, paragraph "Amortising the cost of data movement"), and each warp
// streams rows of the other level through registers, building a & b, a | b,
// a U b and b U a for every staged row a.
template <typename W, int RV>
__global__ void __launch_bounds__(256) k_binary_b(CacheView cv, BinaryPlan plan) {
  using P = PathB<W, RV>;
  extern __shared__ uint4 s_left[];
  __shared__ unsigned long long s_tile;
  typename P::LaneConsts k;
  P::load_consts(cv, k);
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  const unsigned vecs = cv.vecs;
  unsigned long long built = 0;
  while (true) {
    if (threadIdx.x == 0) {
      unsigned long long t = atomicAdd(&cv.ctr->work[plan.work_slot], 1ull);
      if (stop_requested(cv)) t = plan.total_tiles;
      s_tile = t;
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
      const uint32_t total = ln * vecs;
      for (uint32_t i = threadIdx.x; i < total; i += blockDim.x) s_left[i] = __ldg(src + i);
    }
    __syncthreads();
    for (uint32_t rr = warp; rr < rn; rr += nwarps) {
      if (__any_sync(kFull, stop_requested(cv))) break;
      const uint32_t b_id = S.right_start + r0 + rr;
      uint4 b[RV];
      P::load_row(row_ptr(cv, b_id), b);
      for (uint32_t li = 0; li < ln; ++li) {
        const uint32_t a_id = S.left_start + l0 + li;
        if (S.tri && a_id >= b_id) break;  // same level: pairs a < b only (rows ascend)
        uint4 a[RV];
#pragma unroll
        for (int r = 0; r < RV; ++r) a[r] = s_left[li * vecs + lane + 32 * r];
        uint4 c[4][RV];
#pragma unroll
        for (int r = 0; r < RV; ++r) {
          c[0][r] = v_op<W>(kAnd, a[r], b[r], k.lm[r], cv.steps);
          c[1][r] = v_op<W>(kOr, a[r], b[r], k.lm[r], cv.steps);
          c[2][r] = v_op<W>(kUntil, a[r], b[r], k.lm[r], cv.steps);
          c[3][r] = v_op<W>(kUntil, b[r], a[r], k.lm[r], cv.steps);
        }
        const uint64_t d[4] = {pack_desc(kAnd, a_id, b_id), pack_desc(kOr, a_id, b_id),
                               pack_desc(kUntil, a_id, b_id), pack_desc(kUntil, b_id, a_id)};
        P::template batch<4>(cv, k, c, d, plan.ops);
        built += __popc(plan.ops);
      }
    }
    __syncthreads();
  }
  if (lane == 0 && built) atomicAdd(&cv.ctr->built, built);
}

template <typename W, int RV>
__global__ void __launch_bounds__(256) k_desc_b(CacheView cv, const unsigned long long* list,
                                                const unsigned int* list_n, unsigned int list_cap,
                                                unsigned int implicit_atoms) {
  using P = PathB<W, RV>;
  typename P::LaneConsts k;
  P::load_consts(cv, k);
  const int lane = threadIdx.x & 31;
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  unsigned n = implicit_atoms;
  if (list) n = min(*list_n, list_cap);
  for (uint32_t i = warp; i < n; i += nwarps) {
    if (__any_sync(kFull, stop_requested(cv))) break;
    const uint64_t d = list ? list[i] : pack_desc(kAtom, i, 0);
    const uint32_t op = desc_op(d);
    uint4 c[1][RV];
    if (op == kAtom) {
      P::load_row(cv.atoms + size_t(desc_left(d)) * cv.vecs, c[0]);
    } else {
      uint4 a[RV], b[RV];
      P::load_row(row_ptr(cv, desc_left(d)), a);
      if (op == kAnd || op == kOr || op == kUntil) P::load_row(row_ptr(cv, desc_right(d)), b);
      else {
#pragma unroll
        for (int r = 0; r < RV; ++r) b[r] = a[r];
      }
#pragma unroll
      for (int r = 0; r < RV; ++r) c[0][r] = v_op<W>(op, a[r], b[r], k.lm[r], cv.steps);
    }
    const uint64_t dd[1] = {d};
    P::template batch<1>(cv, k, c, dd, 1u);
  }
  if (implicit_atoms && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&cv.ctr->built, (unsigned long long)n);
  (void)lane;
}

// ===========================================================================
// Formula evaluation: one thread per trace word walks a postorder node list
// (x = op, y = left node, z = right node, w = proposition); scratch holds one
// row of words per node.
// ===========================================================================
template <typename W>
__global__ void k_eval(const W* atoms, const W* lenmask, unsigned words, const int4* nodes, int n_nodes, int steps,
                       W* scratch, W* out) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= words) return;
  const W lm = lenmask[t];
  for (int i = 0; i < n_nodes; ++i) {
    const int4 nd = nodes[i];
    W v;
    if (nd.x == int(kAtom)) v = atoms[size_t(nd.w) * words + t];
    else {
      const W a = scratch[size_t(nd.y) * words + t];
      const W b = nd.z >= 0 ? scratch[size_t(nd.z) * words + t] : a;
      v = w_op<W>(uint32_t(nd.x), a, b, lm, steps);
    }
    scratch[size_t(i) * words + t] = v;
  }
  out[t] = scratch[size_t(n_nodes - 1) * words + t];
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

template <typename W, int RV>
struct LaunchB {
  static cudaError_t desc_list(const CacheView& cv, const unsigned long long* list, const unsigned int* list_n,
                               unsigned int cap, unsigned int atoms, const LaunchCfg& lc) {
    const unsigned n = list ? cap : atoms;
    const unsigned blocks = std::max(1u, std::min((n + 7u) / 8u, unsigned(lc.sms * 8)));
    k_desc_b<W, RV><<<blocks, 256, 0, lc.stream>>>(cv, list, list_n, cap, atoms);
    return cudaGetLastError();
  }
  static cudaError_t unary(const CacheView& cv, uint32_t first, uint32_t count, uint32_t ops, const LaunchCfg& lc) {
    static int occ = occupancy_blocks((const void*)k_unary_b<W, RV>, 256, 0);
    const unsigned blocks = std::max(1u, std::min((count + 7u) / 8u, unsigned(lc.sms * occ)));
    k_unary_b<W, RV><<<blocks, 256, 0, lc.stream>>>(cv, first, count, ops);
    return cudaGetLastError();
  }
  static cudaError_t binary(const CacheView& cv, const BinaryPlan& plan, const LaunchCfg& lc) {
    const size_t smem = size_t(plan.tile) * cv.vecs * sizeof(uint4);
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute((const void*)k_binary_b<W, RV>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
      attr = true;
    }
    const int occ = occupancy_blocks((const void*)k_binary_b<W, RV>, 256, smem);
    const unsigned long long blocks = std::max(1ull, std::min(plan.total_tiles, (unsigned long long)lc.sms * occ));
    k_binary_b<W, RV><<<unsigned(blocks), 256, smem, lc.stream>>>(cv, plan);
    return cudaGetLastError();
  }
};

template <typename W>
int Kernels<W>::path_for(unsigned vecs) {
  if (vecs == 1 || vecs == 2 || vecs == 4 || vecs == 8) return 1;
  if (vecs == 32 || vecs == 64 || vecs == 128 || vecs == 256) return 2;
  return 0;
}

#define LSYN_DISPATCH(vecs, CALL_A, CALL_B)             \
  switch (vecs) {                                       \
    case 1: return LaunchA<W, 1>::CALL_A;               \
    case 2: return LaunchA<W, 2>::CALL_A;               \
    case 4: return LaunchA<W, 4>::CALL_A;               \
    case 8: return LaunchA<W, 8>::CALL_A;               \
    case 32: return LaunchB<W, 1>::CALL_B;              \
    case 64: return LaunchB<W, 2>::CALL_B;              \
    case 128: return LaunchB<W, 4>::CALL_B;             \
    case 256: return LaunchB<W, 8>::CALL_B;             \
    default: return cudaErrorInvalidValue;              \
  }

template <typename W>
cudaError_t Kernels<W>::desc_list(const CacheView& cv, const unsigned long long* list, const unsigned int* list_n,
                                  unsigned int cap, unsigned int atoms, const LaunchCfg& lc) {
  LSYN_DISPATCH(cv.vecs, desc_list(cv, list, list_n, cap, atoms, lc), desc_list(cv, list, list_n, cap, atoms, lc))
}

template <typename W>
cudaError_t Kernels<W>::unary(const CacheView& cv, uint32_t first, uint32_t count, uint32_t ops,
                              const LaunchCfg& lc) {
  LSYN_DISPATCH(cv.vecs, unary(cv, first, count, ops, lc), unary(cv, first, count, ops, lc))
}

template <typename W>
cudaError_t Kernels<W>::binary(const CacheView& cv, const BinaryPlan& plan, const LaunchCfg& lc) {
  LSYN_DISPATCH(cv.vecs, binary(cv, plan, lc), binary(cv, plan, lc))
}

template <typename W>
cudaError_t Kernels<W>::eval(const uint4* atoms, const uint4* lenmask, unsigned vecs, const int4* nodes,
                             int n_nodes, int steps, W* scratch, W* out, const LaunchCfg& lc) {
  const unsigned words = vecs * unsigned(sizeof(uint4) / sizeof(W));
  k_eval<W><<<(words + 127u) / 128u, 128, 0, lc.stream>>>(reinterpret_cast<const W*>(atoms),
                                                          reinterpret_cast<const W*>(lenmask), words, nodes,
                                                          n_nodes, steps, scratch, out);
  return cudaGetLastError();
}

}  // namespace lsyn
