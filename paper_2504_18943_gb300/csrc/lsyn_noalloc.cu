// lsyn_eval_noalloc: formula evaluation that allocates no device memory.
//
// Some callers cannot call cudaMalloc: a host process whose memory manager
// owns every device allocation (a serving engine that carves the whole GPU
// into its own pool at start-up and forbids allocations behind its back), or
// a latency-critical loop where a cudaMalloc/cudaFree pair, which can
// synchronise the whole device, is not acceptable. For them this entry point
// evaluates a formula on traces the caller already holds on the device,
// writing into an output buffer the caller provides, and keeps its per-node
// scratch rows in a file-scope device array instead of allocating them.
//
// The scratch array is a fixed 8 MiB per GPU, held until the process exits.
// The CUDA runtime loads a library's device code lazily (by default), so the
// array is reserved on a device when this file's code is first loaded there:
// the first call on each device does that (it also loads the evaluation
// kernels), and may allocate and synchronise inside the driver. A caller whose
// memory manager takes the whole GPU must make that first call, e.g. on a
// one-node formula, before its manager claims the memory, and before any
// stream capture. Every call on a device shares the array and it keeps the
// last call's contents; nothing in it needs clearing (every row is written
// before it is read). Calls that overlap on the GPU (different streams, or
// different host threads on one device) race on it.
#include <cstdint>
#include <cstring>
#include <functional>
#include <mutex>
#include <string>
#include <vector>

#include "lsyn.h"
#include "lsyn_device.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;
constexpr int kNoAllocMaxNodes = 960;  // nodes travel as kernel parameters (4 bytes each)
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_eval_scratch[kNoAllocScratchBytes];

struct NodeTable {
  uint32_t n[kNoAllocMaxNodes];  // op | left << 3 | (right + 1) << 13 | prop << 24
};

std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {};

__device__ __forceinline__ uint32_t reverse_bits(uint32_t x) { return __brev(x); }
__device__ __forceinline__ uint64_t reverse_bits(uint64_t x) { return __brevll(x); }

template <typename W>
__global__ void k_eval_noalloc(const W* atoms, const int32_t* lengths, unsigned n_traces, NodeTable nodes,
                               int n_nodes, W* scratch, W* out) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_traces) return;
  constexpr int kBits = int(sizeof(W) * 8);
  const int len = lengths[t];
  // Length mask in the library's order (position 0 = top bit).
  const W lm = len >= kBits ? ~W(0) : len <= 0 ? W(0) : ~(~W(0) >> len);
  for (int i = 0; i < n_nodes; ++i) {
    const uint32_t nd = nodes.n[i];
    const uint32_t op = nd & 7u;
    W v;
    if (op == lsyn::kAtom) {
      v = reverse_bits(atoms[size_t(nd >> 24) * n_traces + t]) & lm;  // input: bit t = position t
    } else {
      const W a = scratch[size_t((nd >> 3) & 1023u) * n_traces + t];
      const uint32_t rb = (nd >> 13) & 2047u;
      const W b = rb ? scratch[size_t(rb - 1u) * n_traces + t] : a;
      v = lsyn::w_op_logstep<W>(op, a, b, lm, lsyn::WordInfo<W>::kMaxSteps);
    }
    scratch[size_t(i) * n_traces + t] = v;
  }
  out[t] = reverse_bits(scratch[size_t(n_nodes - 1) * n_traces + t]);  // output: bit t = position t
}

bool parse_nodes(const char* s, int n_props, std::vector<uint32_t>* out, std::string* err);

// First use on a device (with that device current): load the evaluation
// kernels and this file's device data there, so that every allocation this
// entry point causes happens now, then look the scratch array's device address
// up (the symbol's host-side name is not a device address). Later calls reuse
// the address.
cudaError_t scratch_address(int device, void** out) {
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_addr[device]) {
    cudaFuncAttributes attr;
    cudaError_t e = cudaFuncGetAttributes(&attr, k_eval_noalloc<uint32_t>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&attr, k_eval_noalloc<uint64_t>);
    void* p = nullptr;
    if (e == cudaSuccess) e = cudaGetSymbolAddress(&p, g_eval_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[device] = p;
  }
  *out = g_scratch_addr[device];
  return cudaSuccess;
}

}  // namespace

extern "C" lsyn_status lsyn_eval_noalloc(int32_t n_props, int32_t n_traces, int32_t word_bits,
                                         const void* atom_words, const int32_t* lengths, const char* formula,
                                         void* dst, void* stream) {
  std::string& g_noalloc_error = lsyn::thread_error();
  g_noalloc_error.clear();
  if (n_props < 1 || n_props > 32 || n_traces < 1 || (word_bits != 32 && word_bits != 64) || !atom_words ||
      !lengths || !formula || !dst) {
    g_noalloc_error = "lsyn_eval_noalloc: bad arguments";
    return LSYN_E_INVAL;
  }
  std::vector<uint32_t> nodes;
  if (!parse_nodes(formula, n_props, &nodes, &g_noalloc_error)) return LSYN_E_INVAL;
  const size_t need = nodes.size() * size_t(n_traces) * size_t(word_bits / 8);
  if (need > kNoAllocScratchBytes) {
    g_noalloc_error = "lsyn_eval_noalloc: nodes x traces x word bytes = " + std::to_string(need) +
                      " exceeds the fixed scratch of " + std::to_string(kNoAllocScratchBytes) + " bytes";
    return LSYN_E_INVAL;
  }
  int device = 0;
  cudaError_t e = cudaGetDevice(&device);
  if (e == cudaSuccess && (device < 0 || device >= kMaxDevices)) e = cudaErrorInvalidDevice;
  void* scratch = nullptr;
  if (e == cudaSuccess) e = scratch_address(device, &scratch);
  if (e != cudaSuccess) {
    g_noalloc_error = std::string("lsyn_eval_noalloc: ") + cudaGetErrorString(e);
    return LSYN_E_CUDA;
  }
  NodeTable table;
  memset(&table, 0, sizeof(table));
  for (size_t i = 0; i < nodes.size(); ++i) table.n[i] = nodes[i];
  const unsigned blocks = (unsigned(n_traces) + 127u) / 128u;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaGetLastError();  // an earlier, unrelated launch error on this thread is not this call's
  if (word_bits == 32)
    k_eval_noalloc<uint32_t><<<blocks, 128, 0, st>>>(static_cast<const uint32_t*>(atom_words), lengths,
                                                    unsigned(n_traces), table, int(nodes.size()),
                                                    static_cast<uint32_t*>(scratch), static_cast<uint32_t*>(dst));
  else
    k_eval_noalloc<uint64_t><<<blocks, 128, 0, st>>>(static_cast<const uint64_t*>(atom_words), lengths,
                                                    unsigned(n_traces), table, int(nodes.size()),
                                                    static_cast<uint64_t*>(scratch), static_cast<uint64_t*>(dst));
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    g_noalloc_error = std::string("lsyn_eval_noalloc: ") + cudaGetErrorString(e);
    return LSYN_E_CUDA;
  }
  return LSYN_OK;
}

namespace {

// Prefix formula text -> packed postorder node list (children first).
bool parse_nodes(const char* s, int n_props, std::vector<uint32_t>* out, std::string* err) {
  size_t i = 0;
  const size_t len = strlen(s);
  int depth = 0;
  auto skip = [&]() { while (i < len && (s[i] == ' ' || s[i] == '\t' || s[i] == '\n')) ++i; };
  std::function<int()> parse;
  parse = [&]() -> int {
    if (++depth > kNoAllocMaxNodes || int(out->size()) >= kNoAllocMaxNodes) {
      *err = "lsyn_eval_noalloc: more than " + std::to_string(kNoAllocMaxNodes) + " nodes";
      return -1;
    }
    skip();
    if (i < len && s[i] == 'p') {
      ++i;
      if (i >= len || s[i] < '0' || s[i] > '9') { *err = "lsyn_eval_noalloc: bad atom"; return -1; }
      int v = 0;
      while (i < len && s[i] >= '0' && s[i] <= '9' && v <= 1000) { v = v * 10 + (s[i] - '0'); ++i; }
      if (v >= n_props) { *err = "lsyn_eval_noalloc: atom out of range"; return -1; }
      out->push_back(lsyn::kAtom | (uint32_t(v) << 24));
      --depth;
      return int(out->size()) - 1;
    }
    if (i >= len || s[i] != '(') { *err = "lsyn_eval_noalloc: expected '(' or atom"; return -1; }
    ++i;
    skip();
    if (i >= len) { *err = "lsyn_eval_noalloc: truncated"; return -1; }
    uint32_t op;
    switch (s[i]) {
      case '!': op = lsyn::kNot; break;
      case '&': op = lsyn::kAnd; break;
      case '|': op = lsyn::kOr; break;
      case 'X': op = lsyn::kNext; break;
      case 'F': op = lsyn::kFuture; break;
      case 'G': op = lsyn::kGlobally; break;
      case 'U': op = lsyn::kUntil; break;
      default: *err = "lsyn_eval_noalloc: unknown operator"; return -1;
    }
    ++i;
    const int a = parse();
    if (a < 0) return -1;
    int b = -1;
    if (op == lsyn::kAnd || op == lsyn::kOr || op == lsyn::kUntil) {
      b = parse();
      if (b < 0) return -1;
    }
    skip();
    if (i >= len || s[i] != ')') { *err = "lsyn_eval_noalloc: expected ')'"; return -1; }
    ++i;
    out->push_back(op | (uint32_t(a) << 3) | (uint32_t(b + 1) << 13));
    --depth;
    return int(out->size()) - 1;
  };
  if (parse() < 0) return false;
  skip();
  if (i != len) { *err = "lsyn_eval_noalloc: trailing text"; return false; }
  return true;
}

}  // namespace
