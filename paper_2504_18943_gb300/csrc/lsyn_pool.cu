// Block pool and growable segments on the driver's virtual-memory interface.
#include "lsyn_pool.h"

#include <algorithm>

#include <cuda.h>
#include <cuda_runtime.h>

namespace lsyn {
namespace {

// The virtual-memory entry points of the driver, looked up once.
struct Vmm {
  CUresult (*create)(CUmemGenericAllocationHandle*, size_t, const CUmemAllocationProp*, unsigned long long) = nullptr;
  CUresult (*release)(CUmemGenericAllocationHandle) = nullptr;
  CUresult (*reserve)(CUdeviceptr*, size_t, size_t, CUdeviceptr, unsigned long long) = nullptr;
  CUresult (*addr_free)(CUdeviceptr, size_t) = nullptr;
  CUresult (*map)(CUdeviceptr, size_t, size_t, CUmemGenericAllocationHandle, unsigned long long) = nullptr;
  CUresult (*unmap)(CUdeviceptr, size_t) = nullptr;
  CUresult (*set_access)(CUdeviceptr, size_t, const CUmemAccessDesc*, size_t) = nullptr;
  CUresult (*granularity)(size_t*, const CUmemAllocationProp*, CUmemAllocationGranularity_flags) = nullptr;
  bool ok = false;
  std::string err;

  template <typename F>
  bool get(const char* name, F* fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p) {
      cudaGetLastError();
      err = std::string("driver entry point ") + name + " not found";
      return false;
    }
    *fn = reinterpret_cast<F>(p);
    return true;
  }

  Vmm() {
    ok = get("cuMemCreate", &create) && get("cuMemRelease", &release) && get("cuMemAddressReserve", &reserve) &&
         get("cuMemAddressFree", &addr_free) && get("cuMemMap", &map) && get("cuMemUnmap", &unmap) &&
         get("cuMemSetAccess", &set_access) && get("cuMemGetAllocationGranularity", &granularity);
  }
};

const Vmm& vmm() {
  static const Vmm v;
  return v;
}

CUmemAllocationProp device_prop(int device) {
  CUmemAllocationProp prop = {};
  prop.type = CU_MEM_ALLOCATION_TYPE_PINNED;
  prop.location.type = CU_MEM_LOCATION_TYPE_DEVICE;
  prop.location.id = device;
  return prop;
}

std::string cu_msg(const char* what, CUresult r) { return std::string(what) + " failed (driver error " + std::to_string(int(r)) + ")"; }

}  // namespace

BlockPool::~BlockPool() {
  if (device_ < 0) return;
  for (auto& kv : free_)
    for (unsigned long long h : kv.second) vmm().release(CUmemGenericAllocationHandle(h));
  free_.clear();
}

bool BlockPool::init(int device, size_t budget, std::string* err) {
  const Vmm& v = vmm();
  if (!v.ok) { *err = v.err; return false; }
  if (cudaSetDevice(device) != cudaSuccess || cudaFree(nullptr) != cudaSuccess) {
    cudaGetLastError();
    *err = "cannot make the device current";
    return false;
  }
  const CUmemAllocationProp prop = device_prop(device);
  size_t g = 0;
  CUresult r = v.granularity(&g, &prop, CU_MEM_ALLOC_GRANULARITY_RECOMMENDED);
  if (r != CUDA_SUCCESS || g == 0) { *err = cu_msg("cuMemGetAllocationGranularity", r); return false; }
  device_ = device;
  gran_ = g;
  budget_ = budget / g * g;
  return true;
}

size_t BlockPool::size_class(size_t bytes) const {
  const size_t units = std::max<size_t>(1, (bytes + gran_ - 1) / gran_);
  size_t p = 1;
  while (p < units) {
    if (p >= 2 && p + p / 2 >= units) return (p + p / 2) * gran_;  // 3 * 2^(i-1)
    p <<= 1;
  }
  return p * gran_;
}

bool BlockPool::release_cached(size_t need) {
  // Return cached blocks (largest first) until `need` more bytes fit the budget.
  while (in_use_ + cached_ + need > budget_ && cached_ > 0) {
    auto it = std::prev(free_.end());
    vmm().release(CUmemGenericAllocationHandle(it->second.back()));
    cached_ -= it->first;
    it->second.pop_back();
    if (it->second.empty()) free_.erase(it);
  }
  return in_use_ + cached_ + need <= budget_;
}

bool BlockPool::take(size_t bytes, unsigned long long* handle, std::string* err) {
  auto it = free_.find(bytes);
  if (it != free_.end() && !it->second.empty()) {
    *handle = it->second.back();
    it->second.pop_back();
    if (it->second.empty()) free_.erase(it);
    cached_ -= bytes;
    in_use_ += bytes;
    return true;
  }
  if (in_use_ + bytes > budget_ || !release_cached(bytes)) {
    *err = "memory pool budget exhausted";
    return false;
  }
  const CUmemAllocationProp prop = device_prop(device_);
  CUmemGenericAllocationHandle h;
  CUresult r = vmm().create(&h, bytes, &prop, 0);
  if (r != CUDA_SUCCESS) {
    // The device may hold less than the budget: drop every cached block, retry once.
    release_cached(budget_);
    r = vmm().create(&h, bytes, &prop, 0);
    if (r != CUDA_SUCCESS) { *err = cu_msg("cuMemCreate", r); return false; }
  }
  *handle = static_cast<unsigned long long>(h);
  in_use_ += bytes;
  return true;
}

void BlockPool::give(size_t bytes, unsigned long long handle) {
  in_use_ -= bytes;
  free_[bytes].push_back(handle);
  cached_ += bytes;
}

Segment& Segment::operator=(Segment&& o) noexcept {
  va_ = o.va_;
  reserved_ = o.reserved_;
  mapped_ = o.mapped_;
  blocks_ = static_cast<std::vector<std::pair<size_t, unsigned long long>>&&>(o.blocks_);
  o.va_ = 0;
  o.reserved_ = o.mapped_ = 0;
  o.blocks_.clear();
  return *this;
}

bool Segment::reserve(BlockPool& pool, size_t max_bytes, std::string* err) {
  const size_t g = pool.granularity();
  // Room for the size classes' rounding on top of the largest size.
  const size_t want = ((max_bytes + g - 1) / g) * g;
  const size_t res = ((want + want / 2 + g - 1) / g) * g + 2 * g;  // a multiple of the granularity
  CUdeviceptr p = 0;
  CUresult r = vmm().reserve(&p, res, g, 0, 0);
  if (r != CUDA_SUCCESS) { *err = cu_msg("cuMemAddressReserve", r); return false; }
  va_ = static_cast<unsigned long long>(p);
  reserved_ = res;
  mapped_ = 0;
  return true;
}

size_t Segment::next_block(const BlockPool& pool, size_t bytes, size_t limit) const {
  if (bytes <= mapped_) return 0;
  const size_t g = pool.granularity();
  const size_t exact = ((bytes - mapped_ + g - 1) / g) * g;  // the remainder, rounded to the granularity
  const size_t want = std::max(bytes, mapped_ + mapped_ / 2);
  size_t add = pool.size_class(want - mapped_);
  if (limit > mapped_) add = std::min(add, std::max(exact, ((limit - mapped_ + g - 1) / g) * g));
  if (mapped_ + add > reserved_) add = exact;
  return mapped_ + add > reserved_ ? ~size_t(0) : add;
}

size_t Segment::grow_cost(const BlockPool& pool, size_t bytes, size_t limit) const {
  return next_block(pool, bytes, limit);
}

bool Segment::grow(BlockPool& pool, size_t bytes, std::string* err, size_t limit) {
  const size_t add = next_block(pool, bytes, limit);
  if (add == 0) return true;
  if (add == ~size_t(0)) { *err = "segment reservation exceeded"; return false; }
  unsigned long long h = 0;
  if (!pool.take(add, &h, err)) return false;
  const CUdeviceptr at = CUdeviceptr(va_ + mapped_);
  CUresult r = vmm().map(at, add, 0, CUmemGenericAllocationHandle(h), 0);
  if (r != CUDA_SUCCESS) {
    pool.give(add, h);
    *err = cu_msg("cuMemMap", r);
    return false;
  }
  CUmemAccessDesc ad = {};
  ad.location.type = CU_MEM_LOCATION_TYPE_DEVICE;
  ad.location.id = pool.device();
  ad.flags = CU_MEM_ACCESS_FLAGS_PROT_READWRITE;
  r = vmm().set_access(at, add, &ad, 1);
  if (r != CUDA_SUCCESS) {
    vmm().unmap(at, add);
    pool.give(add, h);
    *err = cu_msg("cuMemSetAccess", r);
    return false;
  }
  blocks_.push_back({add, h});
  mapped_ += add;
  return true;
}

void Segment::shrink(BlockPool& pool, size_t keep_bytes) {
  while (!blocks_.empty() && mapped_ - blocks_.back().first >= keep_bytes && mapped_ > keep_bytes) {
    const auto b = blocks_.back();
    mapped_ -= b.first;
    vmm().unmap(CUdeviceptr(va_ + mapped_), b.first);
    pool.give(b.first, b.second);
    blocks_.pop_back();
  }
}

void Segment::release(BlockPool& pool) {
  size_t off = 0;
  for (auto& b : blocks_) {
    vmm().unmap(CUdeviceptr(va_ + off), b.first);
    pool.give(b.first, b.second);
    off += b.first;
  }
  blocks_.clear();
  if (va_) vmm().addr_free(CUdeviceptr(va_), reserved_);
  va_ = 0;
  reserved_ = mapped_ = 0;
}

}  // namespace lsyn
