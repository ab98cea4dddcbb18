// Device memory for many language caches that grow level by level.
//
// A cache's arrays (CM arena, provenance, table slots, hash words, deferred
// lists) are Segments: a virtual address range reserved once for the cache's
// largest size, whose prefix is backed by physical blocks mapped on demand, so
// an array grows in place without copying. Blocks come from one BlockPool per
// device: sizes are the allocation granularity times 1, 2, 3, 4, 6, 8, 12, ...
// (powers of two and 1.5 times powers of two), released blocks wait on
// per-size free lists for reuse, and the pool never holds more physical memory
// than its budget (free blocks are returned to the driver when a new size is
// needed). The driver's virtual-memory entry points are looked up at run time
// through the runtime, so the library does not link the driver library.
#pragma once

#include <cstddef>
#include <cstdint>
#include <map>
#include <string>
#include <vector>

namespace lsyn {

class BlockPool {
 public:
  BlockPool() = default;
  BlockPool(const BlockPool&) = delete;
  BlockPool& operator=(const BlockPool&) = delete;
  ~BlockPool();

  // budget: physical bytes the pool may hold (mapped + cached free blocks).
  bool init(int device, size_t budget, std::string* err);
  size_t granularity() const { return gran_; }
  size_t budget() const { return budget_; }
  size_t in_use() const { return in_use_; }
  // Bytes a caller may still map (free budget plus cached blocks).
  size_t available() const { return budget_ - in_use_; }
  // The block size class at or above `bytes`.
  size_t size_class(size_t bytes) const;
  // A block of exactly `bytes` (a size class): from the free list, else new.
  bool take(size_t bytes, unsigned long long* handle, std::string* err);
  void give(size_t bytes, unsigned long long handle);
  int device() const { return device_; }

 private:
  int device_ = -1;
  size_t gran_ = 0;
  size_t budget_ = 0;
  size_t in_use_ = 0;   // bytes of blocks handed out
  size_t cached_ = 0;   // bytes of blocks on the free lists
  std::map<size_t, std::vector<unsigned long long>> free_;
  bool release_cached(size_t need);
};

class Segment {
 public:
  Segment() = default;
  Segment(const Segment&) = delete;
  Segment& operator=(const Segment&) = delete;
  Segment(Segment&& o) noexcept { *this = static_cast<Segment&&>(o); }
  Segment& operator=(Segment&& o) noexcept;
  ~Segment() = default;  // release() must be called with the pool

  // Reserve virtual space for up to `max_bytes` (nothing is mapped yet).
  bool reserve(BlockPool& pool, size_t max_bytes, std::string* err);
  // Map blocks until at least `bytes` are backed, growing by at least half the
  // current size. Returns false (and maps nothing) if the pool cannot supply.
  // `limit` (0: none) bounds the mapping: the segment never needs more.
  bool grow(BlockPool& pool, size_t bytes, std::string* err, size_t limit = 0);
  // Physical bytes grow(bytes, limit) would add.
  size_t grow_cost(const BlockPool& pool, size_t bytes, size_t limit = 0) const;
  // Unmap trailing blocks while at least `keep_bytes` stay mapped (0: all).
  void shrink(BlockPool& pool, size_t keep_bytes);
  void release(BlockPool& pool);
  void* ptr() const { return reinterpret_cast<void*>(static_cast<uintptr_t>(va_)); }
  size_t mapped() const { return mapped_; }
  size_t reserved() const { return reserved_; }

 private:
  unsigned long long va_ = 0;
  size_t reserved_ = 0;
  size_t mapped_ = 0;
  std::vector<std::pair<size_t, unsigned long long>> blocks_;
  size_t next_block(const BlockPool& pool, size_t bytes, size_t limit) const;
};

}  // namespace lsyn
