// Device-memory arena for plans: one reservation up front, sub-allocated
// first-fit with coalescing, so that creating and destroying plans (one per
// served request) calls neither cudaMalloc nor cudaFree.  cudaFree
// synchronises the whole device and would stall the streams of the other
// requests in flight; cudaMalloc can do the same.
#include <map>
#include <mutex>

#include "arena.cuh"

namespace kfm {

namespace {

struct Arena {
  std::mutex mu;
  char* base = nullptr;
  uint64_t size = 0;
  int device = -1;
  std::map<uint64_t, uint64_t> free_;  // offset -> length (coalesced)
  std::map<uint64_t, uint64_t> used_;  // offset -> length
  uint64_t in_use = 0;
};

Arena g_arena;
constexpr uint64_t kAlign = 256;

}  // namespace

void* arena_alloc(uint64_t bytes) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(g_arena.mu);
  if (!g_arena.base || dev != g_arena.device) return nullptr;
  const uint64_t len = (bytes + kAlign - 1) / kAlign * kAlign;
  for (auto it = g_arena.free_.begin(); it != g_arena.free_.end(); ++it) {
    if (it->second < len) continue;
    const uint64_t off = it->first, rest = it->second - len;
    g_arena.free_.erase(it);
    if (rest) g_arena.free_[off + len] = rest;
    g_arena.used_[off] = len;
    g_arena.in_use += len;
    return g_arena.base + off;
  }
  return nullptr;
}

bool arena_owns(const void* p) {
  std::lock_guard<std::mutex> lock(g_arena.mu);
  const char* c = static_cast<const char*>(p);
  return g_arena.base && c >= g_arena.base && c < g_arena.base + g_arena.size;
}

void arena_free(void* p) {
  std::lock_guard<std::mutex> lock(g_arena.mu);
  const uint64_t off = (uint64_t)(static_cast<char*>(p) - g_arena.base);
  auto u = g_arena.used_.find(off);
  if (u == g_arena.used_.end()) return;
  uint64_t start = off, len = u->second;
  g_arena.used_.erase(u);
  g_arena.in_use -= len;
  auto next = g_arena.free_.lower_bound(start);
  if (next != g_arena.free_.end() && next->first == start + len) {  // merge with the following block
    len += next->second;
    next = g_arena.free_.erase(next);
  }
  if (next != g_arena.free_.begin()) {  // merge with the preceding block
    auto prev = std::prev(next);
    if (prev->first + prev->second == start) {
      start = prev->first;
      len += prev->second;
      g_arena.free_.erase(prev);
    }
  }
  g_arena.free_[start] = len;
}

}  // namespace kfm

using namespace kfm;

extern "C" {

kf_status kf_arena_reserve(uint64_t bytes) {
  if (bytes == 0) return KF_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_arena.mu);
  if (g_arena.base) return KF_ERR_STATE;
  int dev = -1;
  KF_CUDA_TRY(cudaGetDevice(&dev));
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return KF_ERR_CUDA;
  }
  g_arena.base = static_cast<char*>(p);
  g_arena.size = bytes / kAlign * kAlign;
  g_arena.device = dev;
  g_arena.free_.clear();
  g_arena.used_.clear();
  g_arena.free_[0] = g_arena.size;
  g_arena.in_use = 0;
  return KF_OK;
}

kf_status kf_arena_release(void) {
  std::lock_guard<std::mutex> lock(g_arena.mu);
  if (!g_arena.base) return KF_OK;
  if (!g_arena.used_.empty()) return KF_ERR_STATE;
  KF_CUDA_TRY(cudaFree(g_arena.base));
  g_arena.base = nullptr;
  g_arena.size = 0;
  g_arena.device = -1;
  g_arena.free_.clear();
  return KF_OK;
}

kf_status kf_arena_stats(uint64_t* reserved, uint64_t* in_use, uint64_t* largest_free) {
  std::lock_guard<std::mutex> lock(g_arena.mu);
  uint64_t big = 0;
  for (auto& f : g_arena.free_) big = f.second > big ? f.second : big;
  if (reserved) *reserved = g_arena.size;
  if (in_use) *in_use = g_arena.in_use;
  if (largest_free) *largest_free = big;
  return KF_OK;
}

}  // extern "C"
