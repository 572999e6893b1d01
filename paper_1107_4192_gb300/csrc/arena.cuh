// Device-memory arena behind kf_arena_reserve (include/kfmeg.h).
#pragma once

#include "common.cuh"

namespace kfm {

// A block of at least `bytes` (256-byte aligned) from the arena of the
// current device, or nullptr when no arena is reserved there or none fits.
void* arena_alloc(uint64_t bytes);
// True when p points into the arena.
bool arena_owns(const void* p);
// Returns a block from arena_alloc; the caller has finished all GPU work on it.
void arena_free(void* p);

}  // namespace kfm
