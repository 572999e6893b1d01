// Shared device/host helpers for the kfmeg CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stdio.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <set>
#include <utility>

#include "../../include/kfmeg.h"

namespace kfm {

// Device status word layout: [0] = kf_status code of the first failure,
// [1] = 1-based time step of the failure, [2] = index inside the failing
// factorisation (pivot) or element, [3] = current step for kernels launched
// with step < 0 (replayed CUDA graphs, whose arguments are fixed).
enum { ST_CODE = 0, ST_STEP = 1, ST_INDEX = 2, ST_CUR = 3, ST_WORDS = 4 };

__device__ __forceinline__ bool status_failed(const int* st) {
  return st != nullptr && *(volatile const int*)st != 0;
}

__device__ __forceinline__ void status_set(int* st, int code, int step, int index) {
  if (st == nullptr) return;
  if (atomicCAS(st + ST_CODE, 0, code) == 0) {
    st[ST_STEP] = step < 0 ? st[ST_CUR] : step;
    st[ST_INDEX] = index;
  }
}

template <typename T> struct Num;
template <> struct Num<double> {
  static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
};
template <> struct Num<float> {
  static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
};

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }

// Returns from the enclosing function with KF_ERR_CUDA on a runtime error.
#define KF_CUDA_TRY(expr)                                                          \
  do {                                                                             \
    cudaError_t e_ = (expr);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      fprintf(stderr, "kfmeg: %s failed: %s (%s:%d)\n", #expr, cudaGetErrorString(e_), \
              __FILE__, __LINE__);                                                 \
      return KF_ERR_CUDA;                                                          \
    }                                                                              \
  } while (0)

#define KF_TRY(expr)                     \
  do {                                   \
    kf_status s_ = (expr);               \
    if (s_ != KF_OK) return s_;          \
  } while (0)

// Checks the last launch error; returns KF_ERR_CUDA on failure.
inline kf_status launch_check(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    fprintf(stderr, "kfmeg: launch of %s failed: %s\n", what, cudaGetErrorString(e));
    return KF_ERR_CUDA;
  }
  return KF_OK;
}

// Counts every kernel launch made through the library (for the launch census);
// atomic because plans may run concurrently from several host threads.
extern std::atomic<int64_t> g_launches;
// Launches made by the calling host thread (per-plan counts are differences of it).
extern thread_local int64_t t_launches;
inline void note_launch(int64_t n = 1) {
  g_launches += n;
  t_launches += n;
}

// Raises the dynamic shared-memory limit of kernel `fn` to `bytes` on the
// current device.  The attribute belongs to one device, so it is set once per
// (kernel, device) pair: a process that uses several GPUs configures each.
inline cudaError_t smem_limit_per_device(const void* fn, int bytes) {
  static std::mutex mu;
  static std::set<std::pair<const void*, int>> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  if (done.count({fn, dev})) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) done.insert({fn, dev});
  return e;
}

}  // namespace kfm
