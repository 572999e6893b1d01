// kfx_posv_right_static: the Cholesky factorisation and right-side solve of
// kfx_posv_right without any device allocation.
//
// Who needs it: callers that cannot call cudaMalloc / cudaFree when they run
// the solve -- for instance a process whose device memory is reserved up
// front by another allocator (a framework's caching allocator holding the
// whole budget), or a latency-critical loop where cudaFree's implicit
// device-wide synchronisation would stall unrelated streams.  kfx_posv_right
// allocates its scratch (the inverses of the diagonal blocks and a status
// word) on every call; this variant keeps that scratch in one fixed-size
// array in device global memory, reserved when the library is loaded.
//
// Rules that follow from the static scratch:
//  - n is limited to KFX_POSV_STATIC_MAX_N; larger n is rejected before any
//    GPU work with KF_ERR_ARG (and a message on stderr).
//  - All calls in the process share the array, on every stream.  Calls whose
//    GPU work overlaps (different host threads, or different streams without
//    an ordering between them) race on it and give wrong results: order them.
//  - The array keeps the previous call's contents; the status word is cleared
//    at the start of each call, the block inverses are always rewritten
//    before they are read.
//  - The device address of the array is looked up (cudaGetSymbolAddress) on
//    the first call made with a given device current, so that first call
//    should come before any stream capture.
//  - Every GPU that loads the library holds the array until the process exits.
#include <mutex>

#include "../../include/kfmeg_kernels.h"
#include "ops.cuh"

using namespace kfm;

namespace {

// Diagonal-block inverses for n up to KFX_POSV_STATIC_MAX_N in either dtype
// (float64: nb = 64, float32: nb = 128, so at most n * 128 * 4 bytes = 2 MiB),
// followed by the status word.
constexpr size_t kDinvBytes = (size_t)KFX_POSV_STATIC_MAX_N * 128 * sizeof(float);
constexpr size_t kScratchBytes = kDinvBytes + 256;
static_assert(kDinvBytes >= (size_t)KFX_POSV_STATIC_MAX_N * 64 * sizeof(double), "float64 blocks fit");

static __device__ __align__(256) unsigned char g_posv_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once per device).
kf_status scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return KF_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_posv_scratch);
    if (e != cudaSuccess || p == nullptr) {
      fprintf(stderr, "kfx_posv_right_static: cudaGetSymbolAddress failed: %s\n", cudaGetErrorString(e));
      cudaGetLastError();
      return KF_ERR_CUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return KF_OK;
}

}  // namespace

extern "C" kf_status kfx_posv_right_static(int32_t dtype, int64_t n, void* A, int64_t lda, int64_t M, void* B,
                                           int64_t ldb, int64_t* fail_index, void* stream) {
  if (fail_index) *fail_index = -1;
  if (dtype != 0 && dtype != 1) return KF_ERR_ARG;
  if (n < 1 || M < 0 || M > INT32_MAX || !A || lda < n) return KF_ERR_ARG;
  if (B && ldb < n) return KF_ERR_ARG;
  if (n > KFX_POSV_STATIC_MAX_N) {
    fprintf(stderr, "kfx_posv_right_static: n = %lld exceeds the static scratch limit %d\n", (long long)n,
            (int)KFX_POSV_STATIC_MAX_N);
    return KF_ERR_ARG;
  }
  void* base = nullptr;
  KF_TRY(scratch_address(&base));
  cudaStream_t s = (cudaStream_t)stream;
  void* dinv = base;
  int* st = reinterpret_cast<int*>(static_cast<unsigned char*>(base) + kDinvBytes);
  KF_CUDA_TRY(cudaMemsetAsync(st, 0, ST_WORDS * sizeof(int), s));
  kf_status r;
  if (dtype == 0) {
    const int nb = potrf_block<double>();
    r = potrf<double>(s, (double*)A, lda, (int)n, (double*)dinv, nb, st, 0);
    if (r == KF_OK && B && M > 0)
      r = trsm_right<double>(s, true, (int)M, (int)n, (double*)A, lda, (double*)dinv, nb, (double*)B, ldb, st);
    if (r == KF_OK && B && M > 0)
      r = trsm_right<double>(s, false, (int)M, (int)n, (double*)A, lda, (double*)dinv, nb, (double*)B, ldb, st);
  } else {
    const int nb = potrf_block<float>();
    r = potrf<float>(s, (float*)A, lda, (int)n, (float*)dinv, nb, st, 0);
    if (r == KF_OK && B && M > 0)
      r = trsm_right<float>(s, true, (int)M, (int)n, (float*)A, lda, (float*)dinv, nb, (float*)B, ldb, st);
    if (r == KF_OK && B && M > 0)
      r = trsm_right<float>(s, false, (int)M, (int)n, (float*)A, lda, (float*)dinv, nb, (float*)B, ldb, st);
  }
  int h[ST_WORDS] = {0, 0, 0, 0};
  KF_CUDA_TRY(cudaMemcpyAsync(h, st, sizeof(h), cudaMemcpyDeviceToHost, s));
  KF_CUDA_TRY(cudaStreamSynchronize(s));
  if (r != KF_OK) return r;
  if (h[ST_CODE] && fail_index) *fail_index = h[ST_INDEX];
  return (kf_status)h[ST_CODE];
}
