// Kernel-level C entry points (include/kfmeg_kernels.h).
#include <vector>

#include "../../include/kfmeg_kernels.h"
#include "ops.cuh"
#include "ozaki.cuh"
#include "solve_tc.cuh"
#include "tc_gemm.cuh"

using namespace kfm;

namespace {

template <typename T>
kf_status gemm_typed(int32_t dtype, int32_t transB, int32_t sym, int64_t M, int64_t N, int64_t K, double alpha,
                     const void* A, int64_t lda, const void* B, int64_t ldb, double beta, void* C, int64_t ldc,
                     cudaStream_t s) {
  GemmParams<T> g;
  g.M = (int)M; g.N = (int)N; g.K = (int)K;
  g.A = (const T*)A; g.lda = lda;
  g.B = (const T*)B; g.ldb = ldb;
  g.alpha = (T)alpha;
  if (beta != 0.0) {
    g.cin = (const T*)C; g.ldcin = ldc; g.beta = (T)beta;
  }
  g.out = (T*)C; g.ldo = ldc;
  g.sym = sym ? 1 : 0;
  return gemm_simt<T>(s, transB != 0, g);
}

}  // namespace

extern "C" {

kf_status kfx_gemm(int32_t dtype, int32_t transB, int32_t sym, int64_t M, int64_t N, int64_t K, double alpha,
                   const void* A, int64_t lda, const void* B, int64_t ldb, double beta, void* C, int64_t ldc,
                   void* stream) {
  if (M < 0 || N < 0 || K < 0 || M > INT32_MAX || N > INT32_MAX || K > INT32_MAX) return KF_ERR_ARG;
  if ((sym && M != N) || !C || (K > 0 && (!A || !B))) return KF_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  kf_status st;
  if (dtype == 0) {
    st = gemm_typed<double>(dtype, transB, sym, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, s);
  } else if (dtype == 1) {
    st = gemm_typed<float>(dtype, transB, sym, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, s);
  } else if (dtype == 2 || dtype == 3) {
    if (!tc_available()) return KF_ERR_UNSUPPORTED;
    GemmParams<float> g;
    g.M = (int)M; g.N = (int)N; g.K = (int)K;
    g.A = (const float*)A; g.lda = lda;
    g.B = (const float*)B; g.ldb = ldb;
    g.alpha = (float)alpha;
    if (beta != 0.0) {
      g.cin = (const float*)C; g.ldcin = ldc; g.beta = (float)beta;
    }
    g.out = (float*)C; g.ldo = ldc;
    g.sym = sym ? 1 : 0;
    TcScratch sc;
    std::vector<void*> mem;
    int64_t rows = M > N ? M : N;
    int64_t ld = round_up(K > 0 ? K : 1, 64);
    auto alloc = [&](void** ptr, size_t bytes) -> kf_status {
      if (cudaMalloc(ptr, bytes) != cudaSuccess) return KF_ERR_CUDA;
      mem.push_back(*ptr);
      return KF_OK;
    };
    int* status = nullptr;
    st = alloc((void**)&status, ST_WORDS * sizeof(int));
    if (st == KF_OK && cudaMemsetAsync(status, 0, ST_WORDS * sizeof(int), s) != cudaSuccess) st = KF_ERR_CUDA;
    if (st == KF_OK) st = tc_scratch_alloc(sc, rows, ld, alloc);
    g.status = status;
    if (st == KF_OK) st = tc_gemm_split(s, sc, g, dtype == 2 ? 2 : 3, transB != 0);
    int h[ST_WORDS] = {0, 0, 0, 0};
    if (status) cudaMemcpyAsync(h, status, sizeof(h), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    for (void* p : mem) cudaFree(p);
    if (st == KF_OK && h[ST_CODE]) st = (kf_status)h[ST_CODE];
  } else {
    return KF_ERR_ARG;
  }
  if (st != KF_OK) return st;
  KF_CUDA_TRY(cudaStreamSynchronize(s));
  return KF_OK;
}

kf_status kfx_gemm_exact(int32_t levels, int64_t M, int64_t N, int64_t K, double alpha, const void* A, int64_t lda,
                         int32_t a_f32, const void* B, int64_t ldb, int32_t b_f32, double beta, double delta, double* C,
                         int64_t ldc, void* stream) {
  if (M < 1 || N < 1 || K < 1 || M > INT32_MAX || N > INT32_MAX || K > (1 << 20)) return KF_ERR_ARG;
  if (!A || !B || !C || lda < K || ldb < K || ldc < N || levels < 4 || levels > 7) return KF_ERR_ARG;
  if (!tc_available()) return KF_ERR_UNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<void*> mem;
  auto alloc = [&](void** ptr, size_t bytes) -> kf_status {
    if (cudaMalloc(ptr, bytes) != cudaSuccess) return KF_ERR_CUDA;
    mem.push_back(*ptr);
    return KF_OK;
  };
  OzSlices sa, sb;
  void *ma = nullptr, *mb = nullptr;
  int* status = nullptr;
  kf_status st = alloc(&ma, oz_slice_bytes(M, K, levels));
  if (st == KF_OK) st = alloc(&mb, oz_slice_bytes(N, K, levels));
  if (st == KF_OK) st = alloc((void**)&status, ST_WORDS * sizeof(int));
  if (st == KF_OK && cudaMemsetAsync(status, 0, ST_WORDS * sizeof(int), s) != cudaSuccess) st = KF_ERR_CUDA;
  if (st == KF_OK) {
    oz_slice_layout(sa, ma, M, K, levels);
    oz_slice_layout(sb, mb, N, K, levels);
    st = oz_slice(s, A, lda, a_f32 ? 0 : 1, M, K, levels, sa);
  }
  if (st == KF_OK) st = oz_slice(s, B, ldb, b_f32 ? 0 : 1, N, K, levels, sb);
  if (st == KF_OK) {
    OzEpilogue e;
    e.alpha = alpha;
    e.delta = delta;
    if (beta != 0.0) {
      e.cin = C;
      e.ldcin = ldc;
      e.beta = beta;
    }
    e.out = C;
    e.ldo = ldc;
    e.status = status;
    st = oz_gemm(s, sa, sb, (int)M, (int)N, (int)K, levels, e);
  }
  int h[ST_WORDS] = {0, 0, 0, 0};
  if (status) cudaMemcpyAsync(h, status, sizeof(h), cudaMemcpyDeviceToHost, s);
  cudaError_t ce = cudaStreamSynchronize(s);
  for (void* p : mem) cudaFree(p);
  if (st != KF_OK) return st;
  if (ce != cudaSuccess) return KF_ERR_CUDA;
  return (kf_status)h[ST_CODE];
}

kf_status kfx_spd_inverse(int32_t mode, int64_t n, const float* A, int64_t lda, double* X, int64_t ldx,
                          int64_t* fail_index, void* stream) {
  if (fail_index) *fail_index = -1;
  if (n < 1 || n > (1 << 16) || !A || !X || lda < n || ldx < n || (mode != 1 && mode != 2)) return KF_ERR_ARG;
  if (!tc_available()) return KF_ERR_UNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t ld = round_up(n, 128);
  std::vector<void*> mem;
  auto alloc = [&](void** ptr, size_t bytes) -> kf_status {
    if (cudaMalloc(ptr, bytes) != cudaSuccess) return KF_ERR_CUDA;
    mem.push_back(*ptr);
    return KF_OK;
  };
  float *L = nullptr, *W = nullptr, *T = nullptr;
  void* rmem = nullptr;
  int* status = nullptr;
  TcScratch sc;
  kf_status st = alloc((void**)&L, n * ld * 4);
  if (st == KF_OK) st = alloc((void**)&W, n * ld * 4);
  if (st == KF_OK) st = alloc((void**)&T, n * ld * 4);
  if (st == KF_OK) st = alloc((void**)&status, ST_WORDS * sizeof(int));
  if (st == KF_OK && mode == 2) st = alloc(&rmem, refine_bytes(n, ld));
  if (st == KF_OK) st = tc_scratch_alloc(sc, n, ld, alloc);
  if (st == KF_OK && (cudaMemsetAsync(status, 0, ST_WORDS * sizeof(int), s) != cudaSuccess ||
                      cudaMemsetAsync(W, 0, n * ld * 4, s) != cudaSuccess))
    st = KF_ERR_CUDA;
  if (st == KF_OK) st = copy2d<float, float>(s, L, ld, A, lda, n, n, true);
  if (st == KF_OK) st = chol_inverse_tc(s, sc, (int)n, L, ld, W, ld, T, ld, status, 1);
  if (st == KF_OK && mode == 1) {
    GemmParams<double> g;  // X = W^T W
    g.M = (int)n; g.N = (int)n; g.K = (int)n;
    g.out = X; g.ldo = ldx;
    g.sym = 1;
    g.tri_a = -1;
    g.tri_b = -1;
    g.status = status;
    st = tc_gemm_ops(s, sc, TcOperand{W, ld, 0, 1}, TcOperand{W, ld, 0, 1}, g, 3);
  } else if (st == KF_OK) {
    RefineBufs rb;
    refine_layout(rb, rmem, n, ld);
    st = refine_inverse_tc(s, sc, (int)n, A, 0, lda, W, ld, rb, 0, nullptr, nullptr, nullptr, 0,
                           X, ldx, status, 1);
  }
  int h[ST_WORDS] = {0, 0, 0, 0};
  if (status) cudaMemcpyAsync(h, status, sizeof(h), cudaMemcpyDeviceToHost, s);
  cudaError_t ce = cudaStreamSynchronize(s);
  for (void* p : mem) cudaFree(p);
  if (st != KF_OK) return st;
  if (ce != cudaSuccess) return KF_ERR_CUDA;
  if (h[ST_CODE] && fail_index) *fail_index = h[ST_INDEX];
  return (kf_status)h[ST_CODE];
}

kf_status kfx_tc_wait_limit(uint64_t ns, uint64_t* previous) {
  const uint64_t prev = g_tc_wait_ns.exchange(ns == 0 ? kTcDefaultWaitNs : ns);
  if (previous) *previous = prev;
  return KF_OK;
}

kf_status kfx_posv_right(int32_t dtype, int64_t n, void* A, int64_t lda, int64_t M, void* B, int64_t ldb,
                         int64_t* fail_index, void* stream) {
  if (fail_index) *fail_index = -1;
  if (n < 1 || n > INT32_MAX || M < 0 || M > INT32_MAX || !A || lda < n) return KF_ERR_ARG;
  if (B && ldb < n) return KF_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  void* dinv = nullptr;
  int* st = nullptr;
  const int nb = dtype == 0 ? potrf_block<double>() : potrf_block<float>();
  const size_t esz = dtype == 0 ? 8 : 4;
  if (dtype != 0 && dtype != 1) return KF_ERR_ARG;
  KF_CUDA_TRY(cudaMalloc(&dinv, (size_t)round_up(n, nb) * nb * esz));
  if (cudaMalloc(&st, ST_WORDS * sizeof(int)) != cudaSuccess) {
    cudaFree(dinv);
    return KF_ERR_CUDA;
  }
  cudaMemsetAsync(st, 0, ST_WORDS * sizeof(int), s);
  kf_status r;
  if (dtype == 0) {
    r = potrf<double>(s, (double*)A, lda, (int)n, (double*)dinv, nb, st, 0);
    if (r == KF_OK && B && M > 0)
      r = trsm_right<double>(s, true, (int)M, (int)n, (double*)A, lda, (double*)dinv, nb, (double*)B, ldb, st);
    if (r == KF_OK && B && M > 0)
      r = trsm_right<double>(s, false, (int)M, (int)n, (double*)A, lda, (double*)dinv, nb, (double*)B, ldb, st);
  } else {
    r = potrf<float>(s, (float*)A, lda, (int)n, (float*)dinv, nb, st, 0);
    if (r == KF_OK && B && M > 0)
      r = trsm_right<float>(s, true, (int)M, (int)n, (float*)A, lda, (float*)dinv, nb, (float*)B, ldb, st);
    if (r == KF_OK && B && M > 0)
      r = trsm_right<float>(s, false, (int)M, (int)n, (float*)A, lda, (float*)dinv, nb, (float*)B, ldb, st);
  }
  int h[ST_WORDS] = {0, 0, 0, 0};
  cudaMemcpyAsync(h, st, sizeof(h), cudaMemcpyDeviceToHost, s);
  cudaError_t e = cudaStreamSynchronize(s);
  cudaFree(dinv);
  cudaFree(st);
  if (e != cudaSuccess) return KF_ERR_CUDA;
  if (r != KF_OK) return r;
  if (h[ST_CODE] && fail_index) *fail_index = h[ST_INDEX];
  return (kf_status)h[ST_CODE];
}

kf_status kfx_spmm_fpft(int32_t dtype, int64_t N, const int64_t* rowptr, const int64_t* col, const double* val,
                        const void* P, int64_t ldp, void* out, int64_t ldo, int32_t q_kind, const double* Q,
                        void* stream) {
  if (N < 1 || !rowptr || !col || !val || !P || !out || ldp < N || ldo < N) return KF_ERR_ARG;
  if (q_kind > 2 || (q_kind >= 0 && !Q)) return KF_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  void* W = nullptr;
  const size_t esz = dtype == 0 ? 8 : 4;
  if (dtype != 0 && dtype != 1) return KF_ERR_ARG;
  KF_CUDA_TRY(cudaMalloc(&W, (size_t)N * N * esz));
  kf_status r = dtype == 0
                    ? spmm_fpft<double>(s, N, rowptr, col, val, (const double*)P, ldp, (double*)W, N, (double*)out,
                                        ldo, q_kind, Q)
                    : spmm_fpft<float>(s, N, rowptr, col, val, (const float*)P, ldp, (float*)W, N, (float*)out, ldo,
                                       q_kind, Q);
  cudaError_t e = cudaStreamSynchronize(s);
  cudaFree(W);
  if (e != cudaSuccess) return KF_ERR_CUDA;
  return r;
}

kf_status kfx_split_bf16(int64_t rows, int64_t cols, const float* A, int64_t lda, void* hi, void* lo, int64_t ldh,
                         void* stream) {
  if (rows < 0 || cols < 0 || ldh < cols || !A || !hi || !lo) return KF_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  __nv_bfloat16* planes[2] = {(__nv_bfloat16*)hi, (__nv_bfloat16*)lo};
  KF_TRY(split_bf16(s, rows, cols, A, lda, planes, 2, ldh));
  KF_CUDA_TRY(cudaStreamSynchronize(s));
  return KF_OK;
}

}  // extern "C"
