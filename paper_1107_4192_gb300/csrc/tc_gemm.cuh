// Tensor-core (tcgen05) split-bf16 GEMM used by the mixed-precision path.
#pragma once

#include <functional>

#include "ops.cuh"

namespace kfm {

// Per-plan scratch: bf16 hi/lo planes of the two operands of one product.
struct TcScratch {
  __nv_bfloat16 *a_hi = nullptr, *a_lo = nullptr, *b_hi = nullptr, *b_lo = nullptr;
  int64_t rows = 0, ld = 0;  // capacity: rows x ld elements per plane
};

uint64_t tc_scratch_bytes(int64_t rows, int64_t ld);
kf_status tc_scratch_alloc(TcScratch& sc, int64_t rows, int64_t ld,
                           const std::function<kf_status(void**, size_t)>& alloc);

// True when this build carries the tcgen05 kernels.
bool tc_available();

// C = A B^T with A: M x K, B: N x K float32 (row-major), computed as
// hi(A) hi(B)^T + hi(A) lo(B)^T + lo(A) hi(B)^T on the tensor cores with
// float32 accumulation, followed by the epilogue of GemmParams.
kf_status tc_gemm_bf16x3(cudaStream_t s, TcScratch& sc, const GemmParams<float>& g);

}  // namespace kfm
