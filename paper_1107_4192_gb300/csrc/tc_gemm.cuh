// Tensor-core (tcgen05) split-bf16 GEMM used by the mixed-precision path.
#pragma once

#include <cuda.h>

#include <functional>

#include "ops.cuh"

namespace kfm {

// Per-plan scratch: up to three bf16 planes of each operand of one product.
struct TcScratch {
  __nv_bfloat16* a[3] = {nullptr, nullptr, nullptr};
  __nv_bfloat16* b[3] = {nullptr, nullptr, nullptr};
  int64_t rows = 0, ld = 0;  // capacity: rows x ld elements per plane
};

uint64_t tc_scratch_bytes(int64_t rows, int64_t ld);
kf_status tc_scratch_alloc(TcScratch& sc, int64_t rows, int64_t ld,
                           const std::function<kf_status(void**, size_t)>& alloc);

// Optional event timing of the tensor-core kernel launches alone (without the
// operand split), installed by a plan while it profiles a phase.
struct TcLaunchTimer {
  virtual void before(cudaStream_t s) = 0;
  virtual void after(cudaStream_t s) = 0;
  virtual ~TcLaunchTimer() = default;
};
extern thread_local TcLaunchTimer* g_tc_timer;

// Limit (ns of %globaltimer) of the tensor-core kernels' pipeline waits,
// passed to each launch; the default is 2 s.
extern std::atomic<uint64_t> g_tc_wait_ns;
constexpr uint64_t kTcDefaultWaitNs = 2000000000ull;

// True when the library was compiled with the tcgen05 kernels.
bool tc_available();

// 2-D TMA map of a bf16 matrix (rows x cols, leading dimension ld elements,
// 16-byte aligned rows) with a box of box_cols x box_rows and the given
// swizzle (32, 64 or 128 bytes; the box row must be that wide).
kf_status tma_map_bf16(CUtensorMap* map, const void* ptr, int64_t rows, int64_t cols, int64_t ld, int box_cols,
                       int box_rows, int swizzle_bytes);

// C = op(A) op(B) for float32 operands: A is M x K (or K x M with g.transA),
// B is N x K when transB (C = A B^T) or K x N otherwise.  Each operand is
// split into `slices` bf16 planes (2 or 3), transposing on the way where
// needed, and the products of slice levels i + j < slices are accumulated in
// float32 on the tensor cores (3 products for 2 slices, 6 for 3), followed by
// the epilogue of GemmParams.  The tensor-core accumulator is promoted into
// float32 registers after every 64-wide k-tile: the tensor cores' own
// accumulation truncates, a bias that would otherwise grow with K.  g.tri_a / g.tri_b skip zero k-tiles of
// triangular operands.
kf_status tc_gemm_split(cudaStream_t s, TcScratch& sc, const GemmParams<float>& g, int slices, bool transB = true);

// An operand given by pointer, leading dimension, precision and orientation:
// the product uses rows of op = (trans ? X^T : X), each of K elements.
struct TcOperand {
  const void* p;
  int64_t ld;
  int f64;    // 1: float64 data (split from its float64 value), 0: float32
  int trans;  // 1: X is stored K x rows and used transposed
};

// As tc_gemm_split with separately described operands; the epilogue (and
// its cin / out / out2) is float64 or float32.  The A / B / transA fields of
// epi are ignored.  Float64 epilogues add the float32 products to float64
// values, which keeps the covariance itself at float64 precision.
kf_status tc_gemm_ops(cudaStream_t s, TcScratch& sc, const TcOperand& A, const TcOperand& B,
                      const GemmParams<double>& epi, int slices);
kf_status tc_gemm_ops(cudaStream_t s, TcScratch& sc, const TcOperand& A, const TcOperand& B,
                      const GemmParams<float>& epi, int slices);

}  // namespace kfm
