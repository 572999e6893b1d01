// Internal (non-ABI) launchers shared by the plan executor and the kernel-level
// entry points.  All matrices are row-major with an explicit leading dimension.
#pragma once

#include "common.cuh"

namespace kfm {

// Epilogue shared by every GEMM flavour.  With acc = sum_k A[i,k] op(B)[k,j]:
//   v_pre = alpha * acc + beta * cin[i,j]          (cin optional)
//   v     = v_pre - csub[i,j]                      (csub optional)
//   out[i,j]  = v                                  (out optional)
//   out2[i,j] = v_pre + Q[i,j]                     (out2 optional; Q per q_kind,
//                                                   q_kind < 0: no Q)
//   diag_out[i] = v_pre at i == j                  (optional, float64)
// sym == 1: M == N, only tiles on or below the diagonal are computed and each
// written element (i >= j) is mirrored to (j, i), so outputs are exactly
// symmetric.  sym == 2: as 1 but without the mirror (lower triangle only).  check_diag != 0: a diagonal v_pre that is not finite and > 0
// sets KF_ERR_NUMERIC in status with the given step.
template <typename T>
struct GemmParams {
  int M = 0, N = 0, K = 0;
  const T* A = nullptr;
  int64_t lda = 0;
  const T* B = nullptr;
  int64_t ldb = 0;
  T alpha = T(1);
  const T* cin = nullptr;
  int64_t ldcin = 0;
  T beta = T(0);
  const T* csub = nullptr;
  int64_t ldcsub = 0;
  T* out = nullptr;
  int64_t ldo = 0;
  T* out2 = nullptr;
  int64_t ldo2 = 0;
  float* outf = nullptr;  // optional float32 copy of out (v), mirrored like out
  int64_t ldof = 0;
  int q_kind = -1;
  const double* q = nullptr;
  int64_t ldq = 0;
  double* diag_out = nullptr;
  int* status = nullptr;
  int check_diag = 0;
  int step = 0;
  int sym = 0;
  // Tensor-core path only: transA = 1 means A is stored K x M (row-major) and
  // is used transposed.  tri_a / tri_b: +1 when row r of the operand as used
  // (A: M x K, op(B): N x K) is zero for k > r, -1 when zero for k < r, so
  // k-tiles outside the band are skipped; 0 = dense.
  int transA = 0;
  int tri_a = 0, tri_b = 0;
  // Smoother gain from an inverse (J = I - Q P^{-1}, F = I): when gain_q is
  // set, out receives delta_ij - q_i (alpha acc + beta cin) with q_i = gain_q[0]
  // (gain_q_kind 0) or gain_q[i] (1); a mirrored element uses q_j; outf (if
  // set) a float32 copy.
  const double* gain_q = nullptr;
  int gain_q_kind = -1;
};

// C = op(A) x op(B) with A: M x K row-major; B: N x K row-major when transB
// (C = A B^T) else K x N row-major (C = A B).  Plain CUDA-core FMA tiles.
template <typename T>
kf_status gemm_simt(cudaStream_t s, bool transB, const GemmParams<T>& p);
// Pipelined float32 product for small operands (gemm_small.cu); needs 16-byte
// aligned A and B, lda, ldb and K multiples of 4 (and N when !transB), and out
// must not overlap an operand, except out == A with N <= 128 (an in-place row
// transform, run with tiles that own whole rows).
enum class SmallAlias { kNone, kSameRows, kOther };
SmallAlias gemm_small_alias(bool transB, const GemmParams<float>& p);
bool gemm_small_ok(bool transB, const GemmParams<float>& p);
kf_status gemm_small(cudaStream_t s, bool transB, const GemmParams<float>& p);

// Blocked right-looking Cholesky A = L L^T of the n x n lower triangle (in
// place; the strict upper triangle is left untouched).  dinv receives the
// inverses of the nb x nb diagonal blocks of L (ceil(n/nb) blocks of nb*nb,
// each row-major with leading dimension nb).  A pivot that is not > 0 sets
// KF_ERR_NOT_PD in status (step, pivot index) and stops the factorisation.
template <typename T>
kf_status potrf(cudaStream_t s, T* A, int64_t lda, int n, T* dinv, int nb, int* status, int step);

template <typename T>
int potrf_block();  // the nb used by potrf for dtype T

// One diagonal block (n <= 64 for float64, <= 128 for float32): L = chol(A)
// in place (lower triangle) and L^{-1} written to dinv (leading dimension
// ldd, zero above the diagonal).  base = index of the block's first pivot.
template <typename T>
kf_status potrf_diag(cudaStream_t s, T* A, int64_t lda, int n, T* dinv, int64_t ldd, int* status, int step,
                     int base);

// B <- B L^{-T} (trans = true) or B <- B L^{-1} (trans = false), B: M x n,
// L: n x n lower triangular from potrf with its diagonal-block inverses dinv.
template <typename T>
kf_status trsm_right(cudaStream_t s, bool trans, int M, int n, const T* L, int64_t ldl,
                     const T* dinv, int nb, T* B, int64_t ldb, int* status);

// ---------------------------------------------------------------- small ops

// dst[i, j] = (Tdst) src[i, j] for i < rows, j < cols; pad columns cols..ld_dst-1 zeroed
// when zero_pad.
template <typename Tdst, typename Tsrc>
kf_status copy2d(cudaStream_t s, Tdst* dst, int64_t ldd, const Tsrc* src, int64_t lds,
                 int64_t rows, int64_t cols, bool zero_pad = false);

// dst = src + Q (Q per q_kind, q_kind < 0: none), dst may alias src.
template <typename Tdst, typename Tsrc>
kf_status add_cov(cudaStream_t s, Tdst* dst, int64_t ldd, const Tsrc* src, int64_t lds, int64_t n,
                  int q_kind, const double* q);

// y[i] = sum_j A[i, j] x[j] (float64 accumulate); y = ybase + sign * A x when ybase.
template <typename T>
kf_status gemv(cudaStream_t s, int64_t rows, int64_t cols, const T* A, int64_t lda,
               const double* x, const double* ybase, double sign, double* y);

// As gemv for a float32 matrix with float64 products and sums (a float64-accurate product of
// the float32 values, e.g. a residual d - P y).
kf_status gemv_f64acc(cudaStream_t s, int64_t rows, int64_t cols, const float* A, int64_t lda, const double* x,
                      const double* ybase, double sign, double* y);

// y[j] = sum_i A[i, j] x[i] (float64), y = ybase + sign A^T x when ybase.
kf_status gemv_t(cudaStream_t s, int64_t rows, int64_t cols, const double* A, int64_t lda, const double* x,
                 const double* ybase, double sign, double* y);

// J = I - Q X (n x n float32) for Q = q I (q_kind 0) or diagonal (q_kind 1).
kf_status identity_minus_q(cudaStream_t s, int64_t n, const float* X, int64_t ldx, int q_kind, const double* q,
                           float* J, int64_t ldj);

// out = a + d - Q y for Q = q I (q_kind 0) or diagonal (q_kind 1), float64 vectors.
kf_status mean_update_q(cudaStream_t s, int64_t n, const double* a, const double* d, int q_kind, const double* q,
                        const double* yv, double* out);

// status[ST_CUR] = step (read by graph-replayed kernels that report failures)
kf_status set_status_step(cudaStream_t s, int* status, int step);

// dst = I (n x n, leading dimension ld), float64.
kf_status eye(cudaStream_t s, int64_t n, double* dst, int64_t ld);

// dst[j][i] = src[i][j] for a rows x cols float64 src.
kf_status transpose(cudaStream_t s, int64_t rows, int64_t cols, const double* src, int64_t lds, double* dst,
                    int64_t ldd);

// d[i] = a[i] - b[i]
kf_status vsub(cudaStream_t s, int64_t n, const double* a, const double* b, double* d);

// innovation: nu = y - H x (m values); non-finite y or nu sets KF_ERR_NUMERIC.
kf_status innovation(cudaStream_t s, int64_t m, int64_t N, const double* H, const double* x,
                     const double* y, double* nu, int* status, int step);

// S = H U^T-product + R (m x m, float64), summing float64 partials from
// split-K chunks of  sum_k H[i, k] Ut[k, j]  (H: m x N float64, Ut: N x m of T).
template <typename T, typename TH>
kf_status innovation_cov(cudaStream_t s, int m, int N, const TH* H, int64_t ldh, const T* Ut,
                         int64_t ldu, int r_kind, const double* R, double* S, int64_t lds,
                         double* partials, int splits);

// Mean prediction x_out = F x (F per f_kind; identity copies).
kf_status predict_mean(cudaStream_t s, int f_kind, int64_t N, const double* F,
                       const int64_t* rowptr, const int64_t* col, const double* x, double* x_out);

// Mesh coupling: out = F P F^T + Q for CSR F (P symmetric, N x N), via
// W = F P (row combinations) then out = W F^T (gathers within each row of W).
template <typename T>
kf_status spmm_fpft(cudaStream_t s, int64_t N, const int64_t* rowptr, const int64_t* col,
                    const double* val, const T* P, int64_t ldp, T* W, int64_t ldw, T* out,
                    int64_t ldo, int q_kind, const double* q);

// B = P F^T for CSR F (B[i, j] = sum_k P[i, k] F[j, k]).
template <typename T>
kf_status spmm_pft(cudaStream_t s, int64_t N, const int64_t* rowptr, const int64_t* col,
                   const double* val, const T* P, int64_t ldp, T* out, int64_t ldo);

// Splits float A (rows x cols, lda) into `n` (2 or 3) bf16 planes:
// plane k = bf16(A - plane 0 - .. - plane k-1) (round to nearest); columns
// cols..ldh-1 of every plane are zeroed.
kf_status split_bf16(cudaStream_t s, int64_t rows, int64_t cols, const float* A, int64_t lda,
                     __nv_bfloat16* const* planes, int n, int64_t ldh);

// Splits the two operands of one product in a single launch: for op = A, B,
// planes (rows x ldh) of src (rows x cols) or of its transpose when trans
// (src is then cols x rows).
struct SplitOp {
  const void* src = nullptr;  // float32, or float64 when f64
  int64_t ld = 0, rows = 0, cols = 0;
  int trans = 0;
  int f64 = 0;
  __nv_bfloat16* planes[3] = {nullptr, nullptr, nullptr};
};
kf_status split_bf16_pair(cudaStream_t s, const SplitOp& a, const SplitOp& b, int n, int64_t ldh);

// As split_bf16 for the transpose: plane[r][k] = split(A[k][r]) for r < rows,
// k < cols, where A is cols x rows with leading dimension lda.
kf_status split_bf16_t(cudaStream_t s, int64_t rows, int64_t cols, const float* A, int64_t lda,
                       __nv_bfloat16* const* planes, int n, int64_t ldh);

// diag_out[i] = A[i, i]
template <typename T>
kf_status diag_extract(cudaStream_t s, int64_t n, const T* A, int64_t lda, double* diag_out);

}  // namespace kfm
