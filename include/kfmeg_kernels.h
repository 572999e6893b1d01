/*
 * Kernel-level entry points of libkfmeg.so: the individual GPU operations
 * that kf_filter / fis_smooth chain together, exposed so they can be checked
 * one by one.  Same conventions as kfmeg.h: DEVICE pointers, row-major with
 * explicit leading dimensions (in elements), work enqueued on `stream`
 * (a cudaStream_t) and finished before return.  dtype: 0 = float64,
 * 1 = float32, 2 = float32 data multiplied as split bf16 (hi*hi + hi*lo +
 * lo*hi) on the tensor cores with float32 accumulation.
 */
#ifndef KFMEG_KERNELS_H
#define KFMEG_KERNELS_H

#include "kfmeg.h"

#ifdef __cplusplus
extern "C" {
#endif

/* C = alpha * A op(B) + beta * C.  A: M x K.  transB = 1: B is N x K and
 * op(B) = B^T; transB = 0: B is K x N.  sym = 1 (M == N): only the lower
 * triangle is computed and mirrored, so C comes out exactly symmetric (the
 * form of every covariance product in eqns 7, 10 and 13).  dtype 2 needs
 * transB = 1.  Returns KF_ERR_ARG on bad sizes, KF_ERR_UNSUPPORTED when the
 * dtype is not available. */
kf_status kfx_gemm(int32_t dtype, int32_t transB, int32_t sym, int64_t M, int64_t N, int64_t K,
                   double alpha, const void* A, int64_t lda, const void* B, int64_t ldb,
                   double beta, void* C, int64_t ldc, void* stream);

/* C = alpha A B^T + beta C + delta I to float64 accuracy on the tensor cores:
 * the exact-slice product (Ozaki et al. 2012; exponent-aligned integer slices
 * as in Mukunoki et al. 2020) that forms the float64 residuals of the
 * smoother-gain solve (eqn 11; see kfx_spd_inverse).  Row i of A and row j of
 * B are cut into `levels` slices of 8 bits below their largest magnitude; the
 * slice products whose levels sum to less than `levels` are accumulated
 * exactly and summed in 64-bit integers, so element (i, j) is within about
 * 2^(5 - 8 levels) K max|A[i,:]| max|B[j,:]| of the exact product (2^-51 for
 * levels = 7, float64 class; 2^-35 for levels = 5).  A row of A or B holding an
 * infinity or NaN gives a NaN row or column of C.
 *   A: M x K, B: N x K (row-major, leading dimensions lda, ldb), float64, or
 *      float32 when a_f32 / b_f32 is set.  C: M x N float64 (in/out when
 *      beta != 0).  K <= 2^20.  levels: 4 to 7.
 * Allocates its slice buffers (about 2 levels (M + N) K bytes) for the call.
 * Returns KF_ERR_ARG on bad sizes, KF_ERR_UNSUPPORTED without tcgen05. */
kf_status kfx_gemm_exact(int32_t levels, int64_t M, int64_t N, int64_t K, double alpha, const void* A, int64_t lda,
                         int32_t a_f32, const void* B, int64_t ldb, int32_t b_f32, double beta, double delta, double* C,
                         int64_t ldc, void* stream);

/* X = A^{-1} for a symmetric positive definite float32 A (n x n, lower
 * triangle read), float64 X (n x n, full), on the tensor cores: the inverse
 * the smoother gain of eqn 11 needs (J_t = P_{t|t} F^T P_{t+1|t}^{-1}).
 *   mode 1: float32-class: recursive Cholesky A = L L^T, W = L^{-1} (split-bf16
 *           products, float32 diagonal blocks), X = W^T W;
 *   mode 2: float64-accurate: mode 1's X refined by two Newton steps
 *           X <- X + X (I - A X) whose residuals I - A X are exact-slice
 *           products (kfx_gemm_exact with 5, then 7 levels): the result
 *           agrees with a float64 inversion to float64 rounding times the
 *           condition number.
 * A non-positive pivot returns KF_ERR_NOT_PD with *fail_index (else -1).
 * Allocates its work buffers for the call. */
kf_status kfx_spd_inverse(int32_t mode, int64_t n, const float* A, int64_t lda, double* X, int64_t ldx,
                          int64_t* fail_index, void* stream);

/* Limit, in nanoseconds of the GPU's global timer, of every pipeline wait
 * (an mbarrier phase a warp of the tensor-core kernels waits for: operands
 * landed, accumulator ready, stage free) in kernels launched after this call;
 * ns = 0 restores the default of 2 s.  A wait that runs out makes the kernel
 * stop issuing work, wait for what it already issued, free its tensor memory
 * and raise KF_ERR_TIMEOUT in the calling entry point's status word, which
 * that entry point returns (its outputs are then undefined).  Limits below
 * 1 ms poll without suspending the waiting warp.  The setting is process-wide
 * (all threads and devices).  *previous (if not NULL) receives the old limit.
 * This is a failure-detection control of the library; the paper has no
 * counterpart. */
kf_status kfx_tc_wait_limit(uint64_t ns, uint64_t* previous);

/* Cholesky A = L L^T (lower, in place, n x n; the upper triangle outside the
 * diagonal blocks is untouched), then B <- B A^{-1} = B L^{-T} L^{-1} for the
 * M x n matrix B (skipped when B is NULL).  This is the solve of the smoother
 * gain, eqn 11 (J = P_{t|t} F^T P_{t+1|t}^{-1}), and of the Kalman gain, eqn 8
 * (K = P H^T S^{-1}).  dtype 0 or 1.  A non-positive pivot returns
 * KF_ERR_NOT_PD with *fail_index = its 0-based index (else -1). */
kf_status kfx_posv_right(int32_t dtype, int64_t n, void* A, int64_t lda, int64_t M, void* B,
                         int64_t ldb, int64_t* fail_index, void* stream);

/* kfx_posv_right without device allocation, for callers that cannot call
 * cudaMalloc / cudaFree when the solve runs (device memory reserved up front
 * by another allocator; loops where cudaFree's device-wide synchronisation
 * would stall other streams).  The paper has no counterpart: this is a
 * calling convention of the library, not part of the method.  Scratch lives
 * in one static device array of about 2 MiB that every GPU loading the
 * library keeps until exit, so n <= KFX_POSV_STATIC_MAX_N (larger n returns
 * KF_ERR_ARG before any GPU work).  All calls share that array: calls whose
 * GPU work overlaps (other threads or unordered streams) race and must be
 * ordered by the caller.  The first call on each device looks up the array's
 * address and should come before any stream capture.  Arguments and results
 * as kfx_posv_right. */
#define KFX_POSV_STATIC_MAX_N 4096
kf_status kfx_posv_right_static(int32_t dtype, int64_t n, void* A, int64_t lda, int64_t M, void* B,
                                int64_t ldb, int64_t* fail_index, void* stream);

/* out = F P F^T + Q for F in compressed-row form (rowptr: N+1, col/val: nnz),
 * the mesh-coupled prediction of eqns 2-3 / eqn 7.  dtype 0 or 1 for P / out;
 * Q per q_kind (kf_cov_kind, float64, NULL allowed with q_kind = -1). */
kf_status kfx_spmm_fpft(int32_t dtype, int64_t N, const int64_t* rowptr, const int64_t* col,
                        const double* val, const void* P, int64_t ldp, void* out, int64_t ldo,
                        int32_t q_kind, const double* Q, void* stream);

/* Splits float32 A (rows x cols) into bf16 planes hi = bf16(A) and
 * lo = bf16(A - hi) (round to nearest), leading dimension ldh >= cols; the
 * pad columns are zeroed.  The operand form of the split-bf16 products. */
kf_status kfx_split_bf16(int64_t rows, int64_t cols, const float* A, int64_t lda, void* hi, void* lo,
                         int64_t ldh, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* KFMEG_KERNELS_H */
