// Tensor-core smoother-gain solve (mixed mode with float32 solve).
#pragma once

#include "ozaki.cuh"
#include "tc_gemm.cuh"

namespace kfm {

// In place: L (n x n, lower triangle used) <- chol(L); W <- L^{-1} (lower, the
// strict upper triangle of W must be zero on entry and stays zero).  T is
// scratch of at least n x n.  A non-positive pivot sets KF_ERR_NOT_PD (step).
kf_status chol_inverse_tc(cudaStream_t s, TcScratch& sc, int n, float* L, int64_t ldl, float* W, int64_t ldw,
                          float* T, int64_t ldt, int* status, int step);

// J = (Bm W^T) W for W = L^{-1} from chol_inverse_tc, i.e. J = Bm (L L^T)^{-1};
// Z is n x n scratch.
kf_status gain_from_inverse_tc(cudaStream_t s, TcScratch& sc, int n, const float* Bm, int64_t ldb, const float* W,
                               int64_t ldw, float* Z, int64_t ldz, float* J, int64_t ldj, int* status);

// F = I with Q = q I or diagonal: J = P_{t|t} (P_{t|t} + Q)^{-1} = I - Q P_{t+1|t}^{-1},
// with P_{t+1|t}^{-1} = W^T W formed on the lower triangle (n^3 / 3 instead of
// the 2 n^3 of the two triangular products); J is written by that product's
// epilogue, so P_{t+1|t}^{-1} itself is never stored.
kf_status gain_identity_tc(cudaStream_t s, TcScratch& sc, int n, const float* W, int64_t ldw, int q_kind,
                           const double* q, float* J, int64_t ldj, int* status);

// Buffers of refine_inverse_tc: three n x ld float64 matrices and the slices
// of P (7 slices) and of the iterate (7 slices).
struct RefineBufs {
  double *X0 = nullptr, *R = nullptr, *X1 = nullptr;
  int64_t ld = 0;
  OzSlices Ps, Xs;
};
uint64_t refine_bytes(int64_t n, int64_t ld);
void refine_layout(RefineBufs& rb, void* mem, int64_t n, int64_t ld);

// Inverse of the symmetric positive definite P (float32, or float64 when p_f64; n x n) to float64
// accuracy, from W = L^{-1} of its float32-class factor (chol_inverse_tc):
//   X0 = W^T W;   R_k = I - P X_k;   X_{k+1} = X_k + X_k R_k   (k = 0, 1)
// (Newton's iteration for the inverse, quadratically convergent from the
// float32-class X0).  The residuals are exact-slice products (5 slice levels
// for R_0, 7 for R_1), the corrections split-bf16 products with float64
// epilogues (X_k R_k is symmetric: lower triangle + mirror).  The last
// correction is fused into its consumer:
//  - gain_q != NULL (F = I, Q = q I or diagonal): J = I - Q X_2 into J64
//    (float64) and Jf (float32), X_2 itself never stored;
//  - gain_q == NULL: X_2 into X2 (float64, n x ldx).
kf_status refine_inverse_tc(cudaStream_t s, TcScratch& sc, int n, const void* P, int p_f64, int64_t ldp, const float* W,
                            int64_t ldw, RefineBufs& rb, int q_kind, const double* gain_q, double* J64, float* Jf,
                            int64_t ldj, double* X2, int64_t ldx, int* status, int step);

}  // namespace kfm
