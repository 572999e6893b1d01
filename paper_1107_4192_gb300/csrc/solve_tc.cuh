// Tensor-core smoother-gain solve (mixed mode with float32 solve).
#pragma once

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

}  // namespace kfm
