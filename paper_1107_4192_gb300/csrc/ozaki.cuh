// Exact-slice products on the tensor cores: float64-accurate C = A B^T from
// bf16 tcgen05 MMAs (the splitting scheme of Ozaki et al. 2012, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", with the exponent-aligned integer
// slices of Mukunoki, Ozaki, Ogita and Imamura 2020, "DGEMM using Tensor Cores,
// and Its Accurate and Reproducible Versions").
//
// Row r of an operand X (rows x K) is written as
//     X[r][k] ~= 2^(e_r - 7) * sum_{p < S} 2^(-8p) q_p[r][k]
// with e_r the exponent of the row's largest magnitude (max |X[r][:]| < 2^e_r)
// and integer slices q_p in [-128, 128], each exact in bf16: the signed
// base-256 digits (each rounded to nearest, ties to even) of X[r][k] rounded
// to the grid 2^(e_r - 7 - 8(S-1)).  A product of two
// slices is an integer below 2^14, so the sum over k of the products of one
// slice level l = p_A + p_B is an exact integer as long as it stays below 2^24:
// the tensor cores' float32 accumulation (which truncates) then loses nothing.
// The products with l < L are kept (L(L+1)/2 slice pairs); the dropped levels
// and the slices' own truncation leave an error in element (i, j) of about
// 2^(-8L+3) K 2^(e_i + e_j) (per term, 2^(-8L+3) of the row maxima's product):
// 2^-37 for L = 5, 2^-53 for L = 7.
#pragma once

#include "tc_gemm.cuh"

namespace kfm {

// Slices of a rows x cols operand: S planes of rows_pad x ldk bf16 (plane p at
// planes + p * rows_pad * ldk; rows >= rows and columns >= cols are zero) and
// the per-row exponents e_r (rows_pad ints, 0 for zero rows).
struct OzSlices {
  __nv_bfloat16* planes = nullptr;
  int* exps = nullptr;
  int64_t rows = 0, rows_pad = 0, ldk = 0;
  int S = 0;       // planes the memory holds
  int filled = 0;  // planes the last oz_slice wrote
};

// Bytes of the planes and exponents for rows x cols with S slices.
uint64_t oz_slice_bytes(int64_t rows, int64_t cols, int S);
// Points `out` at memory of oz_slice_bytes(rows, cols, S) bytes.
void oz_slice_layout(OzSlices& out, void* mem, int64_t rows, int64_t cols, int S);

// Fills `out` (laid out by oz_slice_layout for at least these rows, cols and
// S slices) from X (float64 when f64, else float32; rows x cols, leading
// dimension ld, row-major).  A non-finite row gives NaN slices.
kf_status oz_slice(cudaStream_t s, const void* X, int64_t ld, int f64, int64_t rows, int64_t cols, int S,
                   OzSlices& out);

// Epilogue of the exact-slice product, float64.  With acc = (A B^T)[i][j]:
//   v = alpha acc + beta cin[i][j] + (i == j ? delta : 0) + Radd[i][j]
//   out[i][j] = v,  outf[i][j] = (float) v,  outT[j][i] = v,
//   out2[i][j] = v + Q[i][j],  diag_out[i] = v at i == j
// (each optional; Radd per radd_kind and Q per q_kind as kf_cov_kind, < 0 =
// none).  check_diag: a diagonal v that is not finite and > 0 raises
// KF_ERR_NUMERIC at `step`.  sym (M == N): only i >= j is computed and out,
// outf and out2 are mirrored to (j, i), so they come out exactly symmetric.
struct OzEpilogue {
  double alpha = 1.0, beta = 0.0, delta = 0.0;
  const double* cin = nullptr;
  int64_t ldcin = 0;
  double* out = nullptr;
  int64_t ldo = 0;
  float* outf = nullptr;
  int64_t ldof = 0;
  double* outT = nullptr;
  int64_t ldoT = 0;
  double* out2 = nullptr;
  int64_t ldo2 = 0;
  int q_kind = -1;
  const double* q = nullptr;
  int64_t ldq = 0;
  int radd_kind = -1;
  const double* radd = nullptr;
  int64_t ldradd = 0;
  double* diag_out = nullptr;
  int check_diag = 0;
  int sym = 0;
  int* status = nullptr;  // KF_ERR_TIMEOUT on an expired wait; kernels skip when already failed
  int step = 0;
};

// Optional event timing of the exact-slice kernel launches alone (installed by a plan while it
// profiles the smoother-gain refinement).
extern thread_local TcLaunchTimer* g_oz_timer;

// C = A B^T for A (M x K) and B (N x K) given by their slices, keeping the
// slice levels l < levels (4 to 7; both operands need at least `levels`
// slices).  K <= 2^20.  splits > 1 divides K among that many CTAs per output
// tile, whose float64 partial sums (splits x M x N doubles at `partials`) are
// added in a fixed order by a second kernel that applies the epilogue.
kf_status oz_gemm(cudaStream_t s, const OzSlices& A, const OzSlices& B, int M, int N, int K, int levels,
                  const OzEpilogue& e, int splits = 1, double* partials = nullptr);

}  // namespace kfm
