// Smoother-gain solve on the tensor cores (mixed mode, float32-class solve).
//
// J_t = P_{t|t} F^T P_{t+1|t}^{-1} (eqn 11) is formed as
//   P_{t+1|t} = L L^T,   W = L^{-1},   J_t = ((P_{t|t} F^T) W^T) W,
// so that, apart from the nb x nb diagonal blocks, all O(N^3) work is large
// products that run as three-way split-bf16 GEMMs (six bf16 products with
// float32 accumulation, float32-class accuracy) on the tensor cores:
//  - Cholesky, recursive on halves:  L11 = chol(A11);  L21 = A21 W11^T;
//    A22 <- A22 - L21 L21^T;  L22 = chol(A22);
//  - triangular inverse on the same halves: W21 = -W22 (L21 W11);
//  - the diagonal blocks (nb = 128) are factored and inverted by one CTA each.
// Products with a triangular operand skip the k-tiles outside its band.  The
// small products near the leaves run in float32 on the CUDA cores, where
// their latency is a fraction of a tensor-core launch.
// This replaces the two triangular solves with N right-hand sides by a
// triangular inverse and two triangular products (2.67 N^3 instead of
// 2.33 N^3 flops), in exchange for large, fully parallel products only.
// With F = I and a scalar or diagonal Q the gain needs no product with
// P_{t|t} at all: J_t = P_{t|t} (P_{t|t} + Q)^{-1} = I - Q P_{t+1|t}^{-1}, and
// P_{t+1|t}^{-1} = W^T W costs N^3 / 3 and the gain is formed in the product's
// epilogue (gain_identity_tc).
#include <set>
#include <utility>

#include "solve_tc.cuh"

namespace kfm {

namespace {

struct Ctx {
  cudaStream_t s;
  TcScratch* sc;
  int* status;
  int step;
  float* L;
  int64_t ldl;
  float* W;
  int64_t ldw;
  float* T;
  int64_t ldt;
  int nb;
  std::set<std::pair<int, int>> done;
};

int split_point(int n, int nb) { return (int)round_up((n + 1) / 2, nb); }

// Products up to about 640^3 are latency-bound on the tensor-core path (an
// operand split plus the tensor-core kernel cost ~30 us at any size below
// 512^3); they run as pipelined float32 CUDA-core products instead.
constexpr int64_t kSmallWork = int64_t(1) << 28;

kf_status gemm(Ctx& c, const GemmParams<float>& g, bool transB) {
  if ((int64_t)g.M * g.N * g.K <= kSmallWork) {
    if (gemm_small_ok(transB, g)) return gemm_small(c.s, transB, g);
    if (gemm_small_alias(transB, g) == SmallAlias::kOther && g.A != c.T && g.B != c.T && !g.cin && !g.csub) {
      // in place wider than one tile (L21 = A21 W11^T): through the scratch T
      GemmParams<float> t = g;
      t.out = c.T;
      t.ldo = c.ldt;
      if (gemm_small_ok(transB, t)) {
        KF_TRY(gemm_small(c.s, transB, t));
        return copy2d<float, float>(c.s, g.out, g.ldo, c.T, c.ldt, g.M, g.N);
      }
    }
  }
  // the tensor-core path splits both operands into scratch first, so in place is safe there
  return tc_gemm_split(c.s, *c.sc, g, 3, transB);
}

kf_status trtri_rec(Ctx& c, int off, int n) {
  if (c.done.count({off, n})) return KF_OK;
  if (n <= c.nb) return KF_ERR_ARG;  // leaves come from potrf_diag
  const int n1 = split_point(n, c.nb), n2 = n - n1;
  KF_TRY(trtri_rec(c, off, n1));
  KF_TRY(trtri_rec(c, off + n1, n2));
  // T = L21 W11   (n2 x n1; op(B) = W11^T has row j zero for k < j)
  GemmParams<float> a;
  a.M = n2; a.N = n1; a.K = n1;
  a.A = c.L + (int64_t)(off + n1) * c.ldl + off; a.lda = c.ldl;
  a.B = c.W + (int64_t)off * c.ldw + off; a.ldb = c.ldw;
  a.tri_b = -1;
  a.out = c.T; a.ldo = c.ldt;
  a.status = c.status;
  KF_TRY(gemm(c, a, false));
  // W21 = -W22 T   (W22 lower triangular)
  GemmParams<float> b;
  b.M = n2; b.N = n1; b.K = n2;
  b.A = c.W + (int64_t)(off + n1) * c.ldw + off + n1; b.lda = c.ldw;
  b.tri_a = 1;
  b.B = c.T; b.ldb = c.ldt;
  b.alpha = -1.0f;
  b.out = c.W + (int64_t)(off + n1) * c.ldw + off; b.ldo = c.ldw;
  b.status = c.status;
  KF_TRY(gemm(c, b, false));
  c.done.insert({off, n});
  return KF_OK;
}

kf_status potrf_rec(Ctx& c, int off, int n) {
  if (n <= c.nb) {
    KF_TRY(potrf_diag<float>(c.s, c.L + (int64_t)off * c.ldl + off, c.ldl, n, c.W + (int64_t)off * c.ldw + off,
                             c.ldw, c.status, c.step, off));
    c.done.insert({off, n});
    return KF_OK;
  }
  const int n1 = split_point(n, c.nb), n2 = n - n1;
  KF_TRY(potrf_rec(c, off, n1));
  KF_TRY(trtri_rec(c, off, n1));
  float* A21 = c.L + (int64_t)(off + n1) * c.ldl + off;
  // L21 = A21 W11^T  (row j of W11 is zero for k > j)
  GemmParams<float> p;
  p.M = n2; p.N = n1; p.K = n1;
  p.A = A21; p.lda = c.ldl;
  p.B = c.W + (int64_t)off * c.ldw + off; p.ldb = c.ldw;
  p.tri_b = 1;
  p.out = A21; p.ldo = c.ldl;
  p.status = c.status;
  KF_TRY(gemm(c, p, true));
  // A22 <- A22 - L21 L21^T on the lower triangle
  GemmParams<float> u;
  u.M = n2; u.N = n2; u.K = n1;
  u.A = A21; u.lda = c.ldl;
  u.B = A21; u.ldb = c.ldl;
  u.alpha = -1.0f;
  u.cin = c.L + (int64_t)(off + n1) * c.ldl + off + n1; u.ldcin = c.ldl; u.beta = 1.0f;
  u.out = c.L + (int64_t)(off + n1) * c.ldl + off + n1; u.ldo = c.ldl;
  u.sym = 2;
  u.status = c.status;
  KF_TRY(gemm(c, u, true));
  return potrf_rec(c, off + n1, n2);
}

}  // namespace

kf_status chol_inverse_tc(cudaStream_t s, TcScratch& sc, int n, float* L, int64_t ldl, float* W, int64_t ldw,
                          float* T, int64_t ldt, int* status, int step) {
  Ctx c{s, &sc, status, step, L, ldl, W, ldw, T, ldt, 128, {}};
  KF_TRY(potrf_rec(c, 0, n));
  if (n > c.nb) KF_TRY(trtri_rec(c, 0, n));
  return KF_OK;
}

kf_status gain_from_inverse_tc(cudaStream_t s, TcScratch& sc, int n, const float* Bm, int64_t ldb, const float* W,
                               int64_t ldw, float* Z, int64_t ldz, float* J, int64_t ldj, int* status) {
  GemmParams<float> a;  // Z = Bm W^T  (row j of W zero for k > j)
  a.M = n; a.N = n; a.K = n;
  a.A = Bm; a.lda = ldb;
  a.B = W; a.ldb = ldw;
  a.tri_b = 1;
  a.out = Z; a.ldo = ldz;
  a.status = status;
  KF_TRY(tc_gemm_split(s, sc, a, 3, true));
  GemmParams<float> b;  // J = Z W   (op(B) = W^T, row j zero for k < j)
  b.M = n; b.N = n; b.K = n;
  b.A = Z; b.lda = ldz;
  b.B = W; b.ldb = ldw;
  b.tri_b = -1;
  b.out = J; b.ldo = ldj;
  b.status = status;
  return tc_gemm_split(s, sc, b, 3, false);
}

kf_status gain_identity_tc(cudaStream_t s, TcScratch& sc, int n, const float* W, int64_t ldw, int q_kind,
                           const double* q, float* J, int64_t ldj, int* status) {
  if (q_kind != 0 && q_kind != 1) return KF_ERR_ARG;
  GemmParams<float> g;  // J = I - Q (W^T W): lower triangle computed, the upper one mirrored with q_j
  g.M = n; g.N = n; g.K = n;
  g.out = J; g.ldo = ldj;
  g.gain_q = q;
  g.gain_q_kind = q_kind;
  g.sym = 1;
  g.tri_a = -1;  // row r of W^T is zero for k < r
  g.tri_b = -1;
  g.status = status;
  return tc_gemm_ops(s, sc, TcOperand{W, ldw, 0, 1}, TcOperand{W, ldw, 0, 1}, g, 3);
}

uint64_t refine_bytes(int64_t n, int64_t ld) {
  const uint64_t mat = round_up((int64_t)(n * ld * 8), 256);
  return 3 * mat + 2 * round_up((int64_t)oz_slice_bytes(n, n, 7), 256);
}

void refine_layout(RefineBufs& rb, void* mem, int64_t n, int64_t ld) {
  const uint64_t mat = round_up((int64_t)(n * ld * 8), 256);
  char* p = static_cast<char*>(mem);
  rb.X0 = reinterpret_cast<double*>(p);
  rb.R = reinterpret_cast<double*>(p + mat);
  rb.X1 = reinterpret_cast<double*>(p + 2 * mat);
  rb.ld = ld;
  oz_slice_layout(rb.Ps, p + 3 * mat, n, n, 7);
  oz_slice_layout(rb.Xs, p + 3 * mat + round_up((int64_t)oz_slice_bytes(n, n, 7), 256), n, n, 7);
}

kf_status refine_inverse_tc(cudaStream_t s, TcScratch& sc, int n, const void* P, int p_f64, int64_t ldp, const float* W,
                            int64_t ldw, RefineBufs& rb, int q_kind, const double* gain_q, double* J64, float* Jf,
                            int64_t ldj, double* X2, int64_t ldx, int* status, int step) {
  if (gain_q && q_kind != 0 && q_kind != 1) return KF_ERR_ARG;
  const int64_t ld = rb.ld;
  {
    GemmParams<double> g;  // X0 = W^T W (lower triangle + mirror; row r of W^T is zero for k < r)
    g.M = n; g.N = n; g.K = n;
    g.out = rb.X0; g.ldo = ld;
    g.sym = 1;
    g.tri_a = -1;
    g.tri_b = -1;
    g.status = status;
    KF_TRY(tc_gemm_ops(s, sc, TcOperand{W, ldw, 0, 1}, TcOperand{W, ldw, 0, 1}, g, 3));
  }
  KF_TRY(oz_slice(s, P, ldp, p_f64, n, n, 7, rb.Ps));
  const double* X = rb.X0;
  for (int k = 0; k < 2; ++k) {
    // R_k = I - P X_k  (X_k symmetric: its rows are the product's columns)
    KF_TRY(oz_slice(s, X, ld, 1, n, n, k == 0 ? 5 : 7, rb.Xs));
    OzEpilogue e;
    e.alpha = -1.0;
    e.delta = 1.0;
    e.out = rb.R;
    e.ldo = ld;
    e.status = status;
    e.step = step;
    KF_TRY(oz_gemm(s, rb.Ps, rb.Xs, n, n, n, k == 0 ? 5 : 7, e));
    // X_{k+1} = X_k + X_k R_k;  C = op(A) op(B)^T with op(B) = R_k^T (R_k stored K x N)
    GemmParams<double> g;
    g.M = n; g.N = n; g.K = n;
    g.cin = X; g.ldcin = ld; g.beta = 1.0;
    g.sym = 1;
    g.status = status;
    g.step = step;
    if (k == 0) {
      g.out = rb.X1; g.ldo = ld;
      KF_TRY(tc_gemm_ops(s, sc, TcOperand{X, ld, 1, 0}, TcOperand{rb.R, ld, 1, 1}, g, 3));
      X = rb.X1;
    } else if (gain_q) {
      // the correction is ~1e-9 of X: two bf16 slices (16 bits) leave it accurate to ~1e-14 of X
      g.gain_q = gain_q; g.gain_q_kind = q_kind;
      g.out = J64; g.ldo = ldj;
      g.outf = Jf; g.ldof = ldj;
      KF_TRY(tc_gemm_ops(s, sc, TcOperand{X, ld, 1, 0}, TcOperand{rb.R, ld, 1, 1}, g, 2));
    } else {
      g.out = X2; g.ldo = ldx;
      KF_TRY(tc_gemm_ops(s, sc, TcOperand{X, ld, 1, 0}, TcOperand{rb.R, ld, 1, 1}, g, 2));
    }
  }
  return KF_OK;
}

}  // namespace kfm
