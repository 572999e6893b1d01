// Minimum-norm estimate, eqn 5:  X[t] = lambda C H^T (lambda H C H^T + R)^{-1} y_t
// for all T rows of Y at once, float64 throughout.  G = lambda H C H^T + R is
// factored by the same blocked Cholesky as S_t; W = Y G^{-1} is two right-side
// triangular solves; X = lambda W H C is one product (plus a column scaling
// when C is diagonal).
//
// mne_init: the paper's initialisation from these estimates (Sec. 2.4):
// x0 = X[0] and Q = the sample covariance of the differences X[k+1] - X[k].
#include <vector>

#include "ops.cuh"

using namespace kfm;

namespace {

__global__ void scale_cols_kernel(int64_t rows, int64_t cols, double* X, int64_t ldx, int c_kind, const double* c,
                                  double lam) {
  for (int64_t i = blockIdx.y; i < rows; i += gridDim.y)
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < cols; j += (int64_t)gridDim.x * blockDim.x) {
      double w = c_kind == 0 ? c[0] : c[j];
      X[i * ldx + j] *= lam * w;
    }
}

struct Tmp {
  std::vector<void*> v;
  ~Tmp() {
    for (void* p : v) cudaFree(p);
  }
  kf_status get(double** out, size_t n) {
    void* p = nullptr;
    if (cudaMalloc(&p, n * sizeof(double) + 16) != cudaSuccess) {
      cudaGetLastError();
      return KF_ERR_CUDA;
    }
    v.push_back(p);
    *out = (double*)p;
    return KF_OK;
  }
};

}  // namespace

extern "C" kf_status mne_solve(const double* H, const double* C, int32_t c_kind, const double* R, int32_t r_kind,
                               const double* Y, int64_t N, int64_t m, int64_t T, double lambda, double* X_out,
                               void* stream) {
  if (!H || !C || !R || !Y || !X_out || N < 1 || m < 1 || T < 1) return KF_ERR_ARG;
  if (c_kind < 0 || c_kind > 2 || r_kind < 0 || r_kind > 2 || !(lambda > 0)) return KF_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  Tmp tmp;
  double *HC, *G, *partials, *dinv, *W, *status;
  const int nb = potrf_block<double>();
  const int splits = 8;
  KF_TRY(tmp.get(&HC, (size_t)m * N));
  KF_TRY(tmp.get(&G, (size_t)m * m));
  KF_TRY(tmp.get(&partials, (size_t)splits * m * m));
  KF_TRY(tmp.get(&dinv, (size_t)round_up(m, nb) * nb));
  KF_TRY(tmp.get(&W, (size_t)T * m));
  KF_TRY(tmp.get(&status, ST_WORDS));
  int* st = (int*)status;
  KF_CUDA_TRY(cudaMemsetAsync(st, 0, ST_WORDS * sizeof(int), s));
  // HC = H C  (m x N)
  if (c_kind == KF_COV_DENSE) {
    GemmParams<double> g;
    g.M = (int)m; g.N = (int)N; g.K = (int)N;
    g.A = H; g.lda = N;
    g.B = C; g.ldb = N;
    g.out = HC; g.ldo = N;
    KF_TRY(gemm_simt<double>(s, false, g));
  } else {
    KF_CUDA_TRY(cudaMemcpyAsync(HC, H, (size_t)m * N * 8, cudaMemcpyDeviceToDevice, s));
    dim3 grid((unsigned)std::min<int64_t>(ceil_div(N, 256), 64), (unsigned)std::min<int64_t>(m, 65535));
    scale_cols_kernel<<<grid, 256, 0, s>>>(m, N, HC, N, c_kind, C, 1.0);
    note_launch();
    KF_TRY(launch_check("scale_cols"));
  }
  // G = lambda (H C) H^T + R, symmetric by construction
  {
    GemmParams<double> g;
    g.M = (int)m; g.N = (int)m; g.K = (int)N;
    g.A = HC; g.lda = N;
    g.B = H; g.ldb = N;
    g.alpha = lambda;
    g.out2 = G; g.ldo2 = m;
    g.q_kind = r_kind; g.q = R; g.ldq = m;
    g.sym = 1;
    KF_TRY(gemm_simt<double>(s, true, g));
  }
  KF_TRY(potrf<double>(s, G, m, (int)m, dinv, nb, st, 0));
  KF_CUDA_TRY(cudaMemcpyAsync(W, Y, (size_t)T * m * 8, cudaMemcpyDeviceToDevice, s));
  KF_TRY(trsm_right<double>(s, true, (int)T, (int)m, G, m, dinv, nb, W, m, st));
  KF_TRY(trsm_right<double>(s, false, (int)T, (int)m, G, m, dinv, nb, W, m, st));
  // X = lambda W (H C)
  {
    GemmParams<double> g;
    g.M = (int)T; g.N = (int)N; g.K = (int)m;
    g.A = W; g.lda = m;
    g.B = HC; g.ldb = N;
    g.alpha = lambda;
    g.out = X_out; g.ldo = N;
    KF_TRY(gemm_simt<double>(s, false, g));
  }
  int h[ST_WORDS];
  KF_CUDA_TRY(cudaMemcpyAsync(h, st, sizeof(h), cudaMemcpyDeviceToHost, s));
  KF_CUDA_TRY(cudaStreamSynchronize(s));
  return (kf_status)h[ST_CODE];
}

namespace {

// Dt[i][k] = (X[k+1][i] - X[k][i]) - dbar_i for k < T - 1, where the mean of the
// differences telescopes to dbar_i = (X[T-1][i] - X[0][i]) / (T - 1).
__global__ void centred_differences_kernel(int64_t N, int64_t T, const double* X, double* Dt) {
  const int64_t K = T - 1;
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < N * K; u += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = u / N, i = u % N;  // consecutive threads read consecutive sources of one row
    const double dbar = (X[(T - 1) * N + i] - X[i]) / (double)K;
    Dt[i * K + k] = (X[(k + 1) * N + i] - X[k * N + i]) - dbar;
  }
}

}  // namespace

extern "C" kf_status mne_init(const double* H, const double* C, int32_t c_kind, const double* R, int32_t r_kind,
                              const double* Y, int64_t N, int64_t m, int64_t T, double lambda, double* X_out,
                              double* x0_out, double* Q_out, void* stream) {
  if (!x0_out || !Q_out || T < 3 || N < 1 || N > INT32_MAX) return KF_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  Tmp tmp;
  double* X = X_out;
  if (!X) KF_TRY(tmp.get(&X, (size_t)T * N));
  KF_TRY(mne_solve(H, C, c_kind, R, r_kind, Y, N, m, T, lambda, X, stream));
  KF_CUDA_TRY(cudaMemcpyAsync(x0_out, X, (size_t)N * 8, cudaMemcpyDeviceToDevice, s));
  double* Dt;
  KF_TRY(tmp.get(&Dt, (size_t)N * (T - 1)));
  const unsigned blocks = (unsigned)std::min<int64_t>(ceil_div(N * (T - 1), 256), 152 * 16);
  centred_differences_kernel<<<blocks, 256, 0, s>>>(N, T, X, Dt);
  note_launch();
  KF_TRY(launch_check("centred_differences"));
  GemmParams<double> g;  // Q = Dt Dt^T / (T - 2), lower triangle computed and mirrored
  g.M = (int)N; g.N = (int)N; g.K = (int)(T - 1);
  g.A = Dt; g.lda = T - 1;
  g.B = Dt; g.ldb = T - 1;
  g.alpha = 1.0 / (double)(T - 2);
  g.out = Q_out; g.ldo = N;
  g.sym = 1;
  KF_TRY(gemm_simt<double>(s, true, g));
  KF_CUDA_TRY(cudaStreamSynchronize(s));
  return KF_OK;
}
