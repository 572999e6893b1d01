// Blocked Cholesky factorisation and right-side triangular solves.
//
// Used for the innovation covariance S_t = L L^T (eqn 8, always float64) and
// for the smoother-gain solve J_t = P_{t|t} F^T P_{t+1|t}^{-1} (eqn 11) through
// the Cholesky factor of P_{t+1|t}.  The factorisation is right-looking: each
// nb-wide diagonal block is factored by one CTA in shared memory (which also
// forms the block's inverse), the panel below it is solved as a product with
// that inverse, and the trailing lower triangle is updated by a rank-nb
// product.  The solves reuse the diagonal-block inverses, so every step with
// O(n^3) work is a tiled product.
#include "ops.cuh"

namespace kfm {

template <> int potrf_block<double>() { return 64; }
template <> int potrf_block<float>() { return 128; }

// Factors the n x n (n <= NB) lower triangle at A in shared memory, writes L
// back (lower triangle only) and L^{-1} to dinv (NB x NB, zero above the diagonal).
template <typename T, int NB>
__global__ void __launch_bounds__(256) potrf_diag_kernel(T* A, int64_t lda, int n, T* dinv, int64_t ldd,
                                                         int* status, int step, int base) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int LD = NB + 1;
  T* S = reinterpret_cast<T*>(smem_raw);
  T* X = S + NB * LD;
  __shared__ int fail;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) fail = status_failed(status) ? 1 : 0;  // one read for the whole CTA
  __syncthreads();
  if (fail) return;

  for (int idx = tid; idx < n * n; idx += nt) {
    int i = idx / n, j = idx % n;
    S[i * LD + j] = (j <= i) ? A[(int64_t)i * lda + j] : T(0);
  }
  __syncthreads();

  for (int j = 0; j < n; ++j) {
    if (tid == 0) {
      T d = S[j * LD + j];
      if (!(d > T(0)) || !isfinite((double)d)) {
        fail = 1;
        status_set(status, KF_ERR_NOT_PD, step, base + j);
      } else {
        S[j * LD + j] = Num<T>::sqrt_(d);
      }
    }
    __syncthreads();
    if (fail) return;
    const T ljj = S[j * LD + j];
    for (int i = j + 1 + tid; i < n; i += nt) S[i * LD + j] /= ljj;
    __syncthreads();
    const int r = n - j - 1;
    for (int idx = tid; idx < r * r; idx += nt) {
      int ii = idx / r, kk = idx % r;
      if (kk <= ii) {
        int i = j + 1 + ii, k = j + 1 + kk;
        S[i * LD + k] -= S[i * LD + j] * S[k * LD + j];
      }
    }
    __syncthreads();
  }

  for (int idx = tid; idx < n * n; idx += nt) {
    int i = idx / n, j = idx % n;
    if (j <= i) A[(int64_t)i * lda + j] = S[i * LD + j];
  }

  // X = L^{-1}: thread c owns column c and walks down it (no barrier needed,
  // X[k][c] for k < i was produced by the same thread).
  for (int c = tid; c < NB; c += nt) {
    if (c < n) {
      for (int i = 0; i < c; ++i) X[i * LD + c] = T(0);
      X[c * LD + c] = T(1) / S[c * LD + c];
      for (int i = c + 1; i < n; ++i) {
        T a0 = T(0), a1 = T(0);
        int k = c;
        for (; k + 1 < i; k += 2) {
          a0 = fma(S[i * LD + k], X[k * LD + c], a0);
          a1 = fma(S[i * LD + k + 1], X[(k + 1) * LD + c], a1);
        }
        if (k < i) a0 = fma(S[i * LD + k], X[k * LD + c], a0);
        X[i * LD + c] = -(a0 + a1) / S[i * LD + i];
      }
    }
  }
  __syncthreads();
  for (int idx = tid; idx < n * n; idx += nt) {
    int i = idx / n, j = idx % n;
    dinv[(int64_t)i * ldd + j] = j <= i ? X[i * LD + j] : T(0);
  }
}

template <typename T, int NB>
static kf_status launch_potrf_diag(cudaStream_t s, T* A, int64_t lda, int n, T* dinv, int64_t ldd, int* status,
                                   int step, int base) {
  const size_t smem = 2ull * NB * (NB + 1) * sizeof(T);
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(potrf_diag_kernel<T, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    configured = true;
  }
  potrf_diag_kernel<T, NB><<<1, 256, smem, s>>>(A, lda, n, dinv, ldd, status, step, base);
  ++g_launches;
  return launch_check("potrf_diag");
}

template <typename T>
kf_status potrf_diag(cudaStream_t s, T* A, int64_t lda, int n, T* dinv, int64_t ldd, int* status, int step,
                     int base) {
  if (n <= 64) return launch_potrf_diag<T, 64>(s, A, lda, n, dinv, ldd, status, step, base);
  if (sizeof(T) == 8 || n > 128) return KF_ERR_ARG;
  return launch_potrf_diag<T, 128>(s, A, lda, n, dinv, ldd, status, step, base);
}

template <typename T>
kf_status potrf(cudaStream_t s, T* A, int64_t lda, int n, T* dinv, int nb, int* status, int step) {
  if (nb != potrf_block<T>()) return KF_ERR_ARG;
  for (int k = 0; k < n; k += nb) {
    const int kb = n - k < nb ? n - k : nb;
    T* Akk = A + (int64_t)k * lda + k;
    T* Dk = dinv + (int64_t)(k / nb) * nb * nb;
    KF_TRY(potrf_diag<T>(s, Akk, lda, kb, Dk, nb, status, step, k));
    const int rest = n - k - kb;
    if (rest <= 0) break;
    // panel: L21 = A21 L11^{-T}  (C[r][c] = sum_j A21[r][j] Linv[c][j]); one column tile
    GemmParams<T> g;
    g.M = rest; g.N = kb; g.K = kb;
    g.A = A + (int64_t)(k + kb) * lda + k; g.lda = lda;
    g.B = Dk; g.ldb = nb;
    g.out = A + (int64_t)(k + kb) * lda + k; g.ldo = lda;
    g.status = status;
    KF_TRY(gemm_simt<T>(s, true, g));
    // trailing lower triangle: A22 -= L21 L21^T
    GemmParams<T> h;
    h.M = rest; h.N = rest; h.K = kb;
    h.A = A + (int64_t)(k + kb) * lda + k; h.lda = lda;
    h.B = h.A; h.ldb = lda;
    h.alpha = T(-1);
    h.cin = A + (int64_t)(k + kb) * lda + k + kb; h.ldcin = lda; h.beta = T(1);
    h.out = A + (int64_t)(k + kb) * lda + k + kb; h.ldo = lda;
    h.sym = 2;
    h.status = status;
    KF_TRY(gemm_simt<T>(s, true, h));
  }
  return KF_OK;
}

template <typename T>
kf_status trsm_right(cudaStream_t s, bool trans, int M, int n, const T* L, int64_t ldl,
                     const T* dinv, int nb, T* B, int64_t ldb, int* status) {
  if (M <= 0 || n <= 0) return KF_OK;
  if (trans) {
    // Z L^T = B, block columns in increasing order.
    for (int j = 0; j < n; j += nb) {
      const int jb = n - j < nb ? n - j : nb;
      const T* Dj = dinv + (int64_t)(j / nb) * nb * nb;
      GemmParams<T> g;  // Z_j = B_j L_jj^{-T}, in place (one column tile owns all jb columns)
      g.M = M; g.N = jb; g.K = jb;
      g.A = B + j; g.lda = ldb;
      g.B = Dj; g.ldb = nb;
      g.out = B + j; g.ldo = ldb;
      g.status = status;
      KF_TRY(gemm_simt<T>(s, true, g));
      const int rest = n - j - jb;
      if (rest <= 0) break;
      GemmParams<T> h;  // B[:, j+jb:] -= Z_j L[j+jb:, j:j+jb]^T
      h.M = M; h.N = rest; h.K = jb;
      h.A = B + j; h.lda = ldb;
      h.B = L + (int64_t)(j + jb) * ldl + j; h.ldb = ldl;
      h.alpha = T(-1);
      h.cin = B + j + jb; h.ldcin = ldb; h.beta = T(1);
      h.out = B + j + jb; h.ldo = ldb;
      h.status = status;
      KF_TRY(gemm_simt<T>(s, true, h));
    }
  } else {
    // X L = B, block columns in decreasing order.
    for (int j = ((n - 1) / nb) * nb; j >= 0; j -= nb) {
      const int jb = n - j < nb ? n - j : nb;
      const T* Dj = dinv + (int64_t)(j / nb) * nb * nb;
      GemmParams<T> g;  // X_j = B_j L_jj^{-1}, in place
      g.M = M; g.N = jb; g.K = jb;
      g.A = B + j; g.lda = ldb;
      g.B = Dj; g.ldb = nb;
      g.out = B + j; g.ldo = ldb;
      g.status = status;
      KF_TRY(gemm_simt<T>(s, false, g));
      if (j == 0) break;
      GemmParams<T> h;  // B[:, :j] -= X_j L[j:j+jb, :j]
      h.M = M; h.N = j; h.K = jb;
      h.A = B + j; h.lda = ldb;
      h.B = L + (int64_t)j * ldl; h.ldb = ldl;
      h.alpha = T(-1);
      h.cin = B; h.ldcin = ldb; h.beta = T(1);
      h.out = B; h.ldo = ldb;
      h.status = status;
      KF_TRY(gemm_simt<T>(s, false, h));
    }
  }
  return KF_OK;
}

template kf_status potrf_diag<double>(cudaStream_t, double*, int64_t, int, double*, int64_t, int*, int, int);
template kf_status potrf_diag<float>(cudaStream_t, float*, int64_t, int, float*, int64_t, int*, int, int);
template kf_status potrf<double>(cudaStream_t, double*, int64_t, int, double*, int, int*, int);
template kf_status potrf<float>(cudaStream_t, float*, int64_t, int, float*, int, int*, int);
template kf_status trsm_right<double>(cudaStream_t, bool, int, int, const double*, int64_t,
                                      const double*, int, double*, int64_t, int*);
template kf_status trsm_right<float>(cudaStream_t, bool, int, int, const float*, int64_t,
                                     const float*, int, float*, int64_t, int*);

}  // namespace kfm
