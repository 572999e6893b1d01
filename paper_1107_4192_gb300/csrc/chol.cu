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
#include <mutex>

#include "ops.cuh"

namespace kfm {

template <> int potrf_block<double>() { return 64; }
template <> int potrf_block<float>() { return 128; }

// Factors the n x n (n <= NB) lower triangle at A in shared memory, writes L
// back (lower triangle only) and L^{-1} to dinv (leading dimension ldd, zero
// above the diagonal).  The block is padded to NB with an identity, so the
// algorithm always runs on NB = 32 * P rows:
//   for each 32-wide panel: one warp factors the 32 x 32 diagonal block in
//   registers (shuffles, no block barrier) and inverts it; the rows below are
//   solved against that inverse; the trailing lower triangle gets a rank-32
//   update with register-blocked threads.
// The inverse is then assembled by block forward substitution,
//   X_pq = -X_pp sum_{r=q}^{p-1} L_pr X_rq.
template <typename T, int NB>
struct DiagSmem {
  static constexpr int LD = NB + 1;
  static constexpr int NP = NB / 32;
  static constexpr int TSZ = NP * 32 * 33;
  static constexpr size_t bytes = (2ull * NB * LD + TSZ) * sizeof(T);
};

template <typename T, int BS>
__device__ __forceinline__ void trailing_update(T* S, int LD, int j0, int r0, int tx, int ty) {
  // S[i][k] -= sum_c S[i][j0+c] S[k][j0+c] for i, k >= r0, k <= i; thread block (ty, tx) of BS x BS
  T acc[BS][BS];
#pragma unroll
  for (int a = 0; a < BS; ++a)
#pragma unroll
    for (int b = 0; b < BS; ++b) acc[a][b] = T(0);
  const int i0 = r0 + ty * BS, k0 = r0 + tx * BS;
  if (k0 > i0 + BS - 1) return;  // block entirely above the diagonal
#pragma unroll 2
  for (int c = 0; c < 32; ++c) {
    T li[BS], lk[BS];
#pragma unroll
    for (int a = 0; a < BS; ++a) li[a] = S[(i0 + a) * LD + j0 + c];
#pragma unroll
    for (int b = 0; b < BS; ++b) lk[b] = S[(k0 + b) * LD + j0 + c];
#pragma unroll
    for (int a = 0; a < BS; ++a)
#pragma unroll
      for (int b = 0; b < BS; ++b) acc[a][b] = fma(li[a], lk[b], acc[a][b]);
  }
#pragma unroll
  for (int a = 0; a < BS; ++a)
#pragma unroll
    for (int b = 0; b < BS; ++b)
      if (k0 + b <= i0 + a) S[(i0 + a) * LD + k0 + b] -= acc[a][b];
}

template <typename T, int NB>
__global__ void __launch_bounds__(256, 1) potrf_diag_kernel(T* A, int64_t lda, int n, T* dinv, int64_t ldd,
                                                         int* status, int step, int base) {
  using Cfg = DiagSmem<T, NB>;
  constexpr int LD = Cfg::LD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* S = reinterpret_cast<T*>(smem_raw);
  T* X = S + NB * LD;
  T* Tb = X + NB * LD;
  __shared__ int fail;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid / 32, lane = tid % 32;
  if (tid == 0) fail = status_failed(status) ? 1 : 0;  // one read for the whole CTA
  __syncthreads();
  if (fail) return;

  for (int i = tid / 32; i < NB; i += nt / 32) {
    for (int j = tid % 32; j < NB; j += 32) {
      T v = T(0);
      if (i < n && j < n) {
        if (j <= i) v = A[(int64_t)i * lda + j];
      } else if (i == j) {
        v = T(1);
      }
      S[i * LD + j] = v;
      X[i * LD + j] = T(0);
    }
  }
  __syncthreads();

  for (int p = 0; p < Cfg::NP; ++p) {
    const int j0 = p * 32;
    // (a) one warp: factor and invert the 32 x 32 diagonal block
    if (warp == 0) {
      // Right-looking factorisation of the 32 x 32 block in shared memory, lane i
      // owning row i.  The step loop stays rolled (small code); inside a step
      // the 32 column entries come in registers (shuffles) and the row update
      // is 32 independent predicated load-fma-store triples.
      T* P = S + j0 * LD + j0;
      T* Xp = X + j0 * LD + j0;
      int bad = -1;
      for (int j = 0; j < 32; ++j) {
        const T d = P[j * LD + j];
        if (!(d > T(0) && d < T(INFINITY))) {
          bad = j;
          break;
        }
        T ljj, rinv;
        if constexpr (sizeof(T) == 4) {  // reciprocal square root plus one Newton step (about 1 ulp)
          float r = rsqrtf((float)d);
          r = r * (1.5f - 0.5f * (float)d * r * r);
          rinv = (T)r;
          ljj = d * rinv;
        } else {
          ljj = Num<T>::sqrt_(d);
          rinv = T(1) / ljj;
        }
        T lij = T(0);
        if (lane > j) lij = P[lane * LD + j] * rinv;
        else if (lane == j) lij = ljj;
        if (lane >= j) P[lane * LD + j] = lij;
        Tb[lane] = lij;  // column j, broadcast through shared memory
        __syncwarp();
        T col[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) col[k] = Tb[k];
        // branch-free: every lane touches all 32 entries of its row, with the
        // update masked to j < k <= lane (entries above the diagonal stay zero)
#pragma unroll
        for (int k = 0; k < 32; ++k) {
          const T w = (k > j && k <= lane) ? lij : T(0);
          P[lane * LD + k] = fma(-w, col[k], P[lane * LD + k]);
        }
        __syncwarp();  // the next pivot is read from another lane's row
      }
      __syncwarp();
      if (bad >= 0) {
        if (lane == 0) {
          fail = 1;
          status_set(status, KF_ERR_NOT_PD, step, base + j0 + bad);
        }
      } else {
        // lane c computes column c of the block inverse, rows in order:
        // x_i = (delta_ic - sum_{c<=k<i} L_ik x_k) / L_ii
        for (int i = 0; i < 32; ++i) {
          // branch-free: X is zero above its diagonal (k < lane), and k >= i is masked
          T acc0 = (i == lane) ? T(1) : T(0), acc1 = T(0);
#pragma unroll
          for (int k = 0; k < 32; k += 2) {
            const T l0 = k < i ? P[i * LD + k] : T(0);
            const T l1 = k + 1 < i ? P[i * LD + k + 1] : T(0);
            acc0 = fma(-l0, Xp[k * LD + lane], acc0);
            acc1 = fma(-l1, Xp[(k + 1) * LD + lane], acc1);
          }
          Xp[i * LD + lane] = i >= lane ? (acc0 + acc1) / P[i * LD + i] : T(0);
        }
      }
    }
    __syncthreads();
    if (fail) return;
    const int r0 = j0 + 32, R = NB - r0;
    if (R <= 0) break;
    // (b) panel below: L[i][j0+c] = sum_{k<=c} A[i][j0+k] X[j0+c][j0+k], staged through Tb
    for (int item = tid; item < R * 8; item += nt) {
      const int i = r0 + item / 8, c0 = (item % 8) * 4;
      T o[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll 8
      for (int k = 0; k < 32; ++k) {
        const T av = S[i * LD + j0 + k];
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) o[cc] = fma(av, X[(j0 + c0 + cc) * LD + j0 + k], o[cc]);
      }
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) Tb[(item / 8) * 33 + c0 + cc] = o[cc];
    }
    __syncthreads();
    for (int idx = tid; idx < R * 32; idx += nt) S[(r0 + idx / 32) * LD + j0 + idx % 32] = Tb[(idx / 32) * 33 + idx % 32];
    __syncthreads();
    // (c) trailing rank-32 update of the lower triangle, 16 x 16 threads
    {
      const int tx = tid % 16, ty = tid / 16;
      if (R == 96) trailing_update<T, 6>(S, LD, j0, r0, tx, ty);
      else if (R == 64) trailing_update<T, 4>(S, LD, j0, r0, tx, ty);
      else if (R == 32) trailing_update<T, 2>(S, LD, j0, r0, tx, ty);
    }
    __syncthreads();
  }

  // (d) assemble the inverse: X_pq = -X_pp sum_{r=q}^{p-1} L_pr X_rq
  for (int p = 1; p < Cfg::NP; ++p) {
    for (int item = tid; item < p * 32 * 8; item += nt) {
      const int q = item / 256, rr = (item % 256) / 8, c0 = (item % 8) * 4;
      T o[4] = {T(0), T(0), T(0), T(0)};
      for (int kb = 32 * q; kb < 32 * p; kb += 32) {
#pragma unroll 8
        for (int kk = 0; kk < 32; ++kk) {
          const int k = kb + kk;
          const T lv = S[(32 * p + rr) * LD + k];
#pragma unroll
          for (int cc = 0; cc < 4; ++cc) o[cc] = fma(lv, X[k * LD + 32 * q + c0 + cc], o[cc]);
        }
      }
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) Tb[(q * 32 + rr) * 33 + c0 + cc] = o[cc];
    }
    __syncthreads();
    for (int item = tid; item < p * 32 * 8; item += nt) {
      const int q = item / 256, rr = (item % 256) / 8, c0 = (item % 8) * 4;
      T o[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll 8
      for (int k = 0; k < 32; ++k) {  // X_pp is zero above its diagonal
        const T xv = X[(32 * p + rr) * LD + 32 * p + k];
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) o[cc] = fma(xv, Tb[(q * 32 + k) * 33 + c0 + cc], o[cc]);
      }
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) X[(32 * p + rr) * LD + 32 * q + c0 + cc] = -o[cc];
    }
    __syncthreads();
  }

  for (int i = tid / 32; i < n; i += nt / 32) {
    for (int j = tid % 32; j < n; j += 32) {
      if (j <= i) A[(int64_t)i * lda + j] = S[i * LD + j];
      dinv[(int64_t)i * ldd + j] = j <= i ? X[i * LD + j] : T(0);
    }
  }
}

template <typename T, int NB>
static kf_status launch_potrf_diag(cudaStream_t s, T* A, int64_t lda, int n, T* dinv, int64_t ldd, int* status,
                                   int step, int base) {
  const size_t smem = DiagSmem<T, NB>::bytes;
  static std::once_flag configured;
  static cudaError_t cfg_err = cudaSuccess;
  std::call_once(configured, [&] {
    cfg_err = cudaFuncSetAttribute(potrf_diag_kernel<T, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  KF_CUDA_TRY(cfg_err);
  potrf_diag_kernel<T, NB><<<1, 256, smem, s>>>(A, lda, n, dinv, ldd, status, step, base);
  note_launch();
  return launch_check("potrf_diag");
}

template <typename T>
kf_status potrf_diag(cudaStream_t s, T* A, int64_t lda, int n, T* dinv, int64_t ldd, int* status, int step,
                     int base) {
  if (n <= 32) return launch_potrf_diag<T, 32>(s, A, lda, n, dinv, ldd, status, step, base);
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
