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
// algorithm always runs on NB = 32 * NP rows:
//   for each 32-wide panel, the tall panel (its diagonal block and all rows
//   below) is factored column by column, each warp holding 32 rows in
//   registers; one warp owns the diagonal block and publishes the pivot and
//   the column through shared memory, a named barrier per column;
//   the trailing lower triangle then gets a rank-32 update.
// The inverse follows once L is complete: each 32 x 32 diagonal block is
// inverted by one warp (lane c solves for column c), and the off-diagonal
// blocks are filled by recursive doubling on 32- then 64-wide halves,
//   X_BA = -X_BB (L_BA X_AA).
template <typename T, int NB>
struct DiagSmem {
  static constexpr int LD = NB + 1;     // odd stride: rows and columns both free of bank conflicts
  static constexpr int NP = NB / 32;
  static constexpr int LA = 36;         // 16-byte aligned row stride of the diagonal-block copies
  static constexpr int al(int x) { return (x + 3) / 4 * 4; }
  static constexpr int TSZ = NB >= 64 ? (NB / 2) * (NB / 2 + 1) : 4;
  static constexpr int oS = 0;
  static constexpr int oX = oS + al(NB * LD);
  static constexpr int oT = oX + al(NB * LD);
  static constexpr int oL = oT + al(TSZ);
  static constexpr int oB = oL + NP * 32 * LA;
  static constexpr int oR = oB + 2 * LA;
  static constexpr int total = oR + al(NB);
  static constexpr size_t bytes = (size_t)total * sizeof(T);
};

template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; };
template <> struct Vec16<double> { using type = double2; };

__device__ __forceinline__ void bar_named(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// q ~ 1 / sqrt(d) and l = sqrt(d) for a pivot d
__device__ __forceinline__ void pivot(float d, float& q, float& l) {
  float r = rsqrtf(d);  // one Newton step brings the estimate to about 1 ulp
  r = r * (1.5f - 0.5f * d * r * r);
  q = r;
  l = d * r;
}
__device__ __forceinline__ void pivot(double d, double& q, double& l) {
  l = sqrt(d);
  q = 1.0 / l;
}

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

// One level of the recursive-doubling inverse: for every pair of bs-wide
// diagonal blocks (A above B), stage 0 forms Tm = L_BA X_AA and stage 1 forms
// X_BA = -X_BB Tm.  Thread tiles are 4 x 4 with rows and columns strided by
// bs / 4, so the lanes of a warp read consecutive columns.  X_AA and X_BB are
// lower block-triangular at this point (their upper-right bs/2 quadrant is
// zero: the diagonal inverses are lower triangular, the blocks above the
// diagonal were zeroed), so stage 0 skips, for k < bs/2, the columns in the
// right half (tile columns b >= 2), and stage 1 skips, for k >= bs/2, the rows
// in the upper half (tile rows a < 2).
template <typename T, int NB, int bs, int STAGE>
__device__ __forceinline__ void inverse_stage(const T* S, T* X, T* Tm, int tid) {
  constexpr int LD = NB + 1, R = bs / 4, NPAIR = NB / (2 * bs), LT = bs + 1, H2 = bs / 2;
  for (int t = tid; t < NPAIR * R * R; t += 256) {
    const int q = t / (R * R), ti = (t % (R * R)) / R, tj = t % R;
    const int a0 = 2 * q * bs, b0 = a0 + bs;
    const T* Am = STAGE == 0 ? S + b0 * LD + a0 : X + b0 * LD + b0;
    const T* Bm = STAGE == 0 ? X + a0 * LD + a0 : Tm + q * bs * LT;
    constexpr int ldb = STAGE == 0 ? LD : LT;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
    // k < bs/2: stage 0 has zero B in the right half
    constexpr int B_LO = STAGE == 0 ? 2 : 4;
#pragma unroll 4
    for (int k = 0; k < H2; ++k) {
      T av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = Am[(ti + R * a) * LD + k];
#pragma unroll
      for (int b = 0; b < B_LO; ++b) bv[b] = Bm[k * ldb + tj + R * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < B_LO; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
    // k >= bs/2: stage 1 has zero A in the upper half
    constexpr int A_HI0 = STAGE == 1 ? 2 : 0;
#pragma unroll 4
    for (int k = H2; k < bs; ++k) {
      T av[4], bv[4];
#pragma unroll
      for (int a = A_HI0; a < 4; ++a) av[a] = Am[(ti + R * a) * LD + k];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bm[k * ldb + tj + R * b];
#pragma unroll
      for (int a = A_HI0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
    T* out = STAGE == 0 ? Tm + q * bs * LT : X + b0 * LD + a0;
    constexpr int ldo = STAGE == 0 ? LT : LD;
    const T sgn = STAGE == 0 ? T(1) : T(-1);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) out[(ti + R * a) * ldo + tj + R * b] = sgn * acc[a][b];
  }
}

template <typename T, int NB, int bs>
__device__ __forceinline__ void inverse_level(const T* S, T* X, T* Tm, int tid) {
  inverse_stage<T, NB, bs, 0>(S, X, Tm, tid);
  __syncthreads();
  inverse_stage<T, NB, bs, 1>(S, X, Tm, tid);
  __syncthreads();
}

template <typename T, int NB>
__global__ void __launch_bounds__(256, 1) potrf_diag_kernel(T* A, int64_t lda, int n, T* dinv, int64_t ldd,
                                                         int* status, int step, int base) {
  using Cfg = DiagSmem<T, NB>;
  using V = typename Vec16<T>::type;
  constexpr int LD = Cfg::LD, LA = Cfg::LA, E = 16 / sizeof(T);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  T* S = sm + Cfg::oS;
  T* X = sm + Cfg::oX;
  T* Tm = sm + Cfg::oT;
  T* Lal = sm + Cfg::oL;
  T* buf = sm + Cfg::oB;
  T* rdiag = sm + Cfg::oR;
  __shared__ int fail;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid / 32, lane = tid % 32;
  if (tid == 0) fail = status_failed(status) ? 1 : 0;  // one read for the whole CTA
  __syncthreads();
  if (fail) return;

  // Full, 16-byte aligned blocks move as 16-byte vectors: lane (r, c8) of a
  // warp takes row 4u + r, vector 8v + c8 of its unit, so both the global
  // accesses (four 128-byte rows) and the odd-stride shared stores are
  // conflict-free.  Ragged or unaligned blocks take the scalar path.
  constexpr int VPR = NB / E, UNITS = NB * VPR / 32, CH = VPR / 8;
  const bool vec = n == NB && (reinterpret_cast<uintptr_t>(A) & 15) == 0 && lda % E == 0 &&
                   (reinterpret_cast<uintptr_t>(dinv) & 15) == 0 && ldd % E == 0;
  if (vec) {
    V v[UNITS / 8];
#pragma unroll
    for (int it = 0; it < UNITS / 8; ++it) {
      const int u = it * 8 + warp, i = (u / CH) * 4 + lane / 8, j = ((u % CH) * 8 + lane % 8) * E;
      v[it] = *reinterpret_cast<const V*>(A + (int64_t)i * lda + j);
    }
#pragma unroll
    for (int it = 0; it < UNITS / 8; ++it) {
      const int u = it * 8 + warp, i = (u / CH) * 4 + lane / 8, j = ((u % CH) * 8 + lane % 8) * E;
      const T* ve = reinterpret_cast<const T*>(&v[it]);
#pragma unroll
      for (int e = 0; e < E; ++e) S[i * LD + j + e] = ve[e];  // the upper triangle of S is never read
    }
  } else {
    for (int i = tid / 32; i < NB; i += nt / 32) {
      for (int j = tid % 32; j < NB; j += 32) {
        T v = T(0);
        if (i < n && j < n) {
          if (j <= i) v = A[(int64_t)i * lda + j];
        } else if (i == j) {
          v = T(1);
        }
        S[i * LD + j] = v;
      }
    }
  }
  // the only parts of X read before they are written: the 32 x 32 blocks
  // above the diagonal inside each 64-wide diagonal block
  for (int t = tid; t < (NB / 64) * 1024; t += nt) {
    const int a0 = (t / 1024) * 64, i = (t % 1024) / 32, j = t % 32;
    X[(a0 + i) * LD + a0 + 32 + j] = T(0);
  }
  __syncthreads();

  for (int p = 0; p < Cfg::NP; ++p) {
    const int j0 = 32 * p;
    const int nw = Cfg::NP - p;  // warps holding the tall panel, warp 0 on its diagonal block
    if (warp < nw) {
      const int i = j0 + 32 * warp + lane;
      T r[32];
#pragma unroll
      for (int k = 0; k < 32; ++k) r[k] = S[i * LD + j0 + k];
      int bad = -1;
      T dnext = T(0);  // warp 0: the next pivot, taken before this column's shared-memory round trip
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        T* bj = buf + (j & 1) * LA;  // two buffers: a column is written while the previous one may be read
        T q, l;
        if (warp == 0) {
          const T d = j == 0 ? __shfl_sync(0xffffffffu, r[0], 0) : dnext;
          if (bad < 0 && !(d > T(0) && d < T(INFINITY))) bad = j;
          T ljj;
          pivot(d, q, ljj);
          l = lane > j ? r[j] * q : (lane == j ? ljj : T(0));
          // lane j + 1's diagonal after this column is its entry minus its own l squared,
          // exactly what the update below computes for it
          if (j < 31) dnext = __shfl_sync(0xffffffffu, fma(-l, l, r[j + 1]), j + 1);
          bj[lane] = l;
          if (lane == 0) {
            bj[32] = q;
            rdiag[j0 + j] = q;
          }
        }
        bar_named(1, 32 * nw);
        if (warp != 0) {
          q = bj[32];
          l = r[j] * q;
        }
        r[j] = l;
#pragma unroll
        for (int g = (j + 1) / E; g < 32 / E; ++g) {
          const V v = reinterpret_cast<const V*>(bj)[g];
          const T* ve = reinterpret_cast<const T*>(&v);
#pragma unroll
          for (int e = 0; e < E; ++e)
            if (g * E + e > j) r[g * E + e] = fma(-l, ve[e], r[g * E + e]);
        }
      }
      if (warp == 0) {
#pragma unroll
        for (int k = 0; k < 32; ++k) {
          if (k <= lane) S[i * LD + j0 + k] = r[k];
          Lal[(p * 32 + lane) * LA + k] = k <= lane ? r[k] : T(0);
        }
        if (lane == 0 && bad >= 0) {
          fail = 1;
          status_set(status, KF_ERR_NOT_PD, step, base + j0 + bad);
        }
      } else {
#pragma unroll
        for (int k = 0; k < 32; ++k) S[i * LD + j0 + k] = r[k];
      }
    }
    __syncthreads();
    if (fail) return;
    const int r0 = j0 + 32, R = NB - r0;
    if (R <= 0) break;
    // trailing rank-32 update of the lower triangle, 16 x 16 threads
    {
      const int tx = tid % 16, ty = tid / 16;
      if (R == 96) trailing_update<T, 6>(S, LD, j0, r0, tx, ty);
      else if (R == 64) trailing_update<T, 4>(S, LD, j0, r0, tx, ty);
      else if (R == 32) trailing_update<T, 2>(S, LD, j0, r0, tx, ty);
    }
    __syncthreads();
  }

  // diagonal-block inverses: warp p, lane c: x_i = (delta_ic - sum_{k<i} L_ik x_k) / L_ii
  if (warp < Cfg::NP) {
    const T* Lp = Lal + warp * 32 * LA;
    T x[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      T s = i == lane ? T(1) : T(0);
#pragma unroll
      for (int g = 0; g < (i + E - 1) / E; ++g) {
        const V v = reinterpret_cast<const V*>(Lp + i * LA)[g];
        const T* ve = reinterpret_cast<const T*>(&v);
#pragma unroll
        for (int e = 0; e < E; ++e)
          if (g * E + e < i) s = fma(-ve[e], x[g * E + e], s);
      }
      x[i] = s * rdiag[32 * warp + i];
    }
#pragma unroll
    for (int i = 0; i < 32; ++i) X[(32 * warp + i) * LD + 32 * warp + lane] = x[i];
  }
  __syncthreads();
  if constexpr (NB >= 64) inverse_level<T, NB, 32>(S, X, Tm, tid);
  if constexpr (NB >= 128) inverse_level<T, NB, 64>(S, X, Tm, tid);

  if (vec) {
#pragma unroll 4
    for (int it = 0; it < UNITS / 8; ++it) {
      const int u = it * 8 + warp, i = (u / CH) * 4 + lane / 8, j = ((u % CH) * 8 + lane % 8) * E;
      V lv, xv;
      T* le = reinterpret_cast<T*>(&lv);
      T* xe = reinterpret_cast<T*>(&xv);
#pragma unroll
      for (int e = 0; e < E; ++e) {
        le[e] = S[i * LD + j + e];
        xe[e] = j + e <= i ? X[i * LD + j + e] : T(0);
      }
      *reinterpret_cast<V*>(dinv + (int64_t)i * ldd + j) = xv;
      if (j + E - 1 <= i) {
        *reinterpret_cast<V*>(A + (int64_t)i * lda + j) = lv;
      } else {
#pragma unroll
        for (int e = 0; e < E; ++e)
          if (j + e <= i) A[(int64_t)i * lda + j + e] = le[e];
      }
    }
  } else {
    for (int i = tid / 32; i < n; i += nt / 32) {
      for (int j = tid % 32; j < n; j += 32) {
        if (j <= i) A[(int64_t)i * lda + j] = S[i * LD + j];
        dinv[(int64_t)i * ldd + j] = j <= i ? X[i * LD + j] : T(0);
      }
    }
  }
}

template <typename T, int NB>
static kf_status launch_potrf_diag(cudaStream_t s, T* A, int64_t lda, int n, T* dinv, int64_t ldd, int* status,
                                   int step, int base) {
  const size_t smem = DiagSmem<T, NB>::bytes;
  KF_CUDA_TRY(smem_limit_per_device((const void*)potrf_diag_kernel<T, NB>, (int)smem));
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
  if (nb != potrf_block<T>() && nb != 32) return KF_ERR_ARG;  // 32: small matrices (more, cheaper leaves)
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
