// Bandwidth-bound helper kernels: copies/conversions, covariance additions,
// matrix-vector products for the means (eqns 6, 10, 12), the innovation and
// its covariance S = H P H^T + R (eqn 8), the bf16 hi/lo split, diagonals.
#include "ops.cuh"

namespace kfm {

__device__ __forceinline__ double cov_value(int kind, const double* q, int64_t n, int64_t i, int64_t j) {
  if (kind == 0) return i == j ? q[0] : 0.0;
  if (kind == 1) return i == j ? q[i] : 0.0;
  if (kind == 2) return q[i * n + j];
  return 0.0;
}

// Row-major elementwise kernels move 4 consecutive elements of a row per
// unit with 16-byte accesses where the rows allow it, and each thread keeps
// kUnroll units in flight (the covariance copies and updates are N x N sweeps
// bound by HBM bandwidth).
constexpr int kUnroll = 4;

template <typename T>
__device__ __forceinline__ bool aligned_rows(const T* p, int64_t ld) {
  return (reinterpret_cast<uintptr_t>(p) & 15) == 0 && (ld * (int64_t)sizeof(T)) % 16 == 0;
}

template <typename T>
__device__ __forceinline__ void load4(const T* p, bool vec, int64_t valid, T (&v)[4]) {
  if (vec && valid >= 4) {
    if constexpr (sizeof(T) == 4) {
      const float4 f = *reinterpret_cast<const float4*>(p);
      v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
    } else {
      const double2 a = *reinterpret_cast<const double2*>(p);
      const double2 b = *reinterpret_cast<const double2*>(p + 2);
      v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
  } else {
#pragma unroll
    for (int e = 0; e < 4; ++e) v[e] = e < valid ? p[e] : T(0);
  }
}

template <typename T>
__device__ __forceinline__ void store4(T* p, bool vec, int64_t valid, const T (&v)[4]) {
  if (vec && valid >= 4) {
    if constexpr (sizeof(T) == 4) {
      *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
      *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
      *reinterpret_cast<double2*>(p + 2) = make_double2(v[2], v[3]);
    }
  } else {
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (e < valid) p[e] = v[e];
  }
}

inline unsigned sweep_blocks(int64_t units) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(units, 256 * kUnroll), 152 * 16));
}

template <typename Tdst, typename Tsrc>
__global__ void __launch_bounds__(256) copy2d_kernel(Tdst* dst, int64_t ldd, const Tsrc* src, int64_t lds,
                                                     int64_t rows, int64_t cols, int64_t pad_to) {
  const bool vs = aligned_rows(src, lds), vd = aligned_rows(dst, ldd);
  const int64_t cpr = (pad_to + 3) / 4, units = rows * cpr;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t u0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u0 < units; u0 += stride * kUnroll) {
    Tsrc v[kUnroll][4];
#pragma unroll
    for (int k = 0; k < kUnroll; ++k) {
      const int64_t u = u0 + k * stride;
      if (u < units) {
        const int64_t i = u / cpr, j = (u % cpr) * 4;
        load4<Tsrc>(src + i * lds + j, vs, cols - j, v[k]);  // zero beyond cols
      }
    }
#pragma unroll
    for (int k = 0; k < kUnroll; ++k) {
      const int64_t u = u0 + k * stride;
      if (u < units) {
        const int64_t i = u / cpr, j = (u % cpr) * 4;
        Tdst w[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) w[e] = (Tdst)v[k][e];
        store4<Tdst>(dst + i * ldd + j, vd, pad_to - j, w);
      }
    }
  }
}

template <typename Tdst, typename Tsrc>
kf_status copy2d(cudaStream_t s, Tdst* dst, int64_t ldd, const Tsrc* src, int64_t lds, int64_t rows,
                 int64_t cols, bool zero_pad) {
  if (rows <= 0 || cols <= 0) return KF_OK;
  const int64_t pad_to = zero_pad ? ldd : cols;
  copy2d_kernel<Tdst, Tsrc><<<sweep_blocks(rows * ((pad_to + 3) / 4)), 256, 0, s>>>(dst, ldd, src, lds, rows, cols,
                                                                                     pad_to);
  note_launch();
  return launch_check("copy2d");
}

template <typename Tdst, typename Tsrc>
__global__ void __launch_bounds__(256) add_cov_kernel(Tdst* dst, int64_t ldd, const Tsrc* src, int64_t lds,
                                                      int64_t n, int kind, const double* q) {
  const bool vs = aligned_rows(src, lds), vd = aligned_rows(dst, ldd);
  const int64_t cpr = (n + 3) / 4, units = n * cpr;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t u0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u0 < units; u0 += stride * kUnroll) {
    Tsrc v[kUnroll][4];
#pragma unroll
    for (int k = 0; k < kUnroll; ++k) {
      const int64_t u = u0 + k * stride;
      if (u < units) {
        const int64_t i = u / cpr, j = (u % cpr) * 4;
        load4<Tsrc>(src + i * lds + j, vs, n - j, v[k]);
      }
    }
#pragma unroll
    for (int k = 0; k < kUnroll; ++k) {
      const int64_t u = u0 + k * stride;
      if (u < units) {
        const int64_t i = u / cpr, j = (u % cpr) * 4;
        Tdst w[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) w[e] = (Tdst)((double)v[k][e] + cov_value(kind, q, n, i, j + e));
        store4<Tdst>(dst + i * ldd + j, vd, n - j, w);
      }
    }
  }
}

template <typename Tdst, typename Tsrc>
__global__ void add_diag_kernel(Tdst* dst, int64_t ldd, const Tsrc* src, int64_t lds, int64_t n, int kind,
                                const double* q) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i * ldd + i] = (Tdst)((double)src[i * lds + i] + (kind == 0 ? q[0] : q[i]));
}

template <typename Tdst, typename Tsrc>
kf_status add_cov(cudaStream_t s, Tdst* dst, int64_t ldd, const Tsrc* src, int64_t lds, int64_t n,
                  int q_kind, const double* q) {
  if (n <= 0) return KF_OK;
  if (q_kind == 2 || q_kind < 0) {  // dense Q (or none): every element through float64
    add_cov_kernel<Tdst, Tsrc><<<sweep_blocks(n * ((n + 3) / 4)), 256, 0, s>>>(dst, ldd, src, lds, n, q_kind, q);
    note_launch();
    return launch_check("add_cov");
  }
  // scalar or diagonal Q: a plain copy, then the n diagonal sums (kept apart so that the
  // float64 arithmetic is spent on the diagonal only)
  if (!((const void*)dst == (const void*)src && ldd == lds && sizeof(Tdst) == sizeof(Tsrc)))
    KF_TRY((copy2d<Tdst, Tsrc>(s, dst, ldd, src, lds, n, n)));
  add_diag_kernel<Tdst, Tsrc><<<(unsigned)std::min<int64_t>(ceil_div(n, 256), 1024), 256, 0, s>>>(dst, ldd, src, lds,
                                                                                                 n, q_kind, q);
  note_launch();
  return launch_check("add_diag");
}

// One warp per row; each lane reads 4 consecutive elements per step (16-byte
// loads for aligned rows).  float64 matrices accumulate in float64.  For a
// float32 matrix (the mixed path's J_t and Z) the products and each lane's
// running sum are float32 against a float32 copy of x held in shared memory
// (float64 arithmetic is a small fraction of the float32 rate here), and the
// 32 lane sums are combined in float64.
constexpr int kGemvSmemX = 12288;

template <typename T, bool F64ACC>
__global__ void __launch_bounds__(256) gemv_kernel(int64_t rows, int64_t cols, const T* A, int64_t lda,
                                                   const double* x, const double* ybase, double sign, double* y) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const bool vec = aligned_rows(A, lda);
  if constexpr (sizeof(T) == 4 && !F64ACC) {
    __shared__ float xs[kGemvSmemX];
    if (cols <= kGemvSmemX) {
      for (int64_t j = threadIdx.x; j < cols; j += blockDim.x) xs[j] = (float)x[j];
      __syncthreads();
      for (int64_t i = warp; i < rows; i += nwarps) {
        const T* row = A + i * lda;
        float accf = 0.0f;
#pragma unroll 4
        for (int64_t j = 4 * lane; j < cols; j += 128) {
          T a[4];
          load4<T>(row + j, vec, cols - j, a);
#pragma unroll
          for (int e = 0; e < 4; ++e)
            if (j + e < cols) accf = fmaf(a[e], xs[j + e], accf);
        }
        double acc = accf;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) y[i] = ybase ? ybase[i] + sign * acc : acc;
      }
      return;
    }
  }
  for (int64_t i = warp; i < rows; i += nwarps) {
    const T* row = A + i * lda;
    double acc = 0.0;
    for (int64_t j = 4 * lane; j < cols; j += 128) {
      T a[4];
      load4<T>(row + j, vec, cols - j, a);
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (j + e < cols) acc = fma((double)a[e], x[j + e], acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) y[i] = ybase ? ybase[i] + sign * acc : acc;
  }
}

template <typename T>
kf_status gemv(cudaStream_t s, int64_t rows, int64_t cols, const T* A, int64_t lda, const double* x,
               const double* ybase, double sign, double* y) {
  if (rows <= 0) return KF_OK;
  // float32 rows: 16 rows per block (x is converted once per block)
  const int64_t per_block_rows = sizeof(T) == 4 ? 16 : 8;
  unsigned blocks = (unsigned)std::min<int64_t>(ceil_div(rows, per_block_rows), 4096);
  gemv_kernel<T, false><<<blocks, 256, 0, s>>>(rows, cols, A, lda, x, ybase, sign, y);
  note_launch();
  return launch_check("gemv");
}

kf_status gemv_f64acc(cudaStream_t s, int64_t rows, int64_t cols, const float* A, int64_t lda, const double* x,
                      const double* ybase, double sign, double* y) {
  if (rows <= 0) return KF_OK;
  unsigned blocks = (unsigned)std::min<int64_t>(ceil_div(rows, 8), 4096);
  gemv_kernel<float, true><<<blocks, 256, 0, s>>>(rows, cols, A, lda, x, ybase, sign, y);
  note_launch();
  return launch_check("gemv_f64acc");
}

// y = ybase + sign A^T x: one thread per column, consecutive threads read consecutive columns.
__global__ void gemv_t_kernel(int64_t rows, int64_t cols, const double* A, int64_t lda, const double* x,
                              const double* ybase, double sign, double* y) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < cols; j += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int64_t i = 0; i < rows; ++i) acc = fma(A[i * lda + j], x[i], acc);
    y[j] = ybase ? ybase[j] + sign * acc : acc;
  }
}

kf_status gemv_t(cudaStream_t s, int64_t rows, int64_t cols, const double* A, int64_t lda, const double* x,
                 const double* ybase, double sign, double* y) {
  if (cols <= 0) return KF_OK;
  gemv_t_kernel<<<(unsigned)std::min<int64_t>(ceil_div(cols, 128), 1024), 128, 0, s>>>(rows, cols, A, lda, x, ybase,
                                                                                   sign, y);
  note_launch();
  return launch_check("gemv_t");
}

// J = I - Q X for Q = q I (q_kind 0) or diagonal (1): row i scaled by q_i.
__global__ void identity_minus_q_kernel(int64_t n, const float* X, int64_t ldx, int q_kind, const double* q, float* J,
                                        int64_t ldj) {
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n * n; u += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = u / n, j = u % n;
    const float qi = (float)(q_kind == 0 ? q[0] : q[i]);
    J[i * ldj + j] = (i == j ? 1.0f : 0.0f) - qi * X[i * ldx + j];
  }
}

kf_status identity_minus_q(cudaStream_t s, int64_t n, const float* X, int64_t ldx, int q_kind, const double* q,
                           float* J, int64_t ldj) {
  if (q_kind != 0 && q_kind != 1) return KF_ERR_ARG;
  identity_minus_q_kernel<<<(unsigned)std::min<int64_t>(ceil_div(n * n, 256), 152 * 16), 256, 0, s>>>(n, X, ldx,
                                                                                                  q_kind, q, J, ldj);
  note_launch();
  return launch_check("identity_minus_q");
}

// out = a + d - Q y (Q per q_kind: scalar or diagonal).
__global__ void mean_update_q_kernel(int64_t n, const double* a, const double* d, int q_kind, const double* q,
                                     const double* yv, double* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = a[i] + (d[i] - (q_kind == 0 ? q[0] : q[i]) * yv[i]);
}

kf_status mean_update_q(cudaStream_t s, int64_t n, const double* a, const double* d, int q_kind, const double* q,
                        const double* yv, double* out) {
  if (q_kind != 0 && q_kind != 1) return KF_ERR_ARG;
  mean_update_q_kernel<<<(unsigned)std::min<int64_t>(ceil_div(n, 256), 1024), 256, 0, s>>>(n, a, d, q_kind, q, yv,
                                                                                          out);
  note_launch();
  return launch_check("mean_update_q");
}

__global__ void set_step_kernel(int* status, int step) { status[ST_CUR] = step; }

kf_status set_status_step(cudaStream_t s, int* status, int step) {
  set_step_kernel<<<1, 1, 0, s>>>(status, step);
  note_launch();
  return launch_check("set_step");
}

__global__ void vsub_kernel(int64_t n, const double* a, const double* b, double* d) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    d[i] = a[i] - b[i];
}

kf_status vsub(cudaStream_t s, int64_t n, const double* a, const double* b, double* d) {
  if (n <= 0) return KF_OK;
  vsub_kernel<<<(unsigned)std::min<int64_t>(ceil_div(n, 256), 1024), 256, 0, s>>>(n, a, b, d);
  note_launch();
  return launch_check("vsub");
}

__global__ void innovation_kernel(int64_t m, int64_t N, const double* H, const double* x, const double* y,
                                  double* nu, int* status, int step) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < m; i += nwarps) {
    double acc = 0.0;
    for (int64_t j = lane; j < N; j += 32) acc = fma(H[i * N + j], x[j], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      double v = y[i] - acc;
      nu[i] = v;
      if (!isfinite(v)) status_set(status, KF_ERR_NUMERIC, step, (int)i);
    }
  }
}

kf_status innovation(cudaStream_t s, int64_t m, int64_t N, const double* H, const double* x,
                     const double* y, double* nu, int* status, int step) {
  unsigned blocks = (unsigned)std::min<int64_t>(ceil_div(m * 32, 256), 1024);
  innovation_kernel<<<blocks, 256, 0, s>>>(m, N, H, x, y, nu, status, step);
  note_launch();
  return launch_check("innovation");
}

// partials[split][i][j] = sum_{k in chunk} H[i,k] Ut[k,j]; 32 x 32 output tile per CTA.
// float32 operands are multiplied in float32 over 32-long runs and summed in float64.
template <typename T, typename TH>
__global__ void __launch_bounds__(256) innov_cov_partial_kernel(int m, int N, const TH* H, int64_t ldh,
                                                                const T* Ut, int64_t ldu, double* partials,
                                                                int chunk) {
  __shared__ T Hs[32][33];
  __shared__ T Us[32][33];
  const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  const int split = blockIdx.z;
  const int k_begin = split * chunk;
  const int k_end = min(N, k_begin + chunk);
  const int tid = threadIdx.x;
  const int tx = tid % 32, ty = tid / 32;  // ty: 0..7, each thread 4 rows (ty + 8 r)
  double acc[4] = {0, 0, 0, 0};
  for (int k0 = k_begin; k0 < k_end; k0 += 32) {
    for (int l = tid; l < 32 * 32; l += 256) {
      int r = l / 32, c = l % 32;
      int gi = i0 + r, gk = k0 + c;
      Hs[r][c] = (gi < m && gk < k_end) ? (T)H[(int64_t)gi * ldh + gk] : T(0);
      int gk2 = k0 + r, gj = j0 + c;
      Us[r][c] = (gk2 < k_end && gj < m) ? Ut[(int64_t)gk2 * ldu + gj] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      T a = T(0);
#pragma unroll 8
      for (int kk = 0; kk < 32; ++kk) a = fma(Hs[ty + 8 * r][kk], Us[kk][tx], a);
      acc[r] += (double)a;
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    int gi = i0 + ty + 8 * r, gj = j0 + tx;
    if (gi < m && gj < m) partials[((int64_t)split * m + gi) * m + gj] = acc[r];
  }
}

// S = sym(sum_split partials) + R
__global__ void innov_cov_reduce_kernel(int m, const double* partials, int splits, int r_kind,
                                        const double* R, double* S, int64_t lds) {
  int64_t total = (int64_t)m * m;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(idx / m), j = (int)(idx % m);
    if (j > i) continue;
    double a = 0.0, b = 0.0;
    for (int sp = 0; sp < splits; ++sp) {
      a += partials[((int64_t)sp * m + i) * m + j];
      b += partials[((int64_t)sp * m + j) * m + i];
    }
    double v = 0.5 * (a + b) + cov_value(r_kind, R, m, i, j);
    S[(int64_t)i * lds + j] = v;
    S[(int64_t)j * lds + i] = v;
  }
}

template <typename T, typename TH>
kf_status innovation_cov(cudaStream_t s, int m, int N, const TH* H, int64_t ldh, const T* Ut,
                         int64_t ldu, int r_kind, const double* R, double* S, int64_t lds,
                         double* partials, int splits) {
  int chunk = (int)round_up(ceil_div(N, splits), 32);
  int used = (int)ceil_div(N, chunk);
  dim3 grid((unsigned)ceil_div(m, 32), (unsigned)ceil_div(m, 32), (unsigned)used);
  innov_cov_partial_kernel<T, TH><<<grid, 256, 0, s>>>(m, N, H, ldh, Ut, ldu, partials, chunk);
  note_launch();
  KF_TRY(launch_check("innov_cov_partial"));
  unsigned blocks = (unsigned)std::min<int64_t>(ceil_div((int64_t)m * m, 256), 1024);
  innov_cov_reduce_kernel<<<blocks, 256, 0, s>>>(m, partials, used, r_kind, R, S, lds);
  note_launch();
  return launch_check("innov_cov_reduce");
}

__global__ void spmv_kernel(int64_t N, const int64_t* rowptr, const int64_t* col, const double* val,
                            const double* x, double* y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) acc = fma(val[k], x[col[k]], acc);
    y[i] = acc;
  }
}

kf_status predict_mean(cudaStream_t s, int f_kind, int64_t N, const double* F, const int64_t* rowptr,
                       const int64_t* col, const double* x, double* x_out) {
  if (f_kind == KF_F_IDENTITY) {
    KF_CUDA_TRY(cudaMemcpyAsync(x_out, x, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    return KF_OK;
  }
  if (f_kind == KF_F_CSR) {
    spmv_kernel<<<(unsigned)std::min<int64_t>(ceil_div(N, 256), 1024), 256, 0, s>>>(N, rowptr, col, F, x, x_out);
    note_launch();
    return launch_check("spmv");
  }
  return gemv<double>(s, N, N, F, N, x, nullptr, 1.0, x_out);
}

struct Planes3 {
  __nv_bfloat16* p[3];
};

__global__ void split_bf16_kernel(int64_t rows, int64_t cols, const float* A, int64_t lda, Planes3 pl, int n,
                                  int64_t ldh) {
  for (int64_t i = blockIdx.y; i < rows; i += gridDim.y)
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < ldh; j += (int64_t)gridDim.x * blockDim.x) {
      float r = j < cols ? A[i * lda + j] : 0.0f;
      for (int k = 0; k < n; ++k) {
        __nv_bfloat16 h = __float2bfloat16_rn(r);
        pl.p[k][i * ldh + j] = h;
        r -= __bfloat162float(h);  // exact: r and h agree in their leading bits
      }
    }
}

kf_status split_bf16(cudaStream_t s, int64_t rows, int64_t cols, const float* A, int64_t lda,
                     __nv_bfloat16* const* planes, int n, int64_t ldh) {
  if (rows <= 0) return KF_OK;
  if (n < 1 || n > 3) return KF_ERR_ARG;
  Planes3 pl{{planes[0], n > 1 ? planes[1] : nullptr, n > 2 ? planes[2] : nullptr}};
  dim3 grid((unsigned)std::min<int64_t>(ceil_div(ldh, 256), 64), (unsigned)std::min<int64_t>(rows, 65535));
  split_bf16_kernel<<<grid, 256, 0, s>>>(rows, cols, A, lda, pl, n, ldh);
  note_launch();
  return launch_check("split_bf16");
}

// Transposed split through a 32 x 32 shared-memory tile: reads rows of A
// (coalesced) and writes rows of the planes (coalesced).
__global__ void split_bf16_t_kernel(int64_t rows, int64_t cols, const float* A, int64_t lda, Planes3 pl, int n,
                                    int64_t ldh) {
  __shared__ float tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.x * 32, k0 = (int64_t)blockIdx.y * 32;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;  // 32 x 8 threads
  for (int i = ty; i < 32; i += 8) {
    const int64_t k = k0 + i, r = r0 + tx;
    tile[i][tx] = (k < cols && r < rows) ? A[k * lda + r] : 0.0f;
  }
  __syncthreads();
  for (int i = ty; i < 32; i += 8) {
    const int64_t r = r0 + i, k = k0 + tx;
    if (r >= rows || k >= ldh) continue;
    float v = tile[tx][i];
    for (int s = 0; s < n; ++s) {
      __nv_bfloat16 h = __float2bfloat16_rn(v);
      pl.p[s][r * ldh + k] = h;
      v -= __bfloat162float(h);
    }
  }
}

kf_status split_bf16_t(cudaStream_t s, int64_t rows, int64_t cols, const float* A, int64_t lda,
                       __nv_bfloat16* const* planes, int n, int64_t ldh) {
  if (rows <= 0) return KF_OK;
  if (n < 1 || n > 3 || ceil_div(rows, 32) > 0x7fffffff || ceil_div(ldh, 32) > 65535) return KF_ERR_ARG;
  Planes3 pl{{planes[0], n > 1 ? planes[1] : nullptr, n > 2 ? planes[2] : nullptr}};
  dim3 grid((unsigned)ceil_div(rows, 32), (unsigned)ceil_div(ldh, 32));
  split_bf16_t_kernel<<<grid, 256, 0, s>>>(rows, cols, A, lda, pl, n, ldh);
  note_launch();
  return launch_check("split_bf16_t");
}

__device__ __forceinline__ int64_t ceil_div_d(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Operand split for the split-bf16 products: plane s of row r holds slice s
// of op(X)[r][k] for k < ldh (zero for k >= cols).  The first slice of a
// float64 source is rounded from float64 (so the next slices keep bits below
// float32's), the rest in float32 arithmetic, which is exact for these
// residuals.  Stores are 16 bytes (8 values) per plane.
__device__ __forceinline__ uint4 pack8(const __nv_bfloat16 (&h)[8]) {
  uint32_t w[4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
    w[i] = (uint32_t)__bfloat16_as_ushort(h[2 * i]) | ((uint32_t)__bfloat16_as_ushort(h[2 * i + 1]) << 16);
  return make_uint4(w[0], w[1], w[2], w[3]);
}

template <typename S>
__device__ __forceinline__ void split8(const S (&v)[8], __nv_bfloat16* p0, __nv_bfloat16* p1, __nv_bfloat16* p2,
                                       int n, int64_t off) {
  float rest[8];
  __nv_bfloat16 h[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    if constexpr (sizeof(S) == 8) {
      h[e] = __double2bfloat16(v[e]);
      rest[e] = (float)(v[e] - (double)__bfloat162float(h[e]));
    } else {
      h[e] = __float2bfloat16_rn(v[e]);
      rest[e] = v[e] - __bfloat162float(h[e]);
    }
  }
  *reinterpret_cast<uint4*>(p0 + off) = pack8(h);
  for (int s = 1; s < n; ++s) {
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      h[e] = __float2bfloat16_rn(rest[e]);
      rest[e] -= __bfloat162float(h[e]);
    }
    *reinterpret_cast<uint4*>((s == 1 ? p1 : p2) + off) = pack8(h);
  }
}

// Untransposed source (op(X) = X, rows x cols, row stride ld): one thread per
// 8 consecutive values of a row, 16-byte loads where the row allows.
template <typename S>
__device__ __forceinline__ void split_rows(const SplitOp& op, int n, int64_t ldh) {
  const S* src = static_cast<const S*>(op.src);
  constexpr int VE = 16 / sizeof(S);
  const bool vec = (reinterpret_cast<uintptr_t>(src) & 15) == 0 && op.ld % VE == 0;
  const int64_t per_row = ldh / 8, units = op.rows * per_row;
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < units; u += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = u / per_row, k = (u % per_row) * 8;
    const S* row = src + r * op.ld;
    S v[8];
    if (vec && k + 8 <= op.cols) {
#pragma unroll
      for (int e = 0; e < 8; e += VE) {
        if constexpr (sizeof(S) == 8) {
          const double2 d = *reinterpret_cast<const double2*>(row + k + e);
          v[e] = d.x;
          v[e + 1] = d.y;
        } else {
          const float4 f = *reinterpret_cast<const float4*>(row + k + e);
          v[e] = f.x;
          v[e + 1] = f.y;
          v[e + 2] = f.z;
          v[e + 3] = f.w;
        }
      }
    } else {
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] = k + e < op.cols ? row[k + e] : S(0);
    }
    split8<S>(v, op.planes[0], op.planes[1], op.planes[2], n, r * ldh + k);
  }
}

// Transposed source (stored cols x rows, op(X)[r][k] = X[k][r]): 64 x 64 tiles
// through shared memory, read along source rows, written 8 values per store.
template <typename S>
__device__ __forceinline__ void split_cols(const SplitOp& op, int n, int64_t ldh, S (*tile)[65]) {
  const S* src = static_cast<const S*>(op.src);
  const int64_t tr = ceil_div_d(op.rows, 64), tk = ldh / 64, tiles = tr * tk;
  const int t = threadIdx.x;
  for (int64_t b = blockIdx.x; b < tiles; b += gridDim.x) {
    const int64_t r0 = (b % tr) * 64, k0 = (b / tr) * 64;
    __syncthreads();  // the previous tile's reads are done
    for (int i = t / 64; i < 64; i += 4) {  // tile[i][c] = X[k0 + i][r0 + c]
      const int c = t % 64;
      const int64_t k = k0 + i, r = r0 + c;
      tile[i][c] = (k < op.cols && r < op.rows) ? src[k * op.ld + r] : S(0);
    }
    __syncthreads();
    for (int w = t; w < 64 * 8; w += 256) {
      const int c = w / 8, kc = (w % 8) * 8;
      const int64_t r = r0 + c;
      if (r >= op.rows) continue;
      S v[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] = tile[kc + e][c];
      split8<S>(v, op.planes[0], op.planes[1], op.planes[2], n, r * ldh + k0 + kc);
    }
  }
}

__global__ void __launch_bounds__(256) split_bf16_pair_kernel(SplitOp a, SplitOp b, int n, int64_t ldh) {
  __shared__ double tile_d[64][65];
  const SplitOp op = blockIdx.y == 0 ? a : b;
  if (op.rows <= 0) return;
  if (op.trans) {
    if (op.f64)
      split_cols<double>(op, n, ldh, tile_d);
    else
      split_cols<float>(op, n, ldh, reinterpret_cast<float(*)[65]>(tile_d));
  } else {
    if (op.f64)
      split_rows<double>(op, n, ldh);
    else
      split_rows<float>(op, n, ldh);
  }
}

kf_status split_bf16_pair(cudaStream_t s, const SplitOp& a, const SplitOp& b, int n, int64_t ldh) {
  if (n < 1 || n > 3 || ldh % 64) return KF_ERR_ARG;
  const int64_t rows = std::max(a.rows, b.rows);
  if (rows <= 0) return KF_OK;
  // enough CTAs to fill the GPU for the large operands, fewer for small ones
  const int64_t work = std::max(ceil_div(a.rows, 64) * (ldh / 64), ceil_div(b.rows, 64) * (ldh / 64));
  const dim3 grid((unsigned)std::min<int64_t>(std::max<int64_t>(work, 1), 152 * 8), 2);
  split_bf16_pair_kernel<<<grid, 256, 0, s>>>(a, b, n, ldh);
  note_launch();
  return launch_check("split_bf16_pair");
}

__global__ void eye_kernel(int64_t n, double* d, int64_t ld) {
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n * n; u += (int64_t)gridDim.x * blockDim.x)
    d[(u / n) * ld + u % n] = (u / n == u % n) ? 1.0 : 0.0;
}

kf_status eye(cudaStream_t s, int64_t n, double* dst, int64_t ld) {
  if (n <= 0) return KF_OK;
  eye_kernel<<<(unsigned)std::min<int64_t>(ceil_div(n * n, 256), 4096), 256, 0, s>>>(n, dst, ld);
  note_launch();
  return launch_check("eye");
}

__global__ void transpose_kernel(int64_t rows, int64_t cols, const double* src, int64_t lds, double* dst,
                                 int64_t ldd) {
  __shared__ double tile[32][33];
  const int64_t r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t r = r0 + i, c = c0 + threadIdx.x;
    tile[i][threadIdx.x] = (r < rows && c < cols) ? src[r * lds + c] : 0.0;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t c = c0 + i, r = r0 + threadIdx.x;
    if (c < cols && r < rows) dst[c * ldd + r] = tile[threadIdx.x][i];
  }
}

kf_status transpose(cudaStream_t s, int64_t rows, int64_t cols, const double* src, int64_t lds, double* dst,
                    int64_t ldd) {
  if (rows <= 0 || cols <= 0) return KF_OK;
  transpose_kernel<<<dim3((unsigned)ceil_div(cols, 32), (unsigned)ceil_div(rows, 32)), dim3(32, 8), 0, s>>>(
      rows, cols, src, lds, dst, ldd);
  note_launch();
  return launch_check("transpose");
}

template <typename T>
__global__ void diag_kernel(int64_t n, const T* A, int64_t lda, double* d) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    d[i] = (double)A[i * lda + i];
}

template <typename T>
kf_status diag_extract(cudaStream_t s, int64_t n, const T* A, int64_t lda, double* diag_out) {
  if (n <= 0) return KF_OK;
  diag_kernel<T><<<(unsigned)std::min<int64_t>(ceil_div(n, 256), 1024), 256, 0, s>>>(n, A, lda, diag_out);
  note_launch();
  return launch_check("diag");
}

#define KFM_INST2(D, S)                                                                             \
  template kf_status copy2d<D, S>(cudaStream_t, D*, int64_t, const S*, int64_t, int64_t, int64_t, bool); \
  template kf_status add_cov<D, S>(cudaStream_t, D*, int64_t, const S*, int64_t, int64_t, int, const double*);
KFM_INST2(double, double)
KFM_INST2(float, float)
KFM_INST2(double, float)
KFM_INST2(float, double)
#undef KFM_INST2

template kf_status gemv<double>(cudaStream_t, int64_t, int64_t, const double*, int64_t, const double*,
                                const double*, double, double*);
template kf_status gemv<float>(cudaStream_t, int64_t, int64_t, const float*, int64_t, const double*,
                               const double*, double, double*);
template kf_status innovation_cov<double, double>(cudaStream_t, int, int, const double*, int64_t, const double*,
                                                  int64_t, int, const double*, double*, int64_t, double*, int);
template kf_status innovation_cov<float, double>(cudaStream_t, int, int, const double*, int64_t, const float*,
                                                 int64_t, int, const double*, double*, int64_t, double*, int);
template kf_status innovation_cov<float, float>(cudaStream_t, int, int, const float*, int64_t, const float*,
                                                int64_t, int, const double*, double*, int64_t, double*, int);
template kf_status diag_extract<double>(cudaStream_t, int64_t, const double*, int64_t, double*);
template kf_status diag_extract<float>(cudaStream_t, int64_t, const float*, int64_t, double*);

}  // namespace kfm
