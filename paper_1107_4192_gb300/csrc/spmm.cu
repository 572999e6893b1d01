// Mesh-coupled prediction (eqn 2 generalised to eqn 3): F P F^T + Q with the
// sparse neighbourhood matrix F in compressed-row form (<= 7 entries per row
// for the six-neighbour mesh).  Both passes stream whole rows of an N x N
// matrix, so they are HBM-bound: W = F P combines rows of P, and
// out = W F^T gathers, for each output column j, the entries of one row of W
// at the column indices of row j of F.
#include "ops.cuh"

namespace kfm {

template <typename T>
__global__ void spmm_fp_kernel(int64_t N, const int64_t* rowptr, const int64_t* col, const double* val,
                               const T* P, int64_t ldp, T* W, int64_t ldw) {
  for (int64_t i = blockIdx.x; i < N; i += gridDim.x) {
    const int64_t k0 = rowptr[i], k1 = rowptr[i + 1];
    for (int64_t j = threadIdx.x; j < N; j += blockDim.x) {
      double acc = 0.0;
      for (int64_t k = k0; k < k1; ++k) acc = fma(val[k], (double)P[col[k] * ldp + j], acc);
      W[i * ldw + j] = (T)acc;
    }
  }
}

template <typename T>
__global__ void spmm_wft_kernel(int64_t N, const int64_t* rowptr, const int64_t* col, const double* val,
                                const T* W, int64_t ldw, T* out, int64_t ldo, int q_kind, const double* q) {
  for (int64_t i = blockIdx.x; i < N; i += gridDim.x) {
    const T* wrow = W + i * ldw;
    for (int64_t j = threadIdx.x; j < N; j += blockDim.x) {
      double acc = 0.0;
      for (int64_t k = rowptr[j]; k < rowptr[j + 1]; ++k) acc = fma(val[k], (double)__ldg(wrow + col[k]), acc);
      if (q_kind == 0 && i == j) acc += q[0];
      else if (q_kind == 1 && i == j) acc += q[i];
      else if (q_kind == 2) acc += q[i * N + j];
      out[i * ldo + j] = (T)acc;
    }
  }
}

template <typename T>
kf_status spmm_fpft(cudaStream_t s, int64_t N, const int64_t* rowptr, const int64_t* col, const double* val,
                    const T* P, int64_t ldp, T* W, int64_t ldw, T* out, int64_t ldo, int q_kind,
                    const double* q) {
  if (N <= 0) return KF_OK;
  unsigned blocks = (unsigned)std::min<int64_t>(N, 1 << 20);
  spmm_fp_kernel<T><<<blocks, 256, 0, s>>>(N, rowptr, col, val, P, ldp, W, ldw);
  note_launch();
  KF_TRY(launch_check("spmm_fp"));
  spmm_wft_kernel<T><<<blocks, 256, 0, s>>>(N, rowptr, col, val, W, ldw, out, ldo, q_kind, q);
  note_launch();
  return launch_check("spmm_wft");
}

template <typename T>
kf_status spmm_pft(cudaStream_t s, int64_t N, const int64_t* rowptr, const int64_t* col, const double* val,
                   const T* P, int64_t ldp, T* out, int64_t ldo) {
  if (N <= 0) return KF_OK;
  unsigned blocks = (unsigned)std::min<int64_t>(N, 1 << 20);
  spmm_wft_kernel<T><<<blocks, 256, 0, s>>>(N, rowptr, col, val, P, ldp, out, ldo, -1, nullptr);
  note_launch();
  return launch_check("spmm_pft");
}

template kf_status spmm_fpft<double>(cudaStream_t, int64_t, const int64_t*, const int64_t*, const double*,
                                     const double*, int64_t, double*, int64_t, double*, int64_t, int,
                                     const double*);
template kf_status spmm_fpft<float>(cudaStream_t, int64_t, const int64_t*, const int64_t*, const double*,
                                    const float*, int64_t, float*, int64_t, float*, int64_t, int,
                                    const double*);
template kf_status spmm_pft<double>(cudaStream_t, int64_t, const int64_t*, const int64_t*, const double*,
                                    const double*, int64_t, double*, int64_t);
template kf_status spmm_pft<float>(cudaStream_t, int64_t, const int64_t*, const int64_t*, const double*,
                                   const float*, int64_t, float*, int64_t);

}  // namespace kfm
