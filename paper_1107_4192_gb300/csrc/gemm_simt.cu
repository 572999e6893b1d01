// CUDA-core (FMA) tiled GEMM for float64 and float32 with the fused
// covariance epilogue of ops.cuh.  Used for every float64 product of the
// plain path, the float32 path, and the blocked Cholesky / triangular solves.
#include <utility>

#include "epilogue.cuh"

namespace kfm {

std::atomic<int64_t> g_launches{0};
thread_local int64_t t_launches = 0;

template <typename T> struct SimtCfg;
// float64: 64 x 64 tiles, 4 x 4 outputs per thread (the FP64 pipe is the limit).
template <> struct SimtCfg<double> {
  static constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4, PAD = 2;
};
// float32: 128 x 128 tiles, 8 x 8 outputs per thread.
template <> struct SimtCfg<float> {
  static constexpr int BM = 128, BN = 128, BK = 8, TM = 8, TN = 8, PAD = 4;
};
// float64 products too small to fill the GPU with 64 x 64 tiles (the m x m
// innovation factorisation, its panels): the float64 pipe does about two
// multiply-adds per clock per SM, so such a product is bound by how many SMs
// it reaches.  16 x 16 tiles, one output per thread, same summation order.
struct SimtCfgSmall64 {
  static constexpr int BM = 16, BN = 16, BK = 16, TM = 1, TN = 1, PAD = 1;
};

// Maps a linear block index onto the lower-triangular tile (tm >= tn).
__device__ __forceinline__ void tri_tile(int b, int& tm, int& tn) {
  int r = (int)((sqrtf(8.0f * (float)b + 1.0f) - 1.0f) * 0.5f);
  while ((r + 1) * (r + 2) / 2 <= b) ++r;
  while (r * (r + 1) / 2 > b) --r;
  tm = r;
  tn = b - r * (r + 1) / 2;
}

template <typename T, bool TB, typename C = SimtCfg<T>>
__global__ void __launch_bounds__(256) gemm_simt_kernel(GemmParams<T> p) {
  constexpr int BM = C::BM, BN = C::BN, BK = C::BK, TM = C::TM, TN = C::TN;
  constexpr int LDA_S = BM + C::PAD, LDB_S = BN + C::PAD;
  __shared__ __align__(16) T As[BK * LDA_S];
  __shared__ __align__(16) T Bs[BK * LDB_S];

  int tm, tn;
  if (p.sym) {
    tri_tile(blockIdx.x, tm, tn);
  } else {
    tn = blockIdx.x;
    tm = blockIdx.y;
  }
  __shared__ int skip;
  if (threadIdx.x == 0) skip = status_failed(p.status) ? 1 : 0;  // one read for the whole CTA
  __syncthreads();
  if (skip) return;
  const int m0 = tm * BM, n0 = tn * BN;
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;

  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);

  for (int k0 = 0; k0 < p.K; k0 += BK) {
    // A tile: BM x BK, stored transposed As[kk][row]
#pragma unroll
    for (int l = 0; l < (BM * BK) / 256; ++l) {
      int idx = tid + l * 256;
      int row = idx / BK, kk = idx % BK;
      int gr = m0 + row, gk = k0 + kk;
      T v = T(0);
      if (gr < p.M && gk < p.K) v = p.A[(int64_t)gr * p.lda + gk];
      As[kk * LDA_S + row] = v;
    }
    if (TB) {
#pragma unroll
      for (int l = 0; l < (BN * BK) / 256; ++l) {
        int idx = tid + l * 256;
        int col = idx / BK, kk = idx % BK;
        int gc = n0 + col, gk = k0 + kk;
        T v = T(0);
        if (gc < p.N && gk < p.K) v = p.B[(int64_t)gc * p.ldb + gk];
        Bs[kk * LDB_S + col] = v;
      }
    } else {
#pragma unroll
      for (int l = 0; l < (BN * BK) / 256; ++l) {
        int idx = tid + l * 256;
        int kk = idx / BN, col = idx % BN;
        int gc = n0 + col, gk = k0 + kk;
        T v = T(0);
        if (gc < p.N && gk < p.K) v = p.B[(int64_t)gk * p.ldb + gc];
        Bs[kk * LDB_S + col] = v;
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk * LDA_S + ty * TM + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk * LDB_S + tx * TN + j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }

#pragma unroll
  for (int i = 0; i < TM; ++i) {
    int gi = m0 + ty * TM + i;
    if (gi >= p.M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      int gj = n0 + tx * TN + j;
      if (gj >= p.N) continue;
      if (p.sym && gj > gi) continue;
      epilogue_store(p, gi, gj, acc[i][j]);
    }
  }
}

template <typename T>
kf_status gemm_simt(cudaStream_t s, bool transB, const GemmParams<T>& p) {
  using C = SimtCfg<T>;
  if (p.M <= 0 || p.N <= 0) return KF_OK;
  if (p.K < 0) return KF_ERR_ARG;
  if constexpr (sizeof(T) == 4) {
    // aligned float32 operands take the pipelined kernel (same products, same order)
    if (gemm_small_ok(transB, p)) return gemm_small(s, transB, p);
  }
  if (p.sym && p.M != p.N) return KF_ERR_ARG;
  auto grid_for = [&](int bm, int bn) {
    if (p.sym) {
      const int64_t nt = ceil_div(p.M, bm);
      return dim3((unsigned)(nt * (nt + 1) / 2));
    }
    return dim3((unsigned)ceil_div(p.N, bn), (unsigned)ceil_div(p.M, bm));
  };
  dim3 grid = grid_for(C::BM, C::BN);
  if constexpr (sizeof(T) == 8) {
    // Callers run in-place row transforms (out == A) that rely on one column tile
    // owning all N <= 64 columns; the small tiles are used only when no output
    // element is also an operand element.
    // exact for two blocks of doubles with the same row stride (disjoint column or
    // row ranges of one matrix), a byte-range test otherwise
    auto apart = [](const void* a, size_t ea, int64_t la, int64_t ra, int64_t ca, const void* b, size_t eb,
                    int64_t lb, int64_t rb, int64_t cb) {
      if (!a || !b || ra <= 0 || ca <= 0 || rb <= 0 || cb <= 0) return true;
      const char* a0 = static_cast<const char*>(a);
      const char* b0 = static_cast<const char*>(b);
      const char* a1 = a0 + ((ra - 1) * la + ca) * (int64_t)ea;
      const char* b1 = b0 + ((rb - 1) * lb + cb) * (int64_t)eb;
      if (a1 <= b0 || b1 <= a0) return true;
      if (ea != eb || la != lb || la <= 0) return false;
      const int64_t d = (b0 - a0) / (int64_t)ea;
      if ((b0 - a0) % (int64_t)ea) return false;
      const int64_t dr = d >= 0 ? d / la : -((-d + la - 1) / la), dc = d - dr * la;
      if (dc + cb > la) return false;
      return !(dr < ra && dr + rb > 0 && dc < ca && dc + cb > 0);
    };
    const int64_t rB = transB ? p.N : p.K, cB = transB ? p.K : p.N;
    bool separate = true;
    const void* outs[3] = {p.out, p.out2, p.outf};
    const size_t es[3] = {sizeof(T), sizeof(T), sizeof(float)};
    const int64_t lds[3] = {p.ldo, p.ldo2, p.ldof};
    for (int k = 0; k < 3; ++k)
      if (outs[k] && (!apart(outs[k], es[k], lds[k], p.M, p.N, p.A, sizeof(T), p.lda, p.M, p.K) ||
                      !apart(outs[k], es[k], lds[k], p.M, p.N, p.B, sizeof(T), p.ldb, rB, cB)))
        separate = false;
    if (separate && (int64_t)grid.x * grid.y < 2 * 152) {
      const dim3 g2 = grid_for(SimtCfgSmall64::BM, SimtCfgSmall64::BN);
      if (g2.y <= 65535) {
        if (transB)
          gemm_simt_kernel<T, true, SimtCfgSmall64><<<g2, 256, 0, s>>>(p);
        else
          gemm_simt_kernel<T, false, SimtCfgSmall64><<<g2, 256, 0, s>>>(p);
        note_launch();
        return launch_check("gemm_simt");
      }
    }
  }
  if (grid.y > 65535) return KF_ERR_ARG;
  if (transB)
    gemm_simt_kernel<T, true><<<grid, 256, 0, s>>>(p);
  else
    gemm_simt_kernel<T, false><<<grid, 256, 0, s>>>(p);
  note_launch();
  return launch_check("gemm_simt");
}

template kf_status gemm_simt<double>(cudaStream_t, bool, const GemmParams<double>&);
template kf_status gemm_simt<float>(cudaStream_t, bool, const GemmParams<float>&);

}  // namespace kfm
