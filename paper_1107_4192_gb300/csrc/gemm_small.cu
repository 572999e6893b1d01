// Latency-oriented float32 product for the small and mid-size products of the
// recursive Cholesky / triangular inverse (smoother gain, eqn 11).
//
// At the bottom of the recursion the products are 128..1024 wide and strictly
// sequential, so their cost is latency, not throughput: a split-bf16 tensor-core
// product needs an operand-split launch plus a kernel whose fixed cost (TMEM
// allocation, pipeline fill, accumulator promotion) is larger than the work.
// This kernel reads the float32 operands directly with a four-stage cp.async
// pipeline (16-byte copies, zero fill outside the matrix), keeps 32 x 32 or
// 64 x 64 output tiles so small products still spread over many SMs, skips the
// k-range outside a triangular operand's band, and uses the shared epilogue.
// Products are exact float32 fused multiply-adds with float32 accumulation in
// a fixed order, so results are deterministic.
#include "epilogue.cuh"

namespace kfm {

namespace {

constexpr int kBK = 16, kThreads = 256;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool pred) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int sz = pred ? 16 : 0;  // 0: nothing is read, the 16 bytes are zero-filled
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(sz) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// BM x BN output tile per CTA, (BM / 16) x (BN / 16) outputs per thread.
// A tile stored [m][k] (row stride BK + 4); op(B) tile stored [n][k] when B is
// N x K (TB), else [k][n] (row stride BN + 4).  Thread (ty, tx) owns rows
// ty + 16 i and columns tx + 16 j (TB) or 4 tx + j (not TB), which keeps every
// shared-memory read free of bank conflicts.
template <int BM, int BN, int kStages, bool TB>
__global__ void __launch_bounds__(kThreads) gemm_small_kernel(GemmParams<float> p) {
  constexpr int TM = BM / 16, TN = BN / 16;
  constexpr int LDA = kBK + 4;
  constexpr int LDB = TB ? kBK + 4 : BN + 4;
  constexpr int A_ELEMS = BM * LDA;
  constexpr int B_ELEMS = TB ? BN * LDB : kBK * LDB;
  __shared__ __align__(16) float As[kStages][A_ELEMS];
  __shared__ __align__(16) float Bs[kStages][B_ELEMS];
  __shared__ int skip;

  const int tm = blockIdx.y, tn = blockIdx.x;
  const int m0 = tm * BM, n0 = tn * BN;
  if (p.sym && n0 > m0 + BM - 1) return;  // tile entirely above the diagonal (CTA-uniform)
  const int tid = threadIdx.x;
  if (tid == 0) skip = status_failed(p.status) ? 1 : 0;  // one read for the whole CTA
  __syncthreads();
  if (skip) return;

  // k-range of this tile: triangular operands are zero outside their band
  int k_lo = 0, k_hi = p.K;
  if (p.tri_a > 0) k_hi = min(k_hi, m0 + BM);
  if (p.tri_a < 0) k_lo = max(k_lo, m0);
  if (p.tri_b > 0) k_hi = min(k_hi, n0 + BN);
  if (p.tri_b < 0) k_lo = max(k_lo, n0);
  k_lo = k_lo / kBK * kBK;
  const int nkt = k_hi > k_lo ? (k_hi - k_lo + kBK - 1) / kBK : 0;

  auto load_stage = [&](int st, int kt) {
    const int k0 = k_lo + kt * kBK;
    // A: BM rows x 4 vectors
    for (int v = tid; v < BM * (kBK / 4); v += kThreads) {
      const int r = v / (kBK / 4), kv = (v % (kBK / 4)) * 4;
      const int gr = m0 + r, gk = k0 + kv;
      const bool ok = gr < p.M && gk < p.K;
      cp_async16(&As[st][r * LDA + kv], ok ? p.A + (int64_t)gr * p.lda + gk : p.A, ok);
    }
    if (TB) {
      for (int v = tid; v < BN * (kBK / 4); v += kThreads) {
        const int r = v / (kBK / 4), kv = (v % (kBK / 4)) * 4;
        const int gc = n0 + r, gk = k0 + kv;
        const bool ok = gc < p.N && gk < p.K;
        cp_async16(&Bs[st][r * LDB + kv], ok ? p.B + (int64_t)gc * p.ldb + gk : p.B, ok);
      }
    } else {
      for (int v = tid; v < kBK * (BN / 4); v += kThreads) {
        const int kk = v / (BN / 4), cv = (v % (BN / 4)) * 4;
        const int gk = k0 + kk, gc = n0 + cv;
        const bool ok = gk < p.K && gc < p.N;  // N % 4 == 0 is required by the dispatcher
        cp_async16(&Bs[st][kk * LDB + cv], ok ? p.B + (int64_t)gk * p.ldb + gc : p.B, ok);
      }
    }
  };

  const int tx = tid % 16, ty = tid / 16;
  float acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.0f;

#pragma unroll
  for (int st = 0; st < kStages - 1; ++st) {
    if (st < nkt) load_stage(st, st);
    cp_async_commit();
  }
  for (int kt = 0; kt < nkt; ++kt) {
    cp_async_wait<kStages - 2>();
    __syncthreads();
    const int st = kt % kStages;
    const float* a_s = As[st];
    const float* b_s = Bs[st];
#pragma unroll
    for (int kq = 0; kq < kBK / 4; ++kq) {
      float4 a4[TM];
#pragma unroll
      for (int i = 0; i < TM; ++i) a4[i] = *reinterpret_cast<const float4*>(a_s + (ty + 16 * i) * LDA + 4 * kq);
      if (TB) {
#pragma unroll
        for (int j = 0; j < TN; ++j) {
          const float4 b4 = *reinterpret_cast<const float4*>(b_s + (tx + 16 * j) * LDB + 4 * kq);
#pragma unroll
          for (int i = 0; i < TM; ++i) {
            acc[i][j] = fmaf(a4[i].x, b4.x, acc[i][j]);
            acc[i][j] = fmaf(a4[i].y, b4.y, acc[i][j]);
            acc[i][j] = fmaf(a4[i].z, b4.z, acc[i][j]);
            acc[i][j] = fmaf(a4[i].w, b4.w, acc[i][j]);
          }
        }
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          float bv[TN];
          if constexpr (TN == 8) {
            const float4 b4 = *reinterpret_cast<const float4*>(b_s + (4 * kq + e) * LDB + TN * tx);
            const float4 b5 = *reinterpret_cast<const float4*>(b_s + (4 * kq + e) * LDB + TN * tx + 4);
            bv[0] = b4.x;
            bv[1] = b4.y;
            bv[2] = b4.z;
            bv[3] = b4.w;
            bv[4] = b5.x;
            bv[5] = b5.y;
            bv[6] = b5.z;
            bv[7] = b5.w;
          } else if constexpr (TN == 4) {
            const float4 b4 = *reinterpret_cast<const float4*>(b_s + (4 * kq + e) * LDB + TN * tx);
            bv[0] = b4.x;
            bv[1] = b4.y;
            bv[2] = b4.z;
            bv[3] = b4.w;
          } else {
            static_assert(TN == 2, "32-, 64- or 128-wide tiles");
            const float2 b2 = *reinterpret_cast<const float2*>(b_s + (4 * kq + e) * LDB + TN * tx);
            bv[0] = b2.x;
            bv[1] = b2.y;
          }
#pragma unroll
          for (int i = 0; i < TM; ++i) {
            const float av = e == 0 ? a4[i].x : e == 1 ? a4[i].y : e == 2 ? a4[i].z : a4[i].w;
#pragma unroll
            for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(av, bv[j], acc[i][j]);
          }
        }
      }
    }
    if (kt + kStages - 1 < nkt) load_stage((kt + kStages - 1) % kStages, kt + kStages - 1);
    cp_async_commit();
  }
  cp_async_wait<0>();

#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int gi = m0 + ty + 16 * i;
    if (gi >= p.M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gj = n0 + (TB ? tx + 16 * j : TN * tx + j);
      if (gj >= p.N) continue;
      if (p.sym && gj > gi) continue;
      epilogue_store(p, gi, gj, acc[i][j]);
    }
  }
}

template <int BM, int BN, int STAGES>
kf_status launch_small(cudaStream_t s, bool transB, const GemmParams<float>& p) {
  const dim3 grid((unsigned)ceil_div(p.N, BN), (unsigned)ceil_div(p.M, BM));
  if (grid.y > 65535) return KF_ERR_ARG;
  if (transB)
    gemm_small_kernel<BM, BN, STAGES, true><<<grid, kThreads, 0, s>>>(p);
  else
    gemm_small_kernel<BM, BN, STAGES, false><<<grid, kThreads, 0, s>>>(p);
  note_launch();
  return launch_check("gemm_small");
}

bool aligned16(const void* ptr) { return (reinterpret_cast<uintptr_t>(ptr) & 15) == 0; }

// Whether the ra x ca block at a and the rb x cb block at b (row strides la,
// lb) share an element.  Exact when la == lb and b's columns do not wrap past
// the stride; conservative (true) otherwise.
bool blocks_overlap(const float* a, int64_t la, int64_t ra, int64_t ca, const float* b, int64_t lb, int64_t rb,
                    int64_t cb) {
  if (ra <= 0 || ca <= 0 || rb <= 0 || cb <= 0) return false;
  const float* a_end = a + (ra - 1) * la + ca;
  const float* b_end = b + (rb - 1) * lb + cb;
  if (a_end <= b || b_end <= a) return false;
  if (la != lb || la <= 0) return true;
  const int64_t d = b - a;
  const int64_t dr = d >= 0 ? d / la : -((-d + la - 1) / la);
  const int64_t dc = d - dr * la;  // 0 <= dc < la
  if (dc + cb > la) return true;
  const bool rows = dr < ra && dr + rb > 0;
  const bool cols = dc < ca && dc + cb > 0;
  return rows && cols;
}

}  // namespace

SmallAlias gemm_small_alias(bool transB, const GemmParams<float>& p) {
  if (!p.out) return SmallAlias::kNone;
  const int64_t rb = transB ? p.N : p.K, cb = transB ? p.K : p.N;
  if (blocks_overlap(p.out, p.ldo, p.M, p.N, p.B, p.ldb, rb, cb)) return SmallAlias::kOther;
  if (blocks_overlap(p.out, p.ldo, p.M, p.N, p.A, p.lda, p.M, p.K)) {
    // out and A may be the same rows (an in-place row transform): safe when one
    // CTA owns whole rows of out and reads each A row only from those rows
    return p.A == p.out && p.lda == p.ldo && p.N <= 128 ? SmallAlias::kSameRows : SmallAlias::kOther;
  }
  return SmallAlias::kNone;
}

bool gemm_small_ok(bool transB, const GemmParams<float>& p) {
  if (p.transA || p.M <= 0 || p.N <= 0 || p.K <= 0) return false;
  if (p.K % 4 || !aligned16(p.A) || p.lda % 4 || !aligned16(p.B) || p.ldb % 4) return false;
  if (!transB && p.N % 4) return false;
  if (p.sym && p.M != p.N) return false;
  return gemm_small_alias(transB, p) != SmallAlias::kOther;
}

kf_status gemm_small(cudaStream_t s, bool transB, const GemmParams<float>& p) {
  if (!gemm_small_ok(transB, p)) return KF_ERR_ARG;
  // In place (out == A): every CTA must own all N <= 128 columns of its rows, so
  // that no other CTA writes a row it still reads; the CTA reads its rows
  // completely before its epilogue writes them.
  if (gemm_small_alias(transB, p) == SmallAlias::kSameRows) return launch_small<32, 128, 3>(s, transB, p);
  if ((int64_t)p.M * p.N <= 256 * 256) return launch_small<32, 32, 4>(s, transB, p);
  return launch_small<64, 64, 4>(s, transB, p);
}

}  // namespace kfm
