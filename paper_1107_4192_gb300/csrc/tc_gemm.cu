// Split-bf16 GEMM on the 5th-generation tensor cores (tcgen05).
//
// C = A B^T for float32 A (M x K) and B (N x K).  Each operand is split into
// S bf16 planes x = x_0 + x_1 (+ x_2), x_k = bf16(x - x_0 - .. - x_{k-1});
// the products A_i B_j^T with i + j < S are accumulated in one float32
// accumulator held in tensor memory (TMEM).  S = 2 is "bf16x3"
// (hi hi + hi lo + lo hi, about 16 significant bits); S = 3 is "bf16x6"
// (six products, about 24 bits, float32-class).  This is
// how the mixed-precision path forms the N x N covariance products: the
// smoother's W = J D and P + W J^T (eqn 13), the innovation U^T = P H^T
// (eqn 8) and the update P - K U (eqn 10).
//
// Kernel structure (one 128 x BN output tile per CTA, 6 warps):
//   warp 0  one lane issues TMA loads (cp.async.bulk.tensor, 128-byte
//           swizzle) of the four operand tiles of a 64-wide k-slice into a
//           shared-memory stage and arms the stage's "full" mbarrier;
//   warp 1  allocates TMEM; one lane waits for "full", issues the 12
//           tcgen05.mma (3 products x 4 k16 steps) and commits them to the
//           stage's "empty" mbarrier, which hands the stage back to the TMA
//           lane when the MMAs have read it; at the end it commits to the
//           "accumulator ready" barrier;
//   warps 2-9  read the accumulator with tcgen05.ld (each warp its 32 TMEM
//           lanes = 32 rows, half of the columns), promote it into float32
//           registers after every k-tile, and at the end stage the tile in
//           shared memory and apply the covariance epilogue in coalesced row
//           and (for mirrored symmetric outputs) column sweeps.
// Every mbarrier wait is bounded by %globaltimer: the pipeline waits by a
// limit passed as a kernel argument (2 s unless kfx_tc_wait_limit set another),
// the clean-up waits by their own 2 s.  On expiry the kernel raises
// KF_ERR_TIMEOUT in the status word, stops issuing, waits (bounded) for what
// it already issued, frees TMEM and returns.
#include <cuda.h>

#include <mutex>

#include "epilogue.cuh"
#include "tc_gemm.cuh"
#include "tc_ptx.cuh"

namespace kfm {

namespace {

constexpr int BM = 128;
constexpr int BK = 64;          // one 128-byte swizzle atom of bf16
constexpr int UMMA_K = 16;
constexpr int NUM_THREADS = 320;  // TMA warp, MMA warp, 8 epilogue warps

template <int BN, int S>  // S = bf16 slices per operand: 2 -> 3 products, 3 -> 6 products
struct TcCfg {
  static constexpr int A_BYTES = BM * BK * 2;   // one plane
  static constexpr int B_BYTES = BN * BK * 2;
  static constexpr int STAGE_BYTES = S * A_BYTES + S * B_BYTES;
  static constexpr int STAGES = (200 * 1024) / STAGE_BYTES;
  static_assert(STAGES >= 2, "need a double-buffered pipeline");
  static constexpr int TMEM_COLS = 2 * BN;      // two float32 accumulators (ping-pong between chunks)
  static constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
  // instruction descriptor: D = f32, A = B = bf16, both K-major, N >> 3, M >> 4
  static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                    ((uint32_t)(BM >> 4) << 24);
};

// 128-byte swizzled K-major operand tile: 8-row x 128-byte atoms stacked every 1024 bytes.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) { return smem_desc_sw(addr, 1024, kLayoutSw128); }

struct TcMaps {
  CUtensorMap a[3], b[3];  // bf16 planes of A and B, most significant first
};

constexpr int KC = 1;  // k-tiles accumulated in TMEM before promotion to registers
constexpr int GROUP = 16;  // row tiles per rasterisation group

// Epilogue threads: warps 2..9.  Warp w reads TMEM lanes 32*(w%4)..+31 (its
// lane quadrant) and one half of the BN columns, so each output row is owned
// by one thread per column half.
template <int BN, int S, typename TE>
__global__ void __launch_bounds__(NUM_THREADS, 1)
    tc_gemm_kernel(const __grid_constant__ TcMaps maps, const GemmParams<TE> p, int num_k_tiles, uint64_t wait_ns) {
  using C = TcCfg<BN, S>;
  constexpr int HALF = BN / 2;
  extern __shared__ uint8_t smem_raw[];
  // grouped rasterisation: consecutive CTAs sweep the column tiles of GROUP row tiles together, so a
  // wave of CTAs reads about GROUP row tiles of A and 152 / GROUP column tiles of B from DRAM per k-tile
  // instead of a few row tiles and every column tile of B
  const int tiles_m = (p.M + BM - 1) / BM, tiles_n = (p.N + BN - 1) / BN;
  const int per_group = GROUP * tiles_n;
  const int grp = blockIdx.x / per_group, first_m = grp * GROUP;
  const int gsize = min(tiles_m - first_m, GROUP);
  const int local = blockIdx.x - grp * per_group;
  const int tm = first_m + local % gsize, tn = local / gsize;
  const int m0 = tm * BM, n0 = tn * BN;
  if (p.sym && m0 + BM - 1 < n0) return;  // tile entirely above the diagonal

  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  uint8_t* gbase = smem_raw + (base - smem_u32(smem_raw));
  const uint32_t bars = base + C::STAGES * C::STAGE_BYTES;
  auto full_bar = [&](int s) { return bars + 8u * s; };
  auto empty_bar = [&](int s) { return bars + 8u * (C::STAGES + s); };
  auto accf_bar = [&](int b) { return bars + 8u * (2 * C::STAGES + b); };      // accumulator b ready
  auto acce_bar = [&](int b) { return bars + 8u * (2 * C::STAGES + 2 + b); };  // accumulator b drained
  const uint32_t done_bar = bars + 8u * (2 * C::STAGES + 4);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gbase + C::STAGES * C::STAGE_BYTES + 8 * (2 * C::STAGES + 5));
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* skip_flag = reinterpret_cast<volatile int*>(tmem_slot + 2);
  volatile int never = 0;  // abort flag for the clean-up waits, which must not stop early

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf_bar(b), 1);
      mbar_init(acce_bar(b), 8);
    }
    mbar_init(done_bar, 1);
    *abort_flag = 0;
    *skip_flag = status_failed(p.status) ? 1 : 0;  // read once, shared by the whole CTA
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(C::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const bool skip = *skip_flag != 0;
  // k-tile band of this output tile (triangular operands contribute nothing outside it)
  int kt0 = 0, kt1 = num_k_tiles;
  if (p.tri_a > 0) kt1 = min(kt1, (m0 + BM + BK - 1) / BK);
  if (p.tri_a < 0) kt0 = max(kt0, m0 / BK);
  if (p.tri_b > 0) kt1 = min(kt1, (n0 + BN + BK - 1) / BK);
  if (p.tri_b < 0) kt0 = max(kt0, n0 / BK);
  const int nk = kt1 > kt0 ? kt1 - kt0 : 0;
  const int nchunks = (nk + KC - 1) / KC;
  bool mma_issued = false;

  if (skip) {
    // an earlier kernel failed: do nothing but release TMEM below
  } else if (warp == 0 && lane == 0) {
    // ---------------- TMA producer
    int last_round[8] = {-1, -1, -1, -1, -1, -1, -1, -1};
    for (int it = 0; it < nk; ++it) {
      const int kt = kt0 + it;
      const int s = it % C::STAGES;
      const uint32_t ph = (uint32_t)(it / C::STAGES) & 1u;
      if (!mbar_wait(empty_bar(s), ph ^ 1u, abort_flag, wait_ns)) {
        *abort_flag = 1;
        status_set(p.status, KF_ERR_TIMEOUT, p.step, 1);
        break;
      }
      const uint32_t st = base + s * C::STAGE_BYTES;
      mbar_expect_tx(full_bar(s), C::STAGE_BYTES);
      const int x = kt * BK;
#pragma unroll
      for (int i = 0; i < S; ++i) tma_load_2d(st + i * C::A_BYTES, &maps.a[i], x, m0, full_bar(s));
#pragma unroll
      for (int j = 0; j < S; ++j) tma_load_2d(st + S * C::A_BYTES + j * C::B_BYTES, &maps.b[j], x, n0, full_bar(s));
      last_round[s] = it / C::STAGES;
    }
    if (*abort_flag) {  // let issued copies land before the CTA's shared memory goes away
      for (int s = 0; s < C::STAGES; ++s)
        if (last_round[s] >= 0) mbar_wait(full_bar(s), (uint32_t)last_round[s] & 1u, &never);
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer: chunk c accumulates into TMEM buffer c & 1
    for (int it = 0; it < nk; ++it) {
      const int c = it / KC, buf = c & 1;
      if (it % KC == 0 && !mbar_wait(acce_bar(buf), ((uint32_t)(c >> 1) & 1u) ^ 1u, abort_flag, wait_ns)) {
        *abort_flag = 1;
        status_set(p.status, KF_ERR_TIMEOUT, p.step, 4);
        break;
      }
      const int s = it % C::STAGES;
      const uint32_t ph = (uint32_t)(it / C::STAGES) & 1u;
      if (!mbar_wait(full_bar(s), ph, abort_flag, wait_ns)) {
        *abort_flag = 1;
        status_set(p.status, KF_ERR_TIMEOUT, p.step, 2);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t st = base + s * C::STAGE_BYTES;
      const uint32_t dacc = tmem + (uint32_t)(buf * BN);
      const bool first_of_chunk = (it % KC) == 0;
#pragma unroll
      for (int k = 0; k < BK / UMMA_K; ++k) {
        const uint32_t off = k * UMMA_K * 2;  // bytes along K inside the swizzle atom
        // products of slice levels i + j < S, least significant first
#pragma unroll
        for (int lvl = S - 1; lvl >= 0; --lvl) {
#pragma unroll
          for (int i = 0; i <= lvl; ++i) {
            const int j = lvl - i;
            const uint32_t acc = (!first_of_chunk || k > 0 || lvl != S - 1 || i != 0) ? 1u : 0u;
            mma_bf16(dacc, smem_desc(st + i * C::A_BYTES + off), smem_desc(st + S * C::A_BYTES + j * C::B_BYTES + off),
                     C::IDESC, acc);
          }
        }
      }
      mma_issued = true;
      mma_commit(empty_bar(s));
      if (it % KC == KC - 1 || it == nk - 1) mma_commit(accf_bar(buf));
    }
  } else if (warp >= 2) {
    // ---------------- epilogue: promote each chunk into float32 registers, then store
    const int q = warp % 4, h = (warp - 2) / 4;
    const int gi = m0 + 32 * q + lane;
    float acc[HALF];
#pragma unroll
    for (int j = 0; j < HALF; ++j) acc[j] = 0.0f;
    bool ok = true;
    for (int c = 0; c < nchunks && ok; ++c) {
      const int buf = c & 1;
      if (!mbar_wait(accf_bar(buf), (uint32_t)(c >> 1) & 1u, abort_flag, wait_ns)) {
        if (!*abort_flag) {
          *abort_flag = 1;
          status_set(p.status, KF_ERR_TIMEOUT, p.step, 3);
        }
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int j = 0; j < HALF; j += 32) {
        uint32_t r[32];
        tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * BN + h * HALF + j), r);
#pragma unroll
        for (int e = 0; e < 32; ++e) acc[j + e] += __uint_as_float(r[e]);
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(acce_bar(buf)) : "memory");
    }
    // Stage the tile in shared memory (the operand stages are idle once the
    // last chunk has been promoted), one column half at a time, then sweep it
    // by rows for the direct outputs and by columns for the mirrored ones, so
    // that every global access of a warp covers consecutive addresses.
    constexpr int PITCH = HALF + 1;  // odd pitch: row and column sweeps are both conflict-free
    static_assert((size_t)BM * PITCH * sizeof(TE) <= (size_t)C::STAGES * C::STAGE_BYTES, "tile fits the stages");
    TE* tile = reinterpret_cast<TE*>(gbase);
    const int ew = warp - 2;  // epilogue warp 0..7
    for (int hh = 0; hh < 2; ++hh) {
      if (ok && h == hh) {
        const int r = 32 * q + lane;
#pragma unroll
        for (int j = 0; j < HALF; ++j) tile[r * PITCH + j] = (TE)acc[j];
      }
      asm volatile("bar.sync 1, 256;" ::: "memory");
      const bool go = !*abort_flag;
      const int c0 = n0 + hh * HALF;
      if (go) {
        // row sweep: lane -> column, warp -> rows ew, ew + 8, ...; the cin / csub
        // values of EB elements are loaded before any of them is stored (cin
        // may be the output array, so the compiler would not hoist them)
        constexpr int CPL = HALF / 32, PER = (BM / 8) * CPL, EB = HALF >= 128 ? 4 : 8;
        static_assert(PER % EB == 0, "whole batches");
        for (int b0 = 0; b0 < PER; b0 += EB) {
          TE cv[EB], sv[EB];
#pragma unroll
          for (int k = 0; k < EB; ++k) {
            const int e = b0 + k, r = ew + 8 * (e / CPL), cc = lane + 32 * (e % CPL);
            const int gi2 = m0 + r, gj = c0 + cc;
            const bool valid = gi2 < p.M && gj < p.N && !(p.sym && gj > gi2);
            cv[k] = (valid && p.cin) ? p.cin[(int64_t)gi2 * p.ldcin + gj] : TE(0);
            sv[k] = (valid && p.csub) ? p.csub[(int64_t)gi2 * p.ldcsub + gj] : TE(0);
          }
#pragma unroll
          for (int k = 0; k < EB; ++k) {
            const int e = b0 + k, r = ew + 8 * (e / CPL), cc = lane + 32 * (e % CPL);
            const int gi2 = m0 + r, gj = c0 + cc;
            if (gi2 < p.M && gj < p.N && !(p.sym && gj > gi2))
              tile[r * PITCH + cc] = epilogue_row(p, gi2, gj, tile[r * PITCH + cc], cv[k], sv[k]);
          }
        }
      }
      if (p.sym == 1) {
        asm volatile("bar.sync 1, 256;" ::: "memory");
        if (go && m0 + BM - 1 > c0) {  // the half has elements strictly below the diagonal
          for (int c = ew; c < HALF; c += 8) {
            const int gj = c0 + c;
            if (gj >= p.N) break;
            for (int r = lane; r < BM; r += 32) {
              const int gi2 = m0 + r;
              if (gi2 >= p.M || gi2 <= gj) continue;
              epilogue_mirror(p, gj, gi2, tile[r * PITCH + c]);
            }
          }
        }
      }
      asm volatile("bar.sync 1, 256;" ::: "memory");  // the tile is rewritten by the next half
    }
  }
  // every issued MMA must have finished before TMEM is freed
  if (!skip && warp == 1 && lane == 0) {
    if (mma_issued) {
      mma_commit(done_bar);
      mbar_wait(done_bar, 0, &never);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TMEM_COLS)
                 : "memory");
  }
}

// ------------------------------------------------------------ host side

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(ptr);
    else
      cudaGetLastError();
  });
  return fn;
}

// rows x cols bf16 plane with leading dimension ld (elements), box = 64 x box_rows.
kf_status make_map(CUtensorMap* map, const void* ptr, int64_t rows, int64_t cols, int64_t ld, int box_rows) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return KF_ERR_UNSUPPORTED;
  if ((reinterpret_cast<uintptr_t>(ptr) & 15) || ((ld * 2) & 15) || cols % BK) return KF_ERR_ARG;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? KF_OK : KF_ERR_CUDA;
}

template <int BN, int S, typename TE>
kf_status launch(cudaStream_t s, const GemmParams<TE>& g, const TcScratch& sc, int64_t ldk, bool b_is_a) {
  using C = TcCfg<BN, S>;
  TcMaps maps;
  for (int i = 0; i < S; ++i) {
    KF_TRY(make_map(&maps.a[i], sc.a[i], g.M, ldk, ldk, BM));
    KF_TRY(make_map(&maps.b[i], b_is_a ? sc.a[i] : sc.b[i], g.N, ldk, ldk, BN));
  }
  KF_CUDA_TRY(smem_limit_per_device((const void*)tc_gemm_kernel<BN, S, TE>, (int)C::SMEM));
  const dim3 grid((unsigned)(ceil_div(g.N, BN) * ceil_div(g.M, BM)));
  const int num_k_tiles = (int)(ldk / BK);
  if (g_tc_timer) g_tc_timer->before(s);
  tc_gemm_kernel<BN, S, TE><<<grid, NUM_THREADS, C::SMEM, s>>>(maps, g, num_k_tiles, g_tc_wait_ns.load());
  if (g_tc_timer) g_tc_timer->after(s);
  note_launch();
  return launch_check("tc_gemm");
}

template <typename TE>
kf_status run_split(cudaStream_t s, TcScratch& sc, const TcOperand& A, const TcOperand& B, const GemmParams<TE>& g,
                    int slices) {
  if (g.M <= 0 || g.N <= 0) return KF_OK;
  if (g.sym && g.M != g.N) return KF_ERR_ARG;
  if (slices != 2 && slices != 3) return KF_ERR_ARG;
  if (g.K == 0) {  // epilogue only: no operand tiles to load
    GemmParams<TE> h = g;
    h.transA = 0;
    return gemm_simt<TE>(s, true, h);
  }
  const int64_t ldk = round_up(g.K, BK);
  if (g.M > sc.rows || g.N > sc.rows || ldk > sc.ld) return KF_ERR_ARG;
  SplitOp oa, ob;
  oa.src = A.p; oa.ld = A.ld; oa.rows = g.M; oa.cols = g.K; oa.trans = A.trans; oa.f64 = A.f64;
  ob.src = B.p; ob.ld = B.ld; ob.rows = g.N; ob.cols = g.K; ob.trans = B.trans; ob.f64 = B.f64;
  for (int i = 0; i < slices; ++i) {
    oa.planes[i] = sc.a[i];
    ob.planes[i] = sc.b[i];
  }
  // the same operand on both sides (W^T W): split it once, the B maps read A's planes
  const bool b_is_a = A.p == B.p && A.ld == B.ld && A.trans == B.trans && A.f64 == B.f64 && g.M == g.N;
  if (b_is_a) ob.rows = 0;
  KF_TRY(split_bf16_pair(s, oa, ob, slices, ldk));
  if (slices == 2) return launch<256, 2, TE>(s, g, sc, ldk, b_is_a);
  return launch<128, 3, TE>(s, g, sc, ldk, b_is_a);
}

}  // namespace

thread_local TcLaunchTimer* g_tc_timer = nullptr;
std::atomic<uint64_t> g_tc_wait_ns{WAIT_NS};

uint64_t tc_scratch_bytes(int64_t rows, int64_t ld) { return 6ull * rows * ld * sizeof(__nv_bfloat16); }

kf_status tc_scratch_alloc(TcScratch& sc, int64_t rows, int64_t ld,
                           const std::function<kf_status(void**, size_t)>& alloc) {
  size_t plane = (size_t)rows * ld * sizeof(__nv_bfloat16);
  for (int i = 0; i < 3; ++i) {
    KF_TRY(alloc((void**)&sc.a[i], plane));
    KF_TRY(alloc((void**)&sc.b[i], plane));
  }
  sc.rows = rows;
  sc.ld = ld;
  return KF_OK;
}

kf_status tma_map_bf16(CUtensorMap* map, const void* ptr, int64_t rows, int64_t cols, int64_t ld, int box_cols,
                       int box_rows, int swizzle_bytes) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return KF_ERR_UNSUPPORTED;
  if (box_cols * 2 != swizzle_bytes || (swizzle_bytes != 32 && swizzle_bytes != 64 && swizzle_bytes != 128))
    return KF_ERR_ARG;
  if ((reinterpret_cast<uintptr_t>(ptr) & 15) || ((ld * 2) & 15) || cols % box_cols) return KF_ERR_ARG;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE,
                   swizzle_bytes == 32   ? CU_TENSOR_MAP_SWIZZLE_32B
                   : swizzle_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                         : CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? KF_OK : KF_ERR_CUDA;
}

bool tc_available() {
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return major == 10 && minor == 3 && encode_fn() != nullptr;
}

kf_status tc_gemm_split(cudaStream_t s, TcScratch& sc, const GemmParams<float>& g, int slices, bool transB) {
  TcOperand A{g.A, g.lda, 0, g.transA}, B{g.B, g.ldb, 0, transB ? 0 : 1};
  return run_split<float>(s, sc, A, B, g, slices);
}

kf_status tc_gemm_ops(cudaStream_t s, TcScratch& sc, const TcOperand& A, const TcOperand& B,
                      const GemmParams<double>& epi, int slices) {
  return run_split<double>(s, sc, A, B, epi, slices);
}

kf_status tc_gemm_ops(cudaStream_t s, TcScratch& sc, const TcOperand& A, const TcOperand& B,
                      const GemmParams<float>& epi, int slices) {
  return run_split<float>(s, sc, A, B, epi, slices);
}

}  // namespace kfm
