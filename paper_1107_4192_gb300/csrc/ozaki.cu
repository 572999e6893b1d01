// Exact-slice (Ozaki-scheme) products on the 5th-generation tensor cores.
//
// Slicing (oz_slice_kernel): one CTA per row finds the row's largest
// magnitude, takes its binary exponent e (max < 2^e), rounds each element to
// the integer X_int = RNE(x 2^(7 + 8(S-1) - e)) and writes its signed base-256
// digits (|q_p| <= 128) as bf16 planes, in integer arithmetic on the bits of
// x (the float64 units of this GPU would make float64 slicing the slow part).
//
// Product (oz_gemm_kernel): one 128 x 64 output tile per CTA, 18 warps.
//   warp 0  one lane issues the TMA loads (64-byte swizzle) of all slices of a
//           32-wide k-slice (two MMA k-steps) of A and B into a shared-memory
//           stage;
//   warp 1  allocates TMEM (LV + 1 buffers of 128 x 64 float32, rotating among
//           the levels so a level's drain overlaps the MMAs); the whole warp
//           runs the issue loop (warp-uniform arithmetic) and one elected lane
//           issues, per stage, the MMAs of every slice pair: per A slice, its
//           partner levels in runs of up to four whose buffers are adjacent,
//           one MMA of N = 64 x run each; after the last k-slice of a level's
//           128-wide chunk it commits the level's buffer to its "ready"
//           barrier, and a level's next chunk starts (overwriting) in a buffer
//           the epilogue has drained;
//   warps 2-17 per chunk and level, read the accumulator (an exact integer
//           below 2^24), convert it to an integer and add it into 64-bit
//           fixed-point accumulators in registers (levels 0-2 and levels 3..
//           in two of them); at the end scale by the row and column exponents
//           and apply the float64 epilogue.
// Every pipeline wait is bounded (kernel argument, as in the split-bf16 kernel).
#include "ozaki.cuh"
#include "tc_ptx.cuh"

namespace kfm {

namespace {

constexpr int OZ_BM = 128;      // output rows per CTA (TMEM lanes)
constexpr int OZ_BN = 64;       // output columns per CTA (TMEM columns per level)
constexpr int OZ_KC = 128;      // values of k per exact chunk
constexpr int OZ_EPI_WARPS = 16;  // 4 TMEM lane quadrants x 4 column quarters of 16
constexpr int OZ_GATE_WARP = 2 + OZ_EPI_WARPS;  // waits for each k-step's operands and buffer
constexpr int OZ_THREADS = 32 * (3 + OZ_EPI_WARPS);
constexpr int OZ_GROUP = 8;     // row tiles per rasterisation group (operand reuse in L2)
constexpr int OZ_ROW_PAD = 128;
constexpr int kOzBK = 32;       // k per pipeline stage of the launched kernels (two MMA k-steps)
constexpr int kOzBadRow = 0x7fffffff;  // exponent marking a row that holds an infinity or NaN

// LV slice levels; BK values of k per pipeline stage, one swizzled row of bf16 (16: 32-byte
// swizzle, one MMA k-step; 32: 64-byte swizzle, two k-steps, half the stages and wider TMA rows).
template <int LV, int BK>
struct OzCfg {
  static_assert(BK == 16 || BK == 32, "one 32- or 64-byte swizzled row of bf16 per stage");
  static constexpr int SWZ = BK * 2;                         // swizzle width in bytes
  static constexpr uint32_t LAYOUT = BK == 16 ? kLayoutSw32 : kLayoutSw64;  // descriptor swizzle mode
  static constexpr uint32_t SBO = 8 * SWZ;                   // bytes between 8-row groups
  static constexpr int KS = BK / 16;                         // MMA k-steps per stage
  static constexpr int CK = OZ_KC / BK;                      // stages per exact chunk
  static constexpr int CKS = OZ_KC / 16;                     // k-steps per exact chunk
  static constexpr int A_BYTES = OZ_BM * BK * 2;
  static constexpr int B_BYTES = OZ_BN * BK * 2;
  static constexpr int STAGE_BYTES = LV * (A_BYTES + B_BYTES);
  static constexpr int FIT = (210 * 1024) / STAGE_BYTES;
  static constexpr int STAGES = FIT > 8 ? 8 : FIT;
  static_assert(STAGES >= 2, "double-buffered pipeline");
  // NB = LV + 1 accumulators rotate among the levels (chunk k of level l in buffer (l + k) mod NB),
  // so the buffer a level leaves is drained while the MMAs continue in the spare one
  static constexpr int NB = LV + 1;
  static_assert(NB * OZ_BN <= 512, "one TMEM accumulator per level plus a spare");
  static_assert(LV < CKS && CKS == 8, "one level changes chunk per k-step; eight k-step patterns");
  // a level has at most LV slice pairs whose products are below 2^14 in magnitude, so one
  // chunk of OZ_KC values of k sums to an integer below 2^24: exact in float32
  static_assert(LV * OZ_KC * 16384 <= (1 << 24), "exact chunk");
  static_assert(2 * STAGES + 2 * NB + 1 <= 28, "barriers fit their 256 bytes");
  static constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES + 1024 + 256;
  // instruction descriptor: D = f32, A = B = bf16, both K-major, M >> 4; N >> 3 at bit 17 per MMA
  static constexpr uint32_t IDESC_M = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(OZ_BM >> 4) << 24);
};

struct OzMaps {
  CUtensorMap a, b;  // all slice planes of A (box 32 x 128) and of B (box 32 x 64)
};

// Full epilogue of element (gi, gj), gi >= gj when sym, from its product value c.
__device__ __forceinline__ double oz_qv(int kind, const double* q, int64_t ldq, int i, int j) {
  if (kind == 0) return i == j ? q[0] : 0.0;
  if (kind == 1) return i == j ? q[i] : 0.0;
  if (kind == 2) return q[(int64_t)i * ldq + j];
  return 0.0;
}

__device__ __forceinline__ void oz_apply(const OzEpilogue& e, int gi, int gj, double c) {
  double v = e.alpha * c;
  if (e.cin) v += e.beta * e.cin[(int64_t)gi * e.ldcin + gj];
  if (gi == gj) v += e.delta;
  if (e.radd_kind >= 0) v += oz_qv(e.radd_kind, e.radd, e.ldradd, gi, gj);
  const bool mirror = e.sym && gi != gj;
  if (e.out) {
    e.out[(int64_t)gi * e.ldo + gj] = v;
    if (mirror) e.out[(int64_t)gj * e.ldo + gi] = v;
  }
  if (e.outf) {
    e.outf[(int64_t)gi * e.ldof + gj] = (float)v;
    if (mirror) e.outf[(int64_t)gj * e.ldof + gi] = (float)v;
  }
  if (e.outT) e.outT[(int64_t)gj * e.ldoT + gi] = v;
  if (e.out2) {
    e.out2[(int64_t)gi * e.ldo2 + gj] = v + oz_qv(e.q_kind, e.q, e.ldq, gi, gj);
    if (mirror) e.out2[(int64_t)gj * e.ldo2 + gi] = v + oz_qv(e.q_kind, e.q, e.ldq, gj, gi);
  }
  if (gi == gj) {
    if (e.diag_out) e.diag_out[gi] = v;
    if (e.check_diag && !(v > 0.0 && isfinite(v))) status_set(e.status, KF_ERR_NUMERIC, e.step, gi);
  }
}

struct OzArgs {
  int M, N, nk;                  // nk = k-slices of BK (all of K)
  int kt_per_split;              // k-slices per split (blockIdx.y)
  double* partials;              // splits > 1: raw sums, split s at partials + s M N (ld N)
  int a_rows_pad, b_rows_pad;    // plane p starts at row p * rows_pad of its map
  const int* ea;
  const int* eb;
  OzEpilogue e;
  uint64_t wait_ns;
};

// Sign, integer mantissa and binary exponent of x (x = sign mant 2^exp2), read from its bits;
// false for an infinity or NaN.
__device__ __forceinline__ bool decompose(double x, long long& mant, int& exp2, bool& neg) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7FF);
  neg = (b >> 63) != 0;
  mant = (long long)(b & 0xFFFFFFFFFFFFFull) | (E ? (1ll << 52) : 0ll);
  exp2 = (E ? E : 1) - 1075;
  return E != 0x7FF;
}
__device__ __forceinline__ bool decompose(float x, long long& mant, int& exp2, bool& neg) {
  const unsigned b = __float_as_uint(x);
  const int E = (int)((b >> 23) & 0xFF);
  neg = (b >> 31) != 0;
  mant = (long long)(b & 0x7FFFFFu) | (E ? (1ll << 23) : 0ll);
  exp2 = (E ? E : 1) - 150;
  return E != 0xFF;
}

// Magnitude bits of x as an unsigned integer: ordered like |x| for finite values, and above
// every finite value for infinities and NaNs.
__device__ __forceinline__ unsigned long long mag_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}
__device__ __forceinline__ unsigned long long mag_bits(float x) {
  return ((unsigned long long)(__float_as_uint(x) & 0x7FFFFFFFu)) << 29;  // same order as a double's bits
}
__device__ __forceinline__ int frexp_exponent(unsigned long long mag, bool f32) {
  const double v = f32 ? (double)__uint_as_float((unsigned)(mag >> 29)) : __longlong_as_double((long long)mag);
  int e = 0;
  if (v > 0.0) frexp(v, &e);
  return e;
}

// x 2^shift rounded to the nearest integer, ties to even (exact integer arithmetic).
__device__ __forceinline__ long long fixed_rne(long long mant, int exp2, bool neg, int shift) {
  const int total = exp2 + shift;
  long long r;
  if (total >= 0) {
    // |x| 2^shift < 2^(7 + 8(S-1)) <= 2^55 for every element of the row, so the shift cannot overflow
    r = total >= 63 ? 0 : mant << total;
  } else {
    const int sh = -total;
    if (sh >= 63) {
      r = 0;
    } else {
      long long q = mant >> sh;
      const long long rem = mant & ((1ll << sh) - 1), half = 1ll << (sh - 1);
      if (rem > half || (rem == half && (q & 1))) ++q;
      r = q;
    }
  }
  return neg ? -r : r;
}

// Slices of one row: X[r][k] = 2^(e - 7 - 8(S-1)) X_int with X_int = RNE(X[r][k] 2^(7 + 8(S-1) - e)),
// written in signed base-256 digits q_0 .. q_{S-1} (each rounded to nearest, ties to even, so
// |q_p| <= 128), all in integer arithmetic.
template <typename T>
__global__ void __launch_bounds__(256) oz_slice_kernel(const T* X, int64_t ld, int64_t rows, int64_t cols, int S,
                                                       __nv_bfloat16* planes, int64_t rows_pad, int64_t ldk,
                                                       int* exps) {
  __shared__ unsigned long long red[8];
  const int64_t r = blockIdx.x;
  const T* row = X + r * ld;
  unsigned long long mx = 0;
  if (r < rows)
    for (int64_t k = threadIdx.x; k < cols; k += blockDim.x) {
      const unsigned long long v = mag_bits(row[k]);
      mx = v > mx ? v : mx;
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = v > mx ? v : mx;
  }
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = mx;
  __syncthreads();
  mx = red[0];
  for (int w = 1; w < (int)blockDim.x / 32; ++w) mx = red[w] > mx ? red[w] : mx;
  const bool row_bad = mx >= 0x7FF0000000000000ull;  // an infinity or NaN: zero slices, marked exponent
  const int e = row_bad ? 0 : frexp_exponent(mx, sizeof(T) == 4);  // max |X[r]| < 2^e
  if (threadIdx.x == 0) exps[r] = row_bad ? kOzBadRow : e;
  const int shift = 7 + 8 * (S - 1) - e;
  const int64_t pstride = rows_pad * ldk;
  for (int64_t k0 = threadIdx.x * 8; k0 < ldk; k0 += (int64_t)blockDim.x * 8) {
    long long xi[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      xi[i] = 0;
      if (r < rows && k0 + i < cols && !row_bad) {
        long long mant;
        int exp2;
        bool neg;
        decompose(row[k0 + i], mant, exp2, neg);
        xi[i] = fixed_rne(mant, exp2, neg, shift);
      }
    }
    for (int p = 0; p < S; ++p) {
      const int sp = 8 * (S - 1 - p);
      uint32_t w[4];
#pragma unroll
      for (int i = 0; i < 8; i += 2) {
        __nv_bfloat16 h[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          long long q = xi[i + j];
          if (sp > 0) q = (q + (1ll << (sp - 1)) - 1 + ((q >> sp) & 1)) >> sp;
          xi[i + j] -= q << sp;
          h[j] = __float2bfloat16_rn((float)q);
        }
        w[i / 2] = (uint32_t)__bfloat16_as_ushort(h[0]) | ((uint32_t)__bfloat16_as_ushort(h[1]) << 16);
      }
      *reinterpret_cast<uint4*>(planes + p * pstride + r * ldk + k0) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
}

// One level's drain by an epilogue warp: read its 16 accumulator columns (exact integers below
// 2^24), hand the buffer back to the MMA issuer, and add the values into the 64-bit fixed-point
// sums (levels 0-2 in units of level 2, levels 3.. in units of level LV-1).
template <int L, int LV>
__device__ __forceinline__ void oz_drain(uint32_t taddr, uint32_t dbar, int lane, long long (&hi)[16],
                                         long long (&lo)[16]) {
  if constexpr (L < LV) {
    uint32_t r[16];
    tmem_ld16(taddr, r);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncwarp();
    if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(dbar) : "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const long long v = (long long)__float2int_rn(__uint_as_float(r[j]));
      if constexpr (L < 3)
        hi[j] += v << (8 * (2 - L));
      else
        lo[j] += v << (8 * (LV - 1 - L));
    }
  }
}

// The MMAs of one k-step t with r = t mod CKS.  Level l's exact chunks are staggered by l k-steps
// and chunk k of level l accumulates in TMEM buffer (l + k) mod NB, so at this k-step level l sits
// in buffer (l + [l >= CKS - r] + cm) mod NB, cm = (t / CKS) mod NB.  Per A slice pa, its
// partner levels pa .. LV-1 go in runs of up to four levels, split at the level CKS - r that has
// moved on (fixed by r, so the runs and all shared-memory offsets are compile-time): one MMA with
// N = 64 x run takes the adjacent B slices pb .. pb+run-1 into the run's adjacent accumulators; a
// run whose buffers pass the last one (known from cm at run time) is issued as two MMAs.  The level
// LS that starts a chunk at this k-step gets its own MMA at pa = 0, the chunk's first, which
// overwrites the accumulator instead of adding to it (at the first k-step every level starts, and
// all of pa = 0's MMAs overwrite).  `pre` runs after the MMAs of the first A slices, about half
// of the k-step's work.
template <int LV, int BK, int R, typename Pre>
__device__ __forceinline__ void oz_issue_kstep(bool leader, uint32_t tmem, uint64_t adesc0, uint64_t bdesc0, int cm,
                                               bool first_step, Pre&& pre) {
  using C = OzCfg<LV, BK>;
  constexpr int LS = R == 0 ? 0 : C::CKS - R;
  constexpr int PRE_AFTER = LV >= 5 ? 2 : 1;
#pragma unroll
  for (int pa = 0; pa < LV; ++pa) {
    if (pa == PRE_AFTER) pre();
    int l0 = pa;
#pragma unroll
    for (int l = pa + 1; l <= LV; ++l) {
      if (l == LV || l - l0 == 4 || l == C::CKS - R || (pa == 0 && LS < LV && l == LS + 1)) {
        const int run = l - l0;
        const uint32_t acc = (pa == 0 && (first_step || l0 == LS)) ? 0u : 1u;
        int b = l0 + (l0 >= C::CKS - R ? 1 : 0) + cm;
        if (b >= C::NB) b -= C::NB;
        const int first = min(run, C::NB - b);
        // the start-address field (bits 0-13, 16-byte units) absorbs the in-stage offsets
        const uint64_t ad = adesc0 + (uint64_t)((pa * C::A_BYTES) >> 4);
        const uint64_t bd = bdesc0 + (uint64_t)(((l0 - pa) * C::B_BYTES) >> 4);
        if (leader) {
          mma_bf16(tmem + (uint32_t)(b * OZ_BN), ad, bd, C::IDESC_M | ((uint32_t)(first * OZ_BN) >> 3 << 17), acc);
          if (first < run)
            mma_bf16(tmem, ad, bd + (uint64_t)((first * C::B_BYTES) >> 4),
                     C::IDESC_M | ((uint32_t)((run - first) * OZ_BN) >> 3 << 17), acc);
        }
        l0 = l;
      }
    }
  }
}

// The gate counter: the number of k-steps whose operands have landed and whose starting level's
// buffer has been drained (written by the gate warp with release, read by the MMA warp with acquire).
__device__ __forceinline__ uint32_t oz_gate_load(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.acquire.cta.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ void oz_gate_store(uint32_t addr, uint32_t v) {
  asm volatile("st.release.cta.shared::cta.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
// Bounded wait until the gate passes k-step t; false on timeout or abort.
__device__ __forceinline__ bool oz_gate_wait(uint32_t addr, uint32_t t, volatile int* abort_flag, uint64_t limit_ns,
                                             uint32_t& gate) {
  gate = oz_gate_load(addr);
  if (gate > t) return true;
  const uint64_t t0 = globaltimer();
  for (;;) {
    gate = oz_gate_load(addr);
    if (gate > t) return true;
    if (*abort_flag || globaltimer() - t0 > limit_ns) return false;
  }
}

template <int LV, int BK>
__global__ void __launch_bounds__(OZ_THREADS, 1) oz_gemm_kernel(const __grid_constant__ OzMaps maps, const OzArgs a) {
  using C = OzCfg<LV, BK>;
  extern __shared__ uint8_t smem_raw[];
  // grouped rasterisation: OZ_GROUP row tiles sweep the column tiles together
  const int tiles_m = (a.M + OZ_BM - 1) / OZ_BM, tiles_n = (a.N + OZ_BN - 1) / OZ_BN;
  const int per_group = OZ_GROUP * tiles_n;
  const int t = blockIdx.x, grp = t / per_group, first_m = grp * OZ_GROUP;
  const int gsize = min(tiles_m - first_m, OZ_GROUP);
  const int local = t - grp * per_group;
  const int m0 = (first_m + local % gsize) * OZ_BM, n0 = (local / gsize) * OZ_BN;
  if (a.e.sym && m0 + OZ_BM - 1 < n0) return;  // tile entirely above the diagonal
  // this CTA's k-slices: [kt0, kt0 + nk)
  const int kt0 = blockIdx.y * a.kt_per_split;
  const int nk = min(a.nk - kt0, a.kt_per_split);

  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  uint8_t* gbase = smem_raw + (base - smem_u32(smem_raw));
  const uint32_t bars = base + C::STAGES * C::STAGE_BYTES;
  auto full_bar = [&](int s) { return bars + 8u * s; };
  auto empty_bar = [&](int s) { return bars + 8u * (C::STAGES + s); };
  auto ready_bar = [&](int b) { return bars + 8u * (2 * C::STAGES + b); };          // buffer b holds a chunk
  auto drained_bar = [&](int b) { return bars + 8u * (2 * C::STAGES + C::NB + b); };  // buffer b is free
  const uint32_t done_bar = bars + 8u * (2 * C::STAGES + 2 * C::NB);
  uint32_t* tmem_slot =
      reinterpret_cast<uint32_t*>(gbase + C::STAGES * C::STAGE_BYTES + 8 * (2 * C::STAGES + 2 * C::NB + 1));
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* skip_flag = reinterpret_cast<volatile int*>(tmem_slot + 2);
  const uint32_t gate_addr = smem_u32(tmem_slot + 3);  // k-steps released to the MMA warp
  volatile int never = 0;  // abort flag of the clean-up waits, which must not stop early

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < C::NB; ++b) {
      mbar_init(ready_bar(b), 1);
      mbar_init(drained_bar(b), OZ_EPI_WARPS);
    }
    mbar_init(done_bar, 1);
    *abort_flag = 0;
    *skip_flag = status_failed(a.e.status) ? 1 : 0;
    tmem_slot[3] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const bool skip = *skip_flag != 0 || nk <= 0;
  bool mma_issued = false;
  bool leader = false;  // the MMA warp's issuing lane: it issues every MMA and every commit

  if (skip) {
    // an earlier kernel failed: do nothing but release TMEM below
  } else if (warp == 0 && lane == 0) {
    // ---------------- TMA producer
    int last_round[8] = {-1, -1, -1, -1, -1, -1, -1, -1};
    for (int it = 0; it < nk; ++it) {
      const int s = it % C::STAGES;
      const uint32_t ph = (uint32_t)(it / C::STAGES) & 1u;
      if (!mbar_wait(empty_bar(s), ph ^ 1u, abort_flag, a.wait_ns)) {
        *abort_flag = 1;
        status_set(a.e.status, KF_ERR_TIMEOUT, a.e.step, 11);
        break;
      }
      const uint32_t st = base + s * C::STAGE_BYTES;
      mbar_expect_tx(full_bar(s), C::STAGE_BYTES);
      const int x = (kt0 + it) * BK;
#pragma unroll
      for (int p = 0; p < LV; ++p) tma_load_2d(st + p * C::A_BYTES, &maps.a, x, p * a.a_rows_pad + m0, full_bar(s));
#pragma unroll
      for (int p = 0; p < LV; ++p)
        tma_load_2d(st + LV * C::A_BYTES + p * C::B_BYTES, &maps.b, x, p * a.b_rows_pad + n0, full_bar(s));
      last_round[s] = it / C::STAGES;
    }
    if (*abort_flag) {  // let issued copies land before the CTA's shared memory goes away
      for (int s = 0; s < C::STAGES; ++s)
        if (last_round[s] >= 0) mbar_wait(full_bar(s), (uint32_t)last_round[s] & 1u, &never);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer: the whole warp runs the loop, so the stage, buffer and descriptor
    // arithmetic is warp-uniform; one elected lane issues.  TMEM buffer b = columns [64 b, 64 b + 64).
    // The gate warp tells it which k-steps may start (operands landed, new buffer drained); the
    // MMA queue is shallow, so the issuer does no barrier test of its own between k-steps: it reads
    // the gate counter half-way through each k-step's MMAs, and that load's latency overlaps them.
    leader = elect_one();
    bool ok = true;
    uint32_t gate = 0;  // k-steps released so far (last value read)
    const int nks = nk * C::KS;
    for (int it = 0; it < nk && ok; ++it) {
      const int s = it % C::STAGES;
      const uint32_t st = base + s * C::STAGE_BYTES;
      const uint64_t adesc_s = smem_desc_sw(st, C::SBO, C::LAYOUT);
      const uint64_t bdesc_s = smem_desc_sw(st + LV * C::A_BYTES, C::SBO, C::LAYOUT);
#pragma unroll
      for (int j = 0; j < C::KS; ++j) {
        const int t = it * C::KS + j;  // k-step
        if (gate <= (uint32_t)t) {
          ok = __all_sync(0xffffffffu, oz_gate_wait(gate_addr, (uint32_t)t, abort_flag, a.wait_ns, gate));
          gate = __shfl_sync(0xffffffffu, gate, 0);
          if (!ok) {
            if (lane == 0 && !*abort_flag) {
              *abort_flag = 1;
              status_set(a.e.status, KF_ERR_TIMEOUT, a.e.step, 12);
            }
            break;
          }
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int ck = t / C::CKS, r = t - ck * C::CKS, cm = ck % C::NB;
        auto buf = [&](int l) {  // buffer of level l at this k-step
          const int b = l + cm + (l >= C::CKS - r ? 1 : 0);
          return b >= C::NB ? b - C::NB : b;
        };
        uint32_t gate_ahead = gate;
        auto pre = [&]() { gate_ahead = oz_gate_load(gate_addr); };
        // k-step j reads the next 32 bytes of every swizzled row (start address in 16-byte units)
        const uint64_t adesc0 = adesc_s + (uint64_t)(2 * j), bdesc0 = bdesc_s + (uint64_t)(2 * j);
        switch (r) {
          case 0: oz_issue_kstep<LV, BK, 0>(leader, tmem, adesc0, bdesc0, cm, t == 0, pre); break;
          case 1: oz_issue_kstep<LV, BK, 1>(leader, tmem, adesc0, bdesc0, cm, t == 0, pre); break;
          case 2: oz_issue_kstep<LV, BK, 2>(leader, tmem, adesc0, bdesc0, cm, t == 0, pre); break;
          case 3: oz_issue_kstep<LV, BK, 3>(leader, tmem, adesc0, bdesc0, cm, t == 0, pre); break;
          case 4: oz_issue_kstep<LV, BK, 4>(leader, tmem, adesc0, bdesc0, cm, t == 0, pre); break;
          case 5: oz_issue_kstep<LV, BK, 5>(leader, tmem, adesc0, bdesc0, cm, t == 0, pre); break;
          case 6: oz_issue_kstep<LV, BK, 6>(leader, tmem, adesc0, bdesc0, cm, t == 0, pre); break;
          default: oz_issue_kstep<LV, BK, 7>(leader, tmem, adesc0, bdesc0, cm, t == 0, pre); break;
        }
        __syncwarp();
        mma_issued = true;
        if (leader) {  // the level whose chunk ends here (every level at the last k-step) is ready
#pragma unroll
          for (int l = 0; l < LV; ++l)
            if ((t + l) % C::CKS == C::CKS - 1 || t == nks - 1) mma_commit(ready_bar(buf(l)));
        }
        gate = __shfl_sync(0xffffffffu, max(gate, gate_ahead), 0);
      }
      if (!ok) break;
      if (leader) mma_commit(empty_bar(s));
      __syncwarp();
    }
  } else if (warp == OZ_GATE_WARP) {
    // ---------------- gate: per k-step, wait (bounded) for its stage's operands (at the stage's
    // first k-step) and, when a level starts a chunk there in a buffer used before, for that
    // buffer's drain; then release the k-step to the MMA warp.  Level l's exact chunks are
    // staggered by l k-steps (chunk k covers k-steps [k CKS - l, (k + 1) CKS - l)), so at most one
    // level starts a chunk per k-step, and chunk k of level l accumulates in buffer (l + k) mod NB.
    // That buffer last held chunk k - 1 of level l + 1, which ended two k-steps earlier: its drain
    // has a full k-step of MMAs to finish.
    uint32_t used = 0, par = 0;  // per buffer: used before; parity of its uses so far
    const int nks = nk * C::KS;
    for (int t = 0; t < nks; ++t) {
      const int it = t / C::KS;
      if (t == it * C::KS) {
        const int s = it % C::STAGES;
        const uint32_t ph = (uint32_t)(it / C::STAGES) & 1u;
        if (!__all_sync(0xffffffffu, mbar_wait(full_bar(s), ph, abort_flag, a.wait_ns))) {
          if (lane == 0 && !*abort_flag) {
            *abort_flag = 1;
            status_set(a.e.status, KF_ERR_TIMEOUT, a.e.step, 15);
          }
          break;
        }
      }
      const int ck = t / C::CKS, r = t - ck * C::CKS, cm = ck % C::NB;
      if (t == 0) {
        used = par = (1u << LV) - 1u;
      } else {
        const int ls = r == 0 ? 0 : C::CKS - r;
        if (ls < LV) {
          int b = ls + cm + 1;  // the starting level has moved on: (ls + (t + ls) / CKS) mod NB
          if (r == 0) b = cm;
          if (b >= C::NB) b -= C::NB;
          if ((used >> b) & 1u) {
            if (!__all_sync(0xffffffffu, mbar_wait(drained_bar(b), ((par >> b) & 1u) ^ 1u, abort_flag, a.wait_ns))) {
              if (lane == 0 && !*abort_flag) {
                *abort_flag = 1;
                status_set(a.e.status, KF_ERR_TIMEOUT, a.e.step, 13);
              }
              break;
            }
          }
          used |= 1u << b;
          par ^= 1u << b;
        }
      }
      __syncwarp();
      if (lane == 0) oz_gate_store(gate_addr, (uint32_t)(t + 1));
    }
  } else if (warp >= 2) {
    // ---------------- epilogue: exact level sums into 64-bit fixed point, then scale and store
    const int q = warp % 4, h = (warp - 2) / 4;  // TMEM lane quadrant (fixed by the warp index), column quarter
    const int gi = m0 + 32 * q + lane;
    long long hi[16], lo[16];  // levels 0-2 in units of level 2; levels 3.. in units of level LV-1
#pragma unroll
    for (int j = 0; j < 16; ++j) hi[j] = lo[j] = 0;
    bool ok = true;
    // drain events in the MMA issuer's order: at k-step t, the level whose staggered chunk ends
    // there; at the last k-step, every level
    uint32_t rpar = 0;  // per buffer: parity of its drains so far
    const int nks = nk * C::KS;
    for (int t = 0; t < nks && ok; ++t) {
      const bool final_step = t == nks - 1;
      const int lone = (C::CKS - 1 - t % C::CKS);  // the level whose chunk ends at k-step t
      for (int l = final_step ? 0 : lone; l < (final_step ? LV : min(lone + 1, LV)); ++l) {
        const int b = (l + (t + l) / C::CKS) % C::NB;
        const uint32_t ph = (rpar >> b) & 1u;
        rpar ^= 1u << b;
        if (!mbar_wait(ready_bar(b), ph, abort_flag, a.wait_ns)) {
          if (!*abort_flag) {
            *abort_flag = 1;
            status_set(a.e.status, KF_ERR_TIMEOUT, a.e.step, 14);
          }
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * OZ_BN + h * 16);
        const uint32_t dbar = drained_bar(b);
        // compile-time level, so the shifts are constants and the conversions 32-bit
        switch (l) {
          case 0: oz_drain<0, LV>(taddr, dbar, lane, hi, lo); break;
          case 1: oz_drain<1, LV>(taddr, dbar, lane, hi, lo); break;
          case 2: oz_drain<2, LV>(taddr, dbar, lane, hi, lo); break;
          case 3: oz_drain<3, LV>(taddr, dbar, lane, hi, lo); break;
          case 4: oz_drain<4, LV>(taddr, dbar, lane, hi, lo); break;
          case 5: oz_drain<5, LV>(taddr, dbar, lane, hi, lo); break;
          case 6: oz_drain<6, LV>(taddr, dbar, lane, hi, lo); break;
          default: break;
        }
      }
    }
    // Stage the tile's product values in shared memory (the operand stages are idle once the last
    // chunk has been drained), then sweep it by rows for the direct outputs (lane -> column, so every
    // warp access is contiguous) and by columns for the mirrored and transposed outputs.
    constexpr int PITCH = OZ_BN + 1;  // odd pitch: row and column sweeps are both conflict-free
    static_assert((size_t)OZ_BM * PITCH * sizeof(double) <= (size_t)C::STAGES * C::STAGE_BYTES, "tile fits");
    double* tile = reinterpret_cast<double*>(gbase);
    if (ok) {
      const int ei = gi < a.M ? a.ea[gi] : 0;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int gj = n0 + h * 16 + j;
        const int ej = gj < a.N ? a.eb[gj] : 0;
        const int sc = ei + ej - 14;
        tile[(32 * q + lane) * PITCH + h * 16 + j] =
            (ei == kOzBadRow || ej == kOzBadRow)
                ? __longlong_as_double(0x7ff8000000000000ll)  // a non-finite operand row
                : scalbn((double)hi[j], sc - 16) + scalbn((double)lo[j], sc - 8 * (LV - 1));
      }
    }
    asm volatile("bar.sync 1, %0;" ::"n"(32 * OZ_EPI_WARPS) : "memory");
    const bool go = !*abort_flag;
    const int ew = warp - 2;  // epilogue warp 0..15
    const OzEpilogue& e = a.e;
    double* part = a.partials ? a.partials + (int64_t)blockIdx.y * a.M * a.N : nullptr;
    if (go) {
      for (int r = ew; r < OZ_BM; r += OZ_EPI_WARPS) {
        const int gi2 = m0 + r;
        if (gi2 >= a.M) break;
#pragma unroll
        for (int cc = 0; cc < OZ_BN; cc += 32) {
          const int c = cc + lane, gj = n0 + c;
          if (gj >= a.N || (e.sym && gj > gi2)) continue;
          const double cval = tile[r * PITCH + c];
          if (part) {
            part[(int64_t)gi2 * a.N + gj] = cval;
            continue;
          }
          double v = e.alpha * cval;
          if (e.cin) v += e.beta * e.cin[(int64_t)gi2 * e.ldcin + gj];
          if (gi2 == gj) v += e.delta;
          if (e.radd_kind >= 0) v += oz_qv(e.radd_kind, e.radd, e.ldradd, gi2, gj);
          if (e.out) e.out[(int64_t)gi2 * e.ldo + gj] = v;
          if (e.outf) e.outf[(int64_t)gi2 * e.ldof + gj] = (float)v;
          if (e.out2) e.out2[(int64_t)gi2 * e.ldo2 + gj] = v + oz_qv(e.q_kind, e.q, e.ldq, gi2, gj);
          if (gi2 == gj) {
            if (e.diag_out) e.diag_out[gi2] = v;
            if (e.check_diag && !(v > 0.0 && isfinite(v))) status_set(e.status, KF_ERR_NUMERIC, e.step, gi2);
          }
          tile[r * PITCH + c] = v;  // for the column sweep
        }
      }
    }
    if (!part && (e.sym || e.outT)) {
      asm volatile("bar.sync 1, %0;" ::"n"(32 * OZ_EPI_WARPS) : "memory");
      if (go) {
        for (int c = ew; c < OZ_BN; c += OZ_EPI_WARPS) {
          const int gj = n0 + c;
          if (gj >= a.N) break;
#pragma unroll
          for (int rr = 0; rr < OZ_BM; rr += 32) {
            const int r = rr + lane, gi2 = m0 + r;
            if (gi2 >= a.M || (e.sym && gj > gi2)) continue;
            const double v = tile[r * PITCH + c];
            if (e.outT) e.outT[(int64_t)gj * e.ldoT + gi2] = v;
            if (e.sym && gi2 != gj) {  // mirror (gj, gi2): consecutive lanes write consecutive columns
              if (e.out) e.out[(int64_t)gj * e.ldo + gi2] = v;
              if (e.outf) e.outf[(int64_t)gj * e.ldof + gi2] = (float)v;
              if (e.out2) e.out2[(int64_t)gj * e.ldo2 + gi2] = v + oz_qv(e.q_kind, e.q, e.ldq, gj, gi2);
            }
          }
        }
      }
    }
  }
  // every issued MMA must have finished before TMEM is freed
  if (!skip && warp == 1 && leader && mma_issued) {
    mma_commit(done_bar);
    mbar_wait(done_bar, 0, &never);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

// Sum of the split-K partials in split order, then the epilogue (one thread per element).
__global__ void oz_reduce_kernel(int M, int N, int splits, const double* partials, OzEpilogue e) {
  if (status_failed(e.status)) return;
  const int64_t total = (int64_t)M * N;
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < total; u += (int64_t)gridDim.x * blockDim.x) {
    const int gi = (int)(u / N), gj = (int)(u % N);
    if (e.sym && gj > gi) continue;
    double c = 0.0;
    for (int sp = 0; sp < splits; ++sp) c += partials[(int64_t)sp * total + u];
    oz_apply(e, gi, gj, c);
  }
}

template <int LV, int BK>
kf_status launch_oz(cudaStream_t s, const OzSlices& A, const OzSlices& B, int M, int N, int K, const OzEpilogue& e,
                    int splits, double* partials) {
  using C = OzCfg<LV, BK>;
  OzMaps maps;
  KF_TRY(tma_map_bf16(&maps.a, A.planes, (int64_t)A.S * A.rows_pad, A.ldk, A.ldk, BK, OZ_BM, C::SWZ));
  KF_TRY(tma_map_bf16(&maps.b, B.planes, (int64_t)B.S * B.rows_pad, B.ldk, B.ldk, BK, OZ_BN, C::SWZ));
  OzArgs a;
  a.M = M;
  a.N = N;
  a.nk = (int)ceil_div(K, BK);
  // whole exact chunks per split, so chunk boundaries do not depend on the split
  a.kt_per_split = (int)(ceil_div(ceil_div(K, OZ_KC), splits) * C::CK);
  a.partials = splits > 1 ? partials : nullptr;
  a.a_rows_pad = (int)A.rows_pad;
  a.b_rows_pad = (int)B.rows_pad;
  a.ea = A.exps;
  a.eb = B.exps;
  a.e = e;
  a.wait_ns = g_tc_wait_ns.load();
  KF_CUDA_TRY(smem_limit_per_device((const void*)oz_gemm_kernel<LV, BK>, (int)C::SMEM));
  const int64_t tiles = ceil_div(M, OZ_BM) * ceil_div(N, OZ_BN);
  if (g_oz_timer) g_oz_timer->before(s);
  oz_gemm_kernel<LV, BK><<<dim3((unsigned)tiles, (unsigned)splits), OZ_THREADS, C::SMEM, s>>>(maps, a);
  if (g_oz_timer) g_oz_timer->after(s);
  note_launch();
  KF_TRY(launch_check("oz_gemm"));
  if (splits > 1) {
    const int64_t total = (int64_t)M * N;
    oz_reduce_kernel<<<(unsigned)std::min<int64_t>(ceil_div(total, 256), 4096), 256, 0, s>>>(M, N, splits, partials, e);
    note_launch();
    KF_TRY(launch_check("oz_reduce"));
  }
  return KF_OK;
}

}  // namespace

thread_local TcLaunchTimer* g_oz_timer = nullptr;

uint64_t oz_slice_bytes(int64_t rows, int64_t cols, int S) {
  const uint64_t rp = round_up(std::max<int64_t>(rows, 1), OZ_ROW_PAD), ldk = round_up(std::max<int64_t>(cols, 1), 64);
  return round_up((int64_t)(S * rp * ldk * 2), 256) + rp * 4;
}

void oz_slice_layout(OzSlices& out, void* mem, int64_t rows, int64_t cols, int S) {
  out.rows = rows;
  out.rows_pad = round_up(std::max<int64_t>(rows, 1), OZ_ROW_PAD);
  out.ldk = round_up(std::max<int64_t>(cols, 1), 64);
  out.S = S;
  out.planes = static_cast<__nv_bfloat16*>(mem);
  out.exps = reinterpret_cast<int*>(static_cast<char*>(mem) + round_up((int64_t)(S * out.rows_pad * out.ldk * 2), 256));
}

kf_status oz_slice(cudaStream_t s, const void* X, int64_t ld, int f64, int64_t rows, int64_t cols, int S,
                   OzSlices& out) {
  if (rows < 1 || cols < 1 || S < 1 || S > out.S || rows > out.rows_pad || cols > out.ldk || ld < cols || !X)
    return KF_ERR_ARG;
  out.rows = rows;
  out.filled = S;
  if (f64)
    oz_slice_kernel<double><<<(unsigned)out.rows_pad, 256, 0, s>>>(static_cast<const double*>(X), ld, rows, cols, S,
                                                                   out.planes, out.rows_pad, out.ldk, out.exps);
  else
    oz_slice_kernel<float><<<(unsigned)out.rows_pad, 256, 0, s>>>(static_cast<const float*>(X), ld, rows, cols, S,
                                                                  out.planes, out.rows_pad, out.ldk, out.exps);
  note_launch();
  return launch_check("oz_slice");
}

kf_status oz_gemm(cudaStream_t s, const OzSlices& A, const OzSlices& B, int M, int N, int K, int levels,
                  const OzEpilogue& e, int splits, double* partials) {
  if (M <= 0 || N <= 0) return KF_OK;
  if (K < 1 || K > (1 << 20)) return KF_ERR_ARG;
  if (!e.out && !e.outf && !e.outT && !e.out2 && !e.diag_out) return KF_ERR_ARG;
  if (M > A.rows || N > B.rows || K > A.ldk || K > B.ldk) return KF_ERR_ARG;
  if (A.filled < levels || B.filled < levels || (e.sym && M != N)) return KF_ERR_ARG;
  if (splits < 1 || splits > 64 || (splits > 1 && !partials)) return KF_ERR_ARG;
  // whole exact chunks per split, every split non-empty
  const int64_t chunks = ceil_div(K, OZ_KC);
  splits = (int)std::min<int64_t>(splits, chunks);
  splits = (int)ceil_div(chunks, ceil_div(chunks, splits));
  switch (levels) {
    case 4: return launch_oz<4, kOzBK>(s, A, B, M, N, K, e, splits, partials);
    case 5: return launch_oz<5, kOzBK>(s, A, B, M, N, K, e, splits, partials);
    case 6: return launch_oz<6, kOzBK>(s, A, B, M, N, K, e, splits, partials);
    case 7: return launch_oz<7, kOzBK>(s, A, B, M, N, K, e, splits, partials);
  }
  return KF_ERR_ARG;
}

}  // namespace kfm
