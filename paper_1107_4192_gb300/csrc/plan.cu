// Plan / executor behind the C ABI of include/kfmeg.h.
//
// One plan = one epoch shape (N, m, T) with its precision mode.  It owns:
//  - the working covariance P (bulk dtype, N x ldN with ldN = N rounded up
//    to 128 so every row starts 16-byte aligned),
//  - the covariance store of P_{t|t} (slot 0 holds P0), either complete or as
//    checkpoints every c steps plus one segment buffer, the skipped steps
//    being recomputed forward during the smoother (the covariance recursion
//    does not depend on the data),
//  - the filter's small buffers (U^T = P H^T, the gain K, S and its factor),
//  - the smoother's buffers (factor of P_{t+1|t}, J_t, W = J_t D, D), and
//  - plan-owned copies of F, Q, H, R so fis_smooth needs no caller input.
// Every time step is a fixed launch sequence on the plan's stream; a device
// status word is read once at the end of kf_filter / fis_smooth.
#include <math.h>
#include <string.h>

#include <vector>

#include "arena.cuh"
#include "ops.cuh"
#include "solve_tc.cuh"
#include "tc_gemm.cuh"

using namespace kfm;

namespace {

enum Bulk { BULK_F64 = 0, BULK_F32 = 1, BULK_BF16X3 = 2 };

struct ProfMark {
  int cls;
  cudaEvent_t a, b;
};

constexpr int kSplitsS = 8;   // split-K factor of S = H U^T (CUDA-core paths)
constexpr int kOzSplitsS = 16;  // split-K factor of S = H U^T (exact-slice product)
constexpr int kOzLevels = 5;    // slice levels of the mixed filter's products (about 2^-37 of |A||B|)

}  // namespace

struct kf_plan_s {
  kf_desc d{};
  cudaStream_t s = nullptr;
  int64_t N = 0, m = 0, T = 0, ldN = 0, ldm = 0;
  int bulk = 0, solve = 0;
  bool refine = false;    // KF_SOLVE_FP64_TC: float64-accurate inverse of P_{t+1|t}
  bool mean_refine = false;  // KF_SOLVE_FP64_MEAN: float64-accurate solve of the smoothed mean
  float* X0f = nullptr;      // W^T W (KF_SOLVE_FP64_MEAN)
  // Mixed path with a float64 smoother solve (KF_SOLVE_FP64, _TC, _MEAN): P_{t+1|t} formed in
  // float64 from the float32 store, and F P_{t|t} (non-identity F) for the mean's P_{t|t} F^T y.
  double *Pn64 = nullptr, *FP64 = nullptr;
  double *ysol = nullptr, *rsol = nullptr, *wsol = nullptr;  // its vectors
  int smooth_slices = 2;  // bf16 planes per operand in the smoother products (mixed mode)
  size_t b = 8, sb = 8;   // bytes per bulk / solve element
  int64_t ckpt = 1;       // 1 = every P_{t|t} stored
  int64_t nck = 0;        // checkpoint slots
  int64_t seg_id = -1;    // segment currently held by the segment buffer
  size_t slot = 0;        // bytes of one N x ldN bulk matrix
  std::vector<void*> allocs;

  char* store = nullptr;
  char* seg = nullptr;
  double *xpred = nullptr, *xfilt = nullptr, *xs = nullptr, *nu = nullptr, *dx = nullptr;
  char *P = nullptr, *Ut = nullptr, *Zb = nullptr, *KV = nullptr, *VK = nullptr, *Hb = nullptr, *tmpN = nullptr;
  char *Fb = nullptr, *S0b = nullptr;
  double *S = nullptr, *S0 = nullptr, *Sdinv = nullptr, *partials = nullptr;
  char *Sl = nullptr, *Sldinv = nullptr;
  char *Lb = nullptr, *Ldinv = nullptr, *Jb = nullptr;
  float* Wi = nullptr;    // L^{-1} for the tensor-core solve (mixed mode, float32 solve)
  RefineBufs rb{};        // refinement buffers (KF_SOLVE_FP64_TC)
  double* J64 = nullptr;  // float64 J_t (KF_SOLVE_FP64_TC)
  double *P64 = nullptr, *W64 = nullptr, *U64 = nullptr, *Z64 = nullptr;  // float64 working covariance / first update
  // Mixed filter (exact-slice products): U = H P (m x N, besides U^T in U64), L^{-1} and L^{-T} of the
  // innovation factor, [K V] and [V K] of the Joseph form, split-K partials of S, the slices of every
  // operand (5 levels), and a device 1.0 for identities.
  double *Um = nullptr, *Linv = nullptr, *LinvT = nullptr, *KV64 = nullptr, *VK64 = nullptr, *ozpart = nullptr;
  OzSlices sP, sH, sU, sUt, sL, sLT, sZ, sK, sS0, sKV, sVK;
  // The Cholesky + inverse of P_{t+1|t} is the same launch sequence at every
  // smoother step (only the step number differs, which kernels read from the
  // status word), so it is captured once into a CUDA graph and replayed.
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t chol_graph = nullptr;
  int64_t graph_launches = 0;  // kernels inside one replay of chol_graph
  char *Jm = nullptr, *Wb = nullptr, *Db = nullptr, *Pn = nullptr;
  TcScratch tc{};
  double *F = nullptr, *Q = nullptr, *H = nullptr, *R = nullptr;
  int64_t *Frp = nullptr, *Fcol = nullptr;
  int* status = nullptr;
  int status_h[ST_WORDS] = {0, 0, 0, 0};  // read after a stream synchronisation
  bool filtered = false;
  // staging for kf_solve_host (allocated on first use)
  double *hY = nullptr, *hx0 = nullptr, *hP0 = nullptr, *hQ = nullptr, *hH = nullptr, *hR = nullptr,
         *hF = nullptr, *hxf = nullptr, *hdf = nullptr, *hxs = nullptr, *hds = nullptr;
  int64_t *hFrp = nullptr, *hFcol = nullptr;
  // profiling
  bool prof = false;
  std::vector<ProfMark> marks;
  std::vector<cudaEvent_t> pool;
  int64_t launches = 0;  // kernels launched by this plan's calls

  // Store slots: every P_{t|t} when ckpt == 1; otherwise checkpoints at
  // t = 0, c, 2c, .., a permanent slot for t = 1 (see filter_first_fp64) and a
  // segment buffer for the other steps of one segment.
  char* slot_ptr(int64_t t) {
    if (ckpt == 1) return store + (size_t)t * slot;
    if (t % ckpt == 0) return store + (size_t)(t / ckpt) * slot;
    if (t == 1) return store + (size_t)nck * slot;
    return seg + (size_t)(t % ckpt - 1) * slot;
  }
};

namespace {

size_t cov_count(int kind, int64_t n) { return kind == 0 ? 1 : kind == 1 ? (size_t)n : (size_t)n * n; }

struct Sizes {
  uint64_t workspace = 0, slot = 0;
  int64_t ldN = 0, ldm = 0;
  size_t b = 8, sb = 8;
};

Sizes sizes_for(const kf_desc* d) {
  Sizes z;
  z.b = d->prec == KF_PREC_FP64 ? 8 : 4;
  z.sb = (d->prec == KF_PREC_FP64 || d->solve_prec == KF_SOLVE_FP64) ? 8 : 4;  // KF_SOLVE_FP64_TC: float32 factor
  z.ldN = round_up(d->N, 128);
  z.ldm = round_up(d->m, 64);
  const uint64_t N = d->N, m = d->m, T = d->T, ldN = z.ldN, ldm = z.ldm;
  z.slot = N * ldN * z.b;
  uint64_t w = 0;
  w += 2 * z.slot;                          // P, tmpN
  w += 2 * N * ldm * z.b;                   // Ut, Z
  w += 2 * N * 2 * ldm * z.b;               // KV, VK
  w += m * ldN * z.b;                       // Hb
  w += 2 * m * m * 8 + round_up(m, 64) * 64 * 8 + kSplitsS * m * m * 8;  // S, S0, Sdinv, partials
  w += (m * m + round_up(m, 64) * 64) * z.b + m * m * z.b;               // Sl, Sldinv, S0b
  const int64_t nbs = z.sb == 8 ? 64 : 128;
  w += 2 * N * ldN * z.sb + round_up(N, nbs) * nbs * z.sb;                 // Lb, Jb, Ldinv
  w += (z.sb != z.b ? z.slot : 0) + 3 * z.slot;                            // Jm, Wb, Db, Pn
  if (d->prec == KF_PREC_MIXED_BF16X3 && z.sb == 4) w += z.slot;         // Wi
  if (d->solve_prec == KF_SOLVE_FP64_TC) w += refine_bytes(N, ldN) + N * ldN * 8;  // refinement, J in float64
  if (d->solve_prec == KF_SOLVE_FP64_MEAN) w += z.slot + 3 * N * 8;                 // W^T W, vectors
  if (d->prec == KF_PREC_MIXED_BF16X3 && d->solve_prec != KF_SOLVE_FP32)
    w += N * ldN * 8 * (d->f_kind != KF_F_IDENTITY ? 2 : 1) + 3 * N * 8;          // P_{t+1|t}, F P, vectors
  if (d->prec == KF_PREC_MIXED_BF16X3) {
    // exact-slice filter: U, L^{-1}, L^{-T}, [K V], [V K], S partials, slices
    w += m * ldN * 8 + 2 * m * m * 8 + (d->joseph_every > 0 ? 4 * N * ldm * 8 : 0) + kOzSplitsS * m * m * 8 + 8;
    const int S = kOzLevels;
    w += oz_slice_bytes(N, N, S) + 2 * oz_slice_bytes(m, N, S) + 3 * oz_slice_bytes(N, m, S) +
         3 * oz_slice_bytes(m, m, S) + (d->joseph_every > 0 ? 2 * oz_slice_bytes(N, 2 * ldm, S) : 0) + 12 * 256;
  }
  if (z.b == 4) w += N * ldN * 8 * (d->f_kind != KF_F_IDENTITY ? 2 : 1) + 2 * N * ldm * 8;  // first update
  w += 3 * (T + 1) * N * 8 + m * 8 + N * 8;                                // means
  if (d->f_kind == KF_F_CSR) w += d->f_nnz * 16 + (N + 1) * 8;
  if (d->f_kind == KF_F_DENSE) w += N * N * 8 + z.slot;
  w += cov_count(d->q_kind, N) * 8 + m * N * 8 + cov_count(d->r_kind, m) * 8;
  // split planes: rows up to max(N, m), k up to max(ldN, 2 ldm) (the Joseph product's rank 2m)
  if (d->prec == KF_PREC_MIXED_BF16X3) w += tc_scratch_bytes(std::max(N, m), std::max(ldN, 2 * ldm));
  w += 4096;
  z.workspace = w;
  return z;
}

kf_status validate(const kf_desc* d) {
  if (!d) return KF_ERR_ARG;
  if (d->N < 1 || d->m < 1 || d->T < 1) return KF_ERR_ARG;
  if (d->N > (1ll << 30) || d->m > (1ll << 20) || d->T > (1ll << 30)) return KF_ERR_ARG;
  if (d->f_kind < 0 || d->f_kind > 2) return KF_ERR_ARG;
  if (d->f_kind == KF_F_CSR && d->f_nnz < 1) return KF_ERR_ARG;
  if (d->prec < 0 || d->prec > 2) return KF_ERR_ARG;
  if (d->solve_prec < 0 || d->solve_prec > 3) return KF_ERR_ARG;
  if ((d->solve_prec == KF_SOLVE_FP64_TC || d->solve_prec == KF_SOLVE_FP64_MEAN) && d->prec != KF_PREC_MIXED_BF16X3)
    return KF_ERR_ARG;
  if (d->q_kind < 0 || d->q_kind > 2 || d->r_kind < 0 || d->r_kind > 2) return KF_ERR_ARG;
  if (d->joseph_every < 0 || d->checkpoint_every < 0) return KF_ERR_ARG;
  if (d->split_terms != 0 && d->split_terms != 3 && d->split_terms != 6) return KF_ERR_ARG;
  return KF_OK;
}

kf_status choose_checkpoint(const kf_desc* d, const Sizes& z, int64_t* c_out, uint64_t* store_out) {
  const int64_t T = d->T;
  auto store_bytes = [&](int64_t c) -> uint64_t {
    if (c <= 1) return (uint64_t)(T + 1) * z.slot;
    return (uint64_t)(T / c + 1 + 1 + c - 1) * z.slot;
  };
  if (d->checkpoint_every > 0) {
    int64_t c = d->checkpoint_every > T ? T : d->checkpoint_every;
    if (c < 1) c = 1;
    *c_out = c;
    *store_out = store_bytes(c);
    if (d->mem_budget_bytes && z.workspace + *store_out > d->mem_budget_bytes) return KF_ERR_BUDGET;
    return KF_OK;
  }
  if (!d->mem_budget_bytes || z.workspace + store_bytes(1) <= d->mem_budget_bytes) {
    *c_out = 1;
    *store_out = store_bytes(1);
    return KF_OK;
  }
  int64_t best = -1;
  uint64_t best_bytes = 0;
  for (int64_t c = 2; c <= T; ++c) {
    uint64_t sbytes = store_bytes(c);
    if (best < 0 || sbytes < best_bytes) {
      best = c;
      best_bytes = sbytes;
    }
  }
  if (best < 0 || z.workspace + best_bytes > d->mem_budget_bytes) return KF_ERR_BUDGET;
  *c_out = best;
  *store_out = best_bytes;
  return KF_OK;
}

template <typename X>
kf_status dalloc(kf_plan_s* p, X** out, size_t bytes) {
  void* ptr = nullptr;
  if (bytes == 0) bytes = 16;
  ptr = arena_alloc(bytes);  // the reserved arena first (no device-wide synchronisation)
  cudaError_t e = ptr ? cudaSuccess : cudaMalloc(&ptr, bytes);
  if (e != cudaSuccess) {
    fprintf(stderr, "kfmeg: cudaMalloc(%zu) failed: %s\n", bytes, cudaGetErrorString(e));
    cudaGetLastError();
    return KF_ERR_CUDA;
  }
  p->allocs.push_back(ptr);
  KF_CUDA_TRY(cudaMemsetAsync(ptr, 0, bytes, p->s));
  *out = reinterpret_cast<X*>(ptr);
  return KF_OK;
}

// ------------------------------------------------------------ profiling

struct Prof {
  kf_plan_s* p;
  int cls;
  cudaEvent_t a = nullptr, b = nullptr;
  Prof(kf_plan_s* plan, int c) : p(plan), cls(c) {
    if (!p->prof) return;
    a = take();
    b = take();
    cudaEventRecord(a, p->s);
  }
  ~Prof() {
    if (!p->prof || !a) return;
    cudaEventRecord(b, p->s);
    p->marks.push_back({cls, a, b});
  }
  cudaEvent_t take() {
    if (!p->pool.empty()) {
      cudaEvent_t e = p->pool.back();
      p->pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
};

// Times the tensor-core kernel launches alone while installed (class cls): the split-bf16 kernel,
// or with exact = true the exact-slice kernel.
struct KernelTimer : TcLaunchTimer {
  kf_plan_s* p;
  int cls;
  bool exact;
  cudaEvent_t a = nullptr;
  KernelTimer(kf_plan_s* plan, int c, bool ex = false) : p(plan), cls(c), exact(ex) {
    if (p->prof) (exact ? g_oz_timer : g_tc_timer) = this;
  }
  ~KernelTimer() override {
    if (g_tc_timer == this) g_tc_timer = nullptr;
    if (g_oz_timer == this) g_oz_timer = nullptr;
  }
  cudaEvent_t take() {
    if (!p->pool.empty()) {
      cudaEvent_t e = p->pool.back();
      p->pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
  void before(cudaStream_t s) override {
    a = take();
    cudaEventRecord(a, s);
  }
  void after(cudaStream_t s) override {
    cudaEvent_t b = take();
    cudaEventRecord(b, s);
    p->marks.push_back({cls, a, b});
  }
};

// Times the exact-slice kernel launches alone while installed (class cls).
struct OzKernelTimer : KernelTimer {
  OzKernelTimer(kf_plan_s* plan, int c) : KernelTimer(plan, c, true) {}
};

// ------------------------------------------------------------ GEMM dispatch

// Bulk products: float64 / float32 on the CUDA cores, or split-bf16 on the
// tensor cores in the mixed mode (`slices` bf16 planes per operand: 2 for
// the smoother's covariance products by default, 3 where cancellation makes
// float32-class products necessary, as in the filter update P - K U).
template <typename B>
kf_status gemm_bulk(kf_plan_s* p, bool transB, const GemmParams<B>& g, int slices);

template <>
kf_status gemm_bulk<double>(kf_plan_s* p, bool transB, const GemmParams<double>& g, int) {
  return gemm_simt<double>(p->s, transB, g);
}

template <>
kf_status gemm_bulk<float>(kf_plan_s* p, bool transB, const GemmParams<float>& g, int slices) {
  if (p->bulk == BULK_BF16X3 && transB) return tc_gemm_split(p->s, p->tc, g, slices);
  return gemm_simt<float>(p->s, transB, g);
}

// ------------------------------------------------------------ predict

template <typename B>
kf_status predict_cov(kf_plan_s* p, const B* src, B* dst) {
  Prof pr(p, KF_KC_PREDICT);
  const int64_t N = p->N;
  if (p->d.f_kind == KF_F_IDENTITY)
    return add_cov<B, B>(p->s, dst, p->ldN, src, p->ldN, N, p->d.q_kind, p->Q);
  if (p->d.f_kind == KF_F_CSR)
    return spmm_fpft<B>(p->s, N, p->Frp, p->Fcol, p->F, src, p->ldN, (B*)p->tmpN, p->ldN, dst, p->ldN,
                        p->d.q_kind, p->Q);
  GemmParams<B> g;  // W = F src
  g.M = (int)N; g.N = (int)N; g.K = (int)N;
  g.A = (const B*)p->Fb; g.lda = p->ldN;
  g.B = src; g.ldb = p->ldN;
  g.out = (B*)p->tmpN; g.ldo = p->ldN;
  g.status = p->status;
  KF_TRY(gemm_simt<B>(p->s, false, g));
  GemmParams<B> h;  // dst = W F^T + Q
  h.M = (int)N; h.N = (int)N; h.K = (int)N;
  h.A = (const B*)p->tmpN; h.lda = p->ldN;
  h.B = (const B*)p->Fb; h.ldb = p->ldN;
  h.out2 = dst; h.ldo2 = p->ldN;
  h.q_kind = p->d.q_kind; h.q = p->Q; h.ldq = N;
  h.status = p->status;
  return gemm_simt<B>(p->s, true, h);
}

// ------------------------------------------------------------ filter step

// Covariance part of one filter step t (and the mean update when y != NULL):
// uses the working P = P_{t|t-1}, writes P_{t|t} to its store slot and
// leaves P_{t+1|t} in the working P.
// Block size of the m x m innovation Cholesky (float64): 32-wide leaves and
// panels.  Its float64 work is bound by the float64 pipe of the SMs it reaches,
// so smaller blocks (more parallel panel / trailing products, cheaper leaves)
// finish sooner than the 64-wide blocks used for large float64 matrices.
constexpr int kSBlock = 32;

template <typename B>
kf_status filter_step(kf_plan_s* p, int64_t t, const double* y, double* diag_out) {
  cudaStream_t s = p->s;
  const int N = (int)p->N, m = (int)p->m;
  const int64_t ldN = p->ldN, ldm = p->ldm, ldkv = 2 * p->ldm;
  B* P = (B*)p->P;
  B* Ut = (B*)p->Ut;
  B* KV = (B*)p->KV;
  {
    Prof pr(p, KF_KC_INNOVATION);
    GemmParams<B> g;  // U^T = P H^T  (N x m)
    g.M = N; g.N = m; g.K = N;
    g.A = P; g.lda = ldN;
    g.B = (const B*)p->Hb; g.ldb = ldN;
    g.out = Ut; g.ldo = ldm;
    g.status = p->status;
    KF_TRY(gemm_bulk<B>(p, true, g, 3));
  }
  // S = H U^T + R (float64), then its Cholesky factor in place
  KF_TRY((innovation_cov<B, B>(s, m, N, (const B*)p->Hb, p->ldN, Ut, ldm, p->d.r_kind, p->R, p->S, m, p->partials,
                               kSplitsS)));
  const bool joseph = p->d.joseph_every > 0 && (t % p->d.joseph_every) == 0;
  if (joseph) KF_CUDA_TRY(cudaMemcpyAsync(p->S0, p->S, (size_t)m * m * 8, cudaMemcpyDeviceToDevice, s));
  const int nbS = kSBlock;
  KF_TRY(potrf<double>(s, p->S, m, m, p->Sdinv, nbS, p->status, (int)t));
  const B* L = (const B*)p->S;
  const B* Ld = (const B*)p->Sdinv;
  if (sizeof(B) != sizeof(double)) {
    KF_TRY((copy2d<B, double>(s, (B*)p->Sl, m, p->S, m, m, m)));
    KF_TRY((copy2d<B, double>(s, (B*)p->Sldinv, nbS, p->Sdinv, nbS, round_up(m, nbS), nbS)));
    L = (const B*)p->Sl;
    Ld = (const B*)p->Sldinv;
  }
  // Square-root form of the gain: with S = L L^T, Z = U^T L^{-T} (N x m), so that
  // K = Z L^{-1}, K U = Z Z^T and K nu = Z (L^{-1} nu).  Z needs one triangular
  // solve and is conditioned like L (the square root of cond(S)); the m-sized
  // solve L^{-1} nu of the mean update runs in float64.
  B* Z = (B*)p->Zb;
  KF_TRY((copy2d<B, B>(s, Z, ldm, Ut, ldm, N, m)));
  KF_TRY(trsm_right<B>(s, true, N, m, L, m, Ld, nbS, Z, ldm, p->status));
  if (y) {
    KF_TRY(innovation(s, m, N, p->H, p->xpred + t * N, y, p->nu, p->status, (int)t));
    // nu <- L^{-1} nu  (as the 1 x m row solve nu^T L^{-T}), float64
    KF_TRY(trsm_right<double>(s, true, 1, m, p->S, m, p->Sdinv, nbS, p->nu, m, p->status));
    KF_TRY(gemv<B>(s, N, m, Z, ldm, p->nu, p->xpred + t * N, 1.0, p->xfilt + t * N));
  }
  const bool ident = p->d.f_kind == KF_F_IDENTITY;
  B* dst = (B*)p->slot_ptr(t);
  GemmParams<B> u;  // P_{t|t} = P - Z Z^T  (symmetric by construction), P <- P_{t|t} + Q when F = I
  u.M = N; u.N = N;
  u.A = Z; u.lda = ldm;
  u.alpha = B(-1);
  u.cin = P; u.ldcin = ldN; u.beta = B(1);
  u.out = dst; u.ldo = ldN;
  if (ident) {
    u.out2 = P; u.ldo2 = ldN;
    u.q_kind = p->d.q_kind; u.q = p->Q; u.ldq = N;
  }
  u.diag_out = diag_out;
  u.check_diag = 1;
  u.step = (int)t;
  u.status = p->status;
  u.sym = 1;
  if (joseph) {
    // Joseph form (I - KH) P (I - KH)^T + K R K^T = P - K V^T - V K^T with
    // K = Z L^{-1} and V = U^T - K S / 2: one rank-2m product [K V][V K]^T.
    KF_TRY((copy2d<B, B>(s, KV, ldkv, Z, ldm, N, m)));
    KF_TRY(trsm_right<B>(s, false, N, m, L, m, Ld, nbS, KV, ldkv, p->status));
    KF_TRY((copy2d<B, double>(s, (B*)p->S0b, m, p->S0, m, m, m)));
    GemmParams<B> v;
    v.M = N; v.N = m; v.K = m;
    v.A = KV; v.lda = ldkv;
    v.B = (const B*)p->S0b; v.ldb = m;
    v.alpha = B(-0.5);
    v.cin = Ut; v.ldcin = ldm; v.beta = B(1);
    v.out = KV + ldm; v.ldo = ldkv;
    v.status = p->status;
    KF_TRY(gemm_simt<B>(s, true, v));
    B* VK = (B*)p->VK;
    KF_TRY((copy2d<B, B>(s, VK, ldkv, KV + ldm, ldkv, N, m)));
    KF_TRY((copy2d<B, B>(s, VK + ldm, ldkv, KV, ldkv, N, m)));
    u.A = KV; u.lda = ldkv;
    u.K = (int)ldkv;
    u.B = VK; u.ldb = ldkv;
  } else {
    u.K = p->bulk == BULK_BF16X3 ? (int)ldm : m;
    u.B = Z; u.ldb = ldm;
  }
  {
    Prof pr(p, KF_KC_FILTER_UPDATE);
    KF_TRY(gemm_bulk<B>(p, true, u, 3));
  }
  if (!ident) KF_TRY(predict_cov<B>(p, dst, P));
  return KF_OK;
}

// F P F^T + Q for the float64 working covariance of the mixed mode, in place
// (P -> P_{t+1|t}).  The mesh coupling runs in float64 on the CUDA cores
// (HBM-bound); a dense F uses split-bf16 tensor-core products with a float64
// epilogue.
kf_status predict_cov64(kf_plan_s* p, double* P) {
  Prof pr(p, KF_KC_PREDICT);
  cudaStream_t s = p->s;
  const int N = (int)p->N;
  const int64_t ldN = p->ldN;
  if (p->d.f_kind == KF_F_IDENTITY) return add_cov<double, double>(s, P, ldN, P, ldN, N, p->d.q_kind, p->Q);
  if (p->d.f_kind == KF_F_CSR)
    return spmm_fpft<double>(s, N, p->Frp, p->Fcol, p->F, P, ldN, p->W64, ldN, P, ldN, p->d.q_kind, p->Q);
  GemmParams<double> w;  // W = F P
  w.M = N; w.N = N; w.K = N;
  w.out = p->W64; w.ldo = ldN;
  w.status = p->status;
  KF_TRY(tc_gemm_ops(s, p->tc, TcOperand{p->F, N, 1, 0}, TcOperand{P, ldN, 1, 1}, w, 3));
  GemmParams<double> h;  // P = W F^T + Q
  h.M = N; h.N = N; h.K = N;
  h.out2 = P; h.ldo2 = ldN;
  h.q_kind = p->d.q_kind; h.q = p->Q; h.ldq = N;
  h.status = p->status;
  return tc_gemm_ops(s, p->tc, TcOperand{p->W64, ldN, 1, 0}, TcOperand{p->F, N, 1, 0}, h, 3);
}

// One filter step of the mixed mode.  The working covariance P_{t|t-1} is
// kept in float64 (p->P64) and every product of the step is an exact-slice
// tensor-core product (5 slice levels: about 2^-37 of the operands' row
// maxima, far below float32 rounding) with a float64 epilogue: the filter
// runs at float64-class accuracy, which a long epoch needs because rounding
// errors of P in the directions the sensors do not see are never damped (F = I)
// and the mean integrates the resulting gain errors.  P_{t|t} is rounded to
// float32 only for the smoother's store.
//   U^T = P H^T (N x m) and U (m x N);  S = H U^T + R;  S = L L^T (float64);
//   Z = U^T L^{-T};  x += Z (L^{-1} nu);  P_{t|t} = P - Z Z^T (or Joseph form)
kf_status filter_step_mixed(kf_plan_s* p, int64_t t, const double* y, double* diag_out) {
  cudaStream_t s = p->s;
  const int N = (int)p->N, m = (int)p->m;
  const int64_t ldN = p->ldN, ldm = p->ldm, ldkv = 2 * p->ldm;
  const int LV = kOzLevels;
  double* P = p->P64;
  double* Ut = p->U64;
  {
    Prof pr(p, KF_KC_INNOVATION);
    KF_TRY(oz_slice(s, P, ldN, 1, N, N, LV, p->sP));
    OzEpilogue e;  // U^T = P H^T, and its transpose U
    e.out = Ut; e.ldo = ldm;
    e.outT = p->Um; e.ldoT = ldN;
    e.status = p->status; e.step = (int)t;
    KF_TRY(oz_gemm(s, p->sP, p->sH, N, m, N, LV, e));
  }
  {
    KF_TRY(oz_slice(s, p->Um, ldN, 1, m, N, LV, p->sU));
    OzEpilogue e;  // S = H U^T + R (exactly symmetric)
    e.out = p->S; e.ldo = m;
    e.radd_kind = p->d.r_kind; e.radd = p->R; e.ldradd = m;
    e.sym = 1;
    e.status = p->status; e.step = (int)t;
    KF_TRY(oz_gemm(s, p->sH, p->sU, m, m, N, LV, e, kOzSplitsS, p->ozpart));
  }
  const bool joseph = p->d.joseph_every > 0 && (t % p->d.joseph_every) == 0;
  if (joseph) KF_CUDA_TRY(cudaMemcpyAsync(p->S0, p->S, (size_t)m * m * 8, cudaMemcpyDeviceToDevice, s));
  const int nbS = kSBlock;
  KF_TRY(potrf<double>(s, p->S, m, m, p->Sdinv, nbS, p->status, (int)t));
  // L^{-1} = I L^{-1} (m x m, float64)
  KF_TRY(eye(s, m, p->Linv, m));
  KF_TRY(trsm_right<double>(s, false, m, m, p->S, m, p->Sdinv, nbS, p->Linv, m, p->status));
  double* Z = p->Z64;
  {
    KF_TRY(oz_slice(s, Ut, ldm, 1, N, m, LV, p->sUt));
    KF_TRY(oz_slice(s, p->Linv, m, 1, m, m, LV, p->sL));
    OzEpilogue e;  // Z = U^T L^{-T}:  Z[n][i] = sum_k U^T[n][k] L^{-1}[i][k]
    e.out = Z; e.ldo = ldm;
    e.status = p->status; e.step = (int)t;
    KF_TRY(oz_gemm(s, p->sUt, p->sL, N, m, m, LV, e));
  }
  if (y) {
    KF_TRY(innovation(s, m, N, p->H, p->xpred + t * N, y, p->nu, p->status, (int)t));
    KF_TRY(trsm_right<double>(s, true, 1, m, p->S, m, p->Sdinv, nbS, p->nu, m, p->status));
    KF_TRY(gemv<double>(s, N, m, Z, ldm, p->nu, p->xpred + t * N, 1.0, p->xfilt + t * N));
  }
  const bool ident = p->d.f_kind == KF_F_IDENTITY;
  OzEpilogue u;  // P_{t|t} = P - Z Z^T: float64 result, float32 copy to the store
  u.alpha = -1.0;
  u.cin = P; u.ldcin = ldN; u.beta = 1.0;
  u.outf = (float*)p->slot_ptr(t); u.ldof = ldN;
  if (ident) {
    u.out2 = P; u.ldo2 = ldN;
    u.q_kind = p->d.q_kind; u.q = p->Q; u.ldq = N;
  } else {
    u.out = P; u.ldo = ldN;
  }
  u.diag_out = diag_out;
  u.check_diag = 1;
  u.sym = 1;
  u.status = p->status; u.step = (int)t;
  Prof pr(p, KF_KC_FILTER_UPDATE);
  if (!joseph) {
    KF_TRY(oz_slice(s, Z, ldm, 1, N, m, LV, p->sZ));
    KF_TRY(oz_gemm(s, p->sZ, p->sZ, N, N, m, LV, u));
  } else {
    // Joseph form (I - KH) P (I - KH)^T + K R K^T = P - K V^T - V K^T with K = Z L^{-1} and
    // V = U^T - K S / 2: one rank-2m product [K V][V K]^T.
    double* KV = p->KV64;
    double* VK = p->VK64;
    KF_TRY(oz_slice(s, Z, ldm, 1, N, m, LV, p->sZ));
    KF_TRY(transpose(s, m, m, p->Linv, m, p->LinvT, m));
    KF_TRY(oz_slice(s, p->LinvT, m, 1, m, m, LV, p->sLT));
    OzEpilogue ek;  // K[n][i] = sum_k Z[n][k] L^{-1}[k][i]
    ek.out = KV; ek.ldo = ldkv;
    ek.status = p->status; ek.step = (int)t;
    KF_TRY(oz_gemm(s, p->sZ, p->sLT, N, m, m, LV, ek));
    KF_TRY(oz_slice(s, KV, ldkv, 1, N, m, LV, p->sK));
    KF_TRY(oz_slice(s, p->S0, m, 1, m, m, LV, p->sS0));
    OzEpilogue ev;  // V = U^T - K S / 2  (S symmetric: its rows are its columns)
    ev.alpha = -0.5;
    ev.cin = Ut; ev.ldcin = ldm; ev.beta = 1.0;
    ev.out = KV + ldm; ev.ldo = ldkv;
    ev.status = p->status; ev.step = (int)t;
    KF_TRY(oz_gemm(s, p->sK, p->sS0, N, m, m, LV, ev));
    KF_TRY((copy2d<double, double>(s, VK, ldkv, KV + ldm, ldkv, N, m)));
    KF_TRY((copy2d<double, double>(s, VK + ldm, ldkv, KV, ldkv, N, m)));
    KF_TRY(oz_slice(s, KV, ldkv, 1, N, ldkv, LV, p->sKV));
    KF_TRY(oz_slice(s, VK, ldkv, 1, N, ldkv, LV, p->sVK));
    KF_TRY(oz_gemm(s, p->sKV, p->sVK, N, N, (int)ldkv, LV, u));
  }
  if (!ident) KF_TRY(predict_cov64(p, P));
  return KF_OK;
}

// P_{1|0} = F P0 F^T + Q into the mixed filter's float64 working covariance.
kf_status predict_first64(kf_plan_s* p, const double* P0) {
  cudaStream_t s = p->s;
  const int N = (int)p->N;
  const int64_t ldN = p->ldN;
  double* P = p->P64;
  if (p->d.f_kind == KF_F_IDENTITY) return add_cov<double, double>(s, P, ldN, P0, N, N, p->d.q_kind, p->Q);
  if (p->d.f_kind == KF_F_CSR)
    return spmm_fpft<double>(s, N, p->Frp, p->Fcol, p->F, P0, N, p->W64, ldN, P, ldN, p->d.q_kind, p->Q);
  GemmParams<double> g;  // W = F P0, then P = W F^T + Q
  g.M = N; g.N = N; g.K = N;
  g.A = p->F; g.lda = N;
  g.B = P0; g.ldb = N;
  g.out = p->W64; g.ldo = ldN;
  KF_TRY(gemm_simt<double>(s, false, g));
  GemmParams<double> h;
  h.M = N; h.N = N; h.K = N;
  h.A = p->W64; h.lda = ldN;
  h.B = p->F; h.ldb = N;
  h.out2 = P; h.ldo2 = ldN;
  h.q_kind = p->d.q_kind; h.q = p->Q; h.ldq = N;
  return gemm_simt<double>(s, true, h);
}

// The first update in float64 for the float32 stores.  P0 is usually far
// above the posterior in the directions the sensors see (by 1 + lambda(H P0
// H^T) / r), so P_{1|1} = P_{1|0} - Z Z^T cancels most of its leading digits
// there; in float32 that cancellation leaves errors of order 1e-4 relative in
// the small eigenvalues, which the next steps carry.  From t = 2 on the
// prior is already close to the posterior and float32 is enough.  P_{1|1} is
// rounded to float32 only after the subtraction.
kf_status filter_first_fp64(kf_plan_s* p, const double* P0, const double* y, double* diag_out) {
  cudaStream_t s = p->s;
  const int N = (int)p->N, m = (int)p->m;
  const int64_t ldN = p->ldN, ldm = p->ldm;
  double* P = p->P64;
  if (p->d.f_kind == KF_F_IDENTITY) {
    KF_TRY((add_cov<double, double>(s, P, ldN, P0, N, N, p->d.q_kind, p->Q)));
  } else if (p->d.f_kind == KF_F_CSR) {
    KF_TRY(spmm_fpft<double>(s, N, p->Frp, p->Fcol, p->F, P0, N, p->W64, ldN, P, ldN, p->d.q_kind, p->Q));
  } else {
    GemmParams<double> g;  // W = F P0, then P = W F^T + Q
    g.M = N; g.N = N; g.K = N;
    g.A = p->F; g.lda = N;
    g.B = P0; g.ldb = N;
    g.out = p->W64; g.ldo = ldN;
    KF_TRY(gemm_simt<double>(s, false, g));
    GemmParams<double> h;
    h.M = N; h.N = N; h.K = N;
    h.A = p->W64; h.lda = ldN;
    h.B = p->F; h.ldb = N;
    h.out2 = P; h.ldo2 = ldN;
    h.q_kind = p->d.q_kind; h.q = p->Q; h.ldq = N;
    KF_TRY(gemm_simt<double>(s, true, h));
  }
  GemmParams<double> g;  // U^T = P H^T
  g.M = N; g.N = m; g.K = N;
  g.A = P; g.lda = ldN;
  g.B = p->H; g.ldb = N;
  g.out = p->U64; g.ldo = ldm;
  g.status = p->status;
  KF_TRY(gemm_simt<double>(s, true, g));
  KF_TRY((innovation_cov<double, double>(s, m, N, p->H, N, p->U64, ldm, p->d.r_kind, p->R, p->S, m, p->partials,
                                        kSplitsS)));
  const int nbS = kSBlock;
  KF_TRY(potrf<double>(s, p->S, m, m, p->Sdinv, nbS, p->status, 1));
  KF_TRY((copy2d<double, double>(s, p->Z64, ldm, p->U64, ldm, N, m)));
  KF_TRY(trsm_right<double>(s, true, N, m, p->S, m, p->Sdinv, nbS, p->Z64, ldm, p->status));
  KF_TRY(innovation(s, m, N, p->H, p->xpred + N, y, p->nu, p->status, 1));
  KF_TRY(trsm_right<double>(s, true, 1, m, p->S, m, p->Sdinv, nbS, p->nu, m, p->status));
  KF_TRY(gemv<double>(s, N, m, p->Z64, ldm, p->nu, p->xpred + N, 1.0, p->xfilt + N));
  GemmParams<double> u;  // P_{1|1} = P_{1|0} - Z Z^T
  u.M = N; u.N = N; u.K = m;
  u.A = p->Z64; u.lda = ldm;
  u.B = p->Z64; u.ldb = ldm;
  u.alpha = -1.0;
  u.cin = P; u.ldcin = ldN; u.beta = 1.0;
  u.out = P; u.ldo = ldN;
  u.diag_out = diag_out;
  u.check_diag = 1;
  u.step = 1;
  u.status = p->status;
  u.sym = 1;
  KF_TRY(gemm_simt<double>(s, true, u));
  float* dst = (float*)p->slot_ptr(1);
  KF_TRY((copy2d<float, double>(s, dst, ldN, P, ldN, N, N)));
  if (p->d.f_kind == KF_F_IDENTITY) return add_cov<float, double>(s, (float*)p->P, ldN, P, ldN, N, p->d.q_kind, p->Q);
  return predict_cov<float>(p, dst, (float*)p->P);
}

template <typename B>
kf_status recompute_segment(kf_plan_s* p, int64_t k) {
  const int64_t c = p->ckpt, t1 = std::min<int64_t>(k * c + c - 1, p->T);
  // segment 0 restarts from the kept P_{1|1}, the others from their checkpoint
  const int64_t t0 = k == 0 ? 1 : k * c;
  if (p->bulk == BULK_BF16X3) {
    KF_TRY((copy2d<double, float>(p->s, p->P64, p->ldN, (const float*)p->slot_ptr(t0), p->ldN, p->N, p->N)));
    KF_TRY(predict_cov64(p, p->P64));
    for (int64_t t = t0 + 1; t <= t1; ++t) KF_TRY(filter_step_mixed(p, t, nullptr, nullptr));
    p->seg_id = k;
    return KF_OK;
  }
  KF_TRY(predict_cov<B>(p, (const B*)p->slot_ptr(t0), (B*)p->P));
  for (int64_t t = t0 + 1; t <= t1; ++t) KF_TRY(filter_step<B>(p, t, nullptr, nullptr));
  p->seg_id = k;
  return KF_OK;
}

template <typename B>
kf_status get_P(kf_plan_s* p, int64_t t, const B** out) {
  if (p->ckpt > 1 && t % p->ckpt != 0 && t != 1 && p->seg_id != t / p->ckpt)
    KF_TRY(recompute_segment<B>(p, t / p->ckpt));
  *out = (const B*)p->slot_ptr(t);
  return KF_OK;
}

kf_status read_status(kf_plan_s* p, int64_t* fail_step) {
  KF_CUDA_TRY(cudaMemcpyAsync(p->status_h, p->status, ST_WORDS * sizeof(int), cudaMemcpyDeviceToHost, p->s));
  KF_CUDA_TRY(cudaStreamSynchronize(p->s));
  if (fail_step) *fail_step = p->status_h[ST_CODE] ? p->status_h[ST_STEP] : 0;
  return (kf_status)p->status_h[ST_CODE];
}

template <typename B>
kf_status run_filter(kf_plan_s* p, const double* Y, const double* x0, const double* P0, double* x_filt,
                     double* diagP_filt, int64_t* fail_step) {
  cudaStream_t s = p->s;
  const int64_t N = p->N, m = p->m, T = p->T;
  KF_CUDA_TRY(cudaMemsetAsync(p->status, 0, ST_WORDS * sizeof(int), s));
  KF_CUDA_TRY(cudaMemcpyAsync(p->xfilt, x0, N * 8, cudaMemcpyDeviceToDevice, s));
  // P0 into store slot 0 (bulk dtype), then P_{1|0}
  KF_TRY((copy2d<B, double>(s, (B*)p->slot_ptr(0), p->ldN, P0, N, N, N)));
  if (p->bulk == BULK_BF16X3) {
    KF_TRY(oz_slice(s, p->H, N, 1, m, N, kOzLevels, p->sH));  // the lead field's slices, once per epoch
    KF_TRY(predict_first64(p, P0));
  } else {
    KF_TRY(predict_cov<B>(p, (const B*)p->slot_ptr(0), (B*)p->P));
  }
  for (int64_t t = 1; t <= T; ++t) {
    KF_TRY(predict_mean(s, p->d.f_kind, N, p->F, p->Frp, p->Fcol, p->xfilt + (t - 1) * N, p->xpred + t * N));
    double* dg = diagP_filt ? diagP_filt + (t - 1) * N : nullptr;
    if (p->bulk == BULK_BF16X3)
      KF_TRY(filter_step_mixed(p, t, Y + (t - 1) * m, dg));
    else if (t == 1 && sizeof(B) == 4)
      KF_TRY(filter_first_fp64(p, P0, Y, dg));
    else
      KF_TRY(filter_step<B>(p, t, Y + (t - 1) * m, dg));
    if (p->ckpt > 1 && t % p->ckpt != 0) p->seg_id = t / p->ckpt;
  }
  KF_CUDA_TRY(cudaMemcpyAsync(x_filt, p->xfilt + N, (size_t)T * N * 8, cudaMemcpyDeviceToDevice, s));
  return read_status(p, fail_step);
}

// P_{t+1|t} = F P_{t|t} F^T + Q in float64 from the float32 stored P_{t|t} (Pn64), keeping F P_{t|t}
// in FP64 for non-identity F: the matrix every float64 smoother solve of the mixed path inverts,
// so that all of them compute the same J_t = P_{t|t} F^T P_{t+1|t}^{-1} (eqn 11).
kf_status predict_store64(kf_plan_s* p, const float* Pt) {
  cudaStream_t s = p->s;
  const int64_t N = p->N, ldN = p->ldN;
  if (p->d.f_kind == KF_F_IDENTITY)
    return add_cov<double, float>(s, p->Pn64, ldN, Pt, ldN, N, p->d.q_kind, p->Q);
  KF_TRY((copy2d<double, float>(s, p->W64, ldN, Pt, ldN, N, N)));  // float64 copy of P_{t|t}
  if (p->d.f_kind == KF_F_CSR)
    return spmm_fpft<double>(s, N, p->Frp, p->Fcol, p->F, p->W64, ldN, p->FP64, ldN, p->Pn64, ldN, p->d.q_kind,
                             p->Q);
  GemmParams<double> g;  // F P, then (F P) F^T + Q
  g.M = (int)N; g.N = (int)N; g.K = (int)N;
  g.A = p->F; g.lda = N;
  g.B = p->W64; g.ldb = ldN;
  g.out = p->FP64; g.ldo = ldN;
  KF_TRY(gemm_simt<double>(s, false, g));
  GemmParams<double> h;
  h.M = (int)N; h.N = (int)N; h.K = (int)N;
  h.A = p->FP64; h.lda = ldN;
  h.B = p->F; h.ldb = N;
  h.out2 = p->Pn64; h.ldo2 = ldN;
  h.q_kind = p->d.q_kind; h.q = p->Q; h.ldq = N;
  return gemm_simt<double>(s, true, h);
}

// Cholesky + inverse of the working P_{t+1|t} (in Lb) for smoother step `step`,
// replayed from a CUDA graph after the first step has run eagerly.
kf_status chol_inverse_step(kf_plan_s* p, float* Lb, int step) {
  const int N = (int)p->N;
  if (!p->chol_graph && p->cap_stream == nullptr) {
    // first use: run eagerly (also configures every kernel), then capture
    KF_TRY(chol_inverse_tc(p->s, p->tc, N, Lb, p->ldN, p->Wi, p->ldN, (float*)p->tmpN, p->ldN, p->status, step));
    if (cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      p->cap_stream = nullptr;
      return KF_OK;
    }
    const int64_t l0 = t_launches;
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      return KF_OK;
    }
    kf_status st = chol_inverse_tc(p->cap_stream, p->tc, N, Lb, p->ldN, p->Wi, p->ldN, (float*)p->tmpN, p->ldN,
                                   p->status, -1);
    cudaError_t e = cudaStreamEndCapture(p->cap_stream, &graph);
    if (st == KF_OK && e == cudaSuccess && graph &&
        cudaGraphInstantiate(&p->chol_graph, graph, 0) == cudaSuccess) {
      p->graph_launches = t_launches - l0;
    } else {
      p->chol_graph = nullptr;
    }
    g_launches -= t_launches - l0;  // the capture launched nothing
    t_launches = l0;
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return KF_OK;
  }
  if (!p->chol_graph)
    return chol_inverse_tc(p->s, p->tc, N, Lb, p->ldN, p->Wi, p->ldN, (float*)p->tmpN, p->ldN, p->status, step);
  KF_TRY(set_status_step(p->s, p->status, step));
  KF_CUDA_TRY(cudaGraphLaunch(p->chol_graph, p->s));
  note_launch(p->graph_launches);
  return KF_OK;
}

template <typename B, typename V>
kf_status run_smoother(kf_plan_s* p, double* x_smooth, double* diagP_smooth, double* P_full, int64_t t_full,
                       int64_t* fail_step) {
  cudaStream_t s = p->s;
  const int64_t N = p->N, T = p->T, ldN = p->ldN;
  const int nbs = potrf_block<V>();
  KF_CUDA_TRY(cudaMemsetAsync(p->status, 0, ST_WORDS * sizeof(int), s));
  B* Pn = (B*)p->Pn;
  B* Db = (B*)p->Db;
  B* Wb = (B*)p->Wb;
  V* Lb = (V*)p->Lb;
  V* Jb = (V*)p->Jb;
  B* Jm = sizeof(V) == sizeof(B) ? (B*)p->Jb : (B*)p->Jm;
  // a float64 solve in the mixed path: one float64 definition of P_{t+1|t} and of the mean (above)
  const bool fp64sv = p->bulk == BULK_BF16X3 && (sizeof(V) == 8 || p->refine || p->mean_refine);
  // t = T: smoothed = filtered
  KF_CUDA_TRY(cudaMemcpyAsync(p->xs + T * N, p->xfilt + T * N, N * 8, cudaMemcpyDeviceToDevice, s));
  const B* PT;
  if (T >= 2) {
    const B* Ptm1;
    KF_TRY(get_P<B>(p, T - 1, &Ptm1));
    KF_TRY(predict_cov<B>(p, Ptm1, Pn));
  }
  KF_TRY(get_P<B>(p, T, &PT));
  if (diagP_smooth) KF_TRY(diag_extract<B>(s, N, PT, ldN, diagP_smooth + (T - 1) * N));
  if (P_full && t_full == T) KF_TRY((copy2d<double, B>(s, P_full, N, PT, ldN, N, N)));
  if (T >= 2) {
    GemmParams<B> g;  // D_T = P_{T|T} - P_{T|T-1}  (K = 0 product: epilogue only)
    g.M = (int)N; g.N = (int)N; g.K = 0;
    g.cin = PT; g.ldcin = ldN; g.beta = B(1);
    g.csub = Pn; g.ldcsub = ldN;
    g.out = Db; g.ldo = ldN;
    g.sym = 1;
    g.status = p->status;
    KF_TRY(gemm_simt<B>(s, true, g));
  }
  for (int64_t t = T - 1; t >= 1; --t) {
    const B* Pt;
    {
      Prof pr(p, KF_KC_SMOOTH_SOLVE);
      KF_TRY(get_P<B>(p, t, &Pt));
      // P_{t+1|t} = L L^T: the bulk prediction, or for a float64 solve of the mixed path the
      // float64 prediction from the stored P_{t|t} (the float32 factor of the tensor-core solves is
      // then its float32 rounding, a preconditioner the refinement corrects)
      if (fp64sv) {
        KF_TRY(predict_store64(p, (const float*)Pt));
        KF_TRY((copy2d<V, double>(s, Lb, ldN, p->Pn64, ldN, N, N)));
      } else {
        KF_TRY((copy2d<V, B>(s, Lb, ldN, Pn, ldN, N, N)));
      }
      const bool tc_solve = p->bulk == BULK_BF16X3 && sizeof(V) == 4;
      {
        Prof pf(p, KF_KC_SOLVE_FACTOR);
        if (tc_solve)
          KF_TRY(chol_inverse_step(p, (float*)Lb, (int)(t + 1)));
        else
          KF_TRY(potrf<V>(s, Lb, ldN, (int)N, (V*)p->Ldinv, nbs, p->status, (int)(t + 1)));
      }
      // J_t = P_{t|t} F^T P_{t+1|t}^{-1}
      const B* Bm = Pt;
      if (p->d.f_kind == KF_F_CSR) {
        KF_TRY(spmm_pft<B>(s, N, p->Frp, p->Fcol, p->F, Pt, ldN, (B*)p->tmpN, ldN));
        Bm = (const B*)p->tmpN;
      } else if (p->d.f_kind == KF_F_DENSE) {
        GemmParams<B> f;
        f.M = (int)N; f.N = (int)N; f.K = (int)N;
        f.A = Pt; f.lda = ldN;
        f.B = (const B*)p->Fb; f.ldb = ldN;
        f.out = (B*)p->tmpN; f.ldo = ldN;
        f.status = p->status;
        KF_TRY(gemm_simt<B>(s, true, f));
        Bm = (const B*)p->tmpN;
      }
      Prof pg(p, KF_KC_SOLVE_GAIN);
      if (tc_solve && p->refine) {
        // float64-accurate P_{t+1|t}^{-1} from the float32-class factor; J_t in float64 (mean) and
        // float32 (covariance products)
        Prof pr(p, KF_KC_SOLVE_REFINE);
        OzKernelTimer kt(p, KF_KC_REFINE_EXACT_KERNEL);
        const bool ident = p->d.f_kind == KF_F_IDENTITY && p->d.q_kind != KF_COV_DENSE;
        KF_TRY(refine_inverse_tc(s, p->tc, (int)N, p->Pn64, 1, ldN, p->Wi, ldN, p->rb, p->d.q_kind,
                                 ident ? p->Q : nullptr, p->J64, (float*)Jb, ldN, p->rb.X0, ldN, p->status,
                                 (int)(t + 1)));
        if (!ident) {
          // J = (P_{t|t} F^T) X for the covariance products (X = P_{t+1|t}^{-1} symmetric: its rows are
          // its columns); the mean uses X itself below
          GemmParams<float> g;
          g.M = (int)N; g.N = (int)N; g.K = (int)N;
          g.out = (float*)Jb; g.ldo = ldN;
          g.status = p->status;
          KF_TRY(tc_gemm_ops(s, p->tc, TcOperand{Bm, ldN, 0, 0}, TcOperand{p->rb.X0, ldN, 1, 0}, g, 3));
        }
      } else if (tc_solve && p->mean_refine) {
        // the float32-class inverse X0 = W^T W: preconditioner of the mean's solve below and, for
        // F = I with a scalar or diagonal Q, the gain J = I - Q X0 of the covariance products
        GemmParams<float> g;
        g.M = (int)N; g.N = (int)N; g.K = (int)N;
        g.out = p->X0f; g.ldo = ldN;
        g.sym = 1;
        g.tri_a = -1;
        g.tri_b = -1;
        g.status = p->status;
        KF_TRY(tc_gemm_ops(s, p->tc, TcOperand{p->Wi, ldN, 0, 1}, TcOperand{p->Wi, ldN, 0, 1}, g, 3));
        if (p->d.f_kind == KF_F_IDENTITY && p->d.q_kind != KF_COV_DENSE) {
          KF_TRY(identity_minus_q(s, N, p->X0f, ldN, p->d.q_kind, p->Q, (float*)Jb, ldN));
        } else {
          if (Bm != Pt) {  // Bm lives in tmpN, which the products below use as scratch
            KF_TRY((copy2d<B, B>(s, (B*)Jb, ldN, Bm, ldN, N, N)));
            Bm = (const B*)Jb;
          }
          KF_TRY(gain_from_inverse_tc(s, p->tc, (int)N, (const float*)Bm, ldN, p->Wi, ldN, (float*)p->tmpN, ldN,
                                      (float*)Jb, ldN, p->status));
        }
      } else if (tc_solve && p->d.f_kind == KF_F_IDENTITY && p->d.q_kind != KF_COV_DENSE) {
        KF_TRY(gain_identity_tc(s, p->tc, (int)N, p->Wi, ldN, p->d.q_kind, p->Q, (float*)Jb, ldN, p->status));
      } else if (tc_solve) {
        if (Bm != Pt) {  // Bm lives in tmpN, which the products below use as scratch
          KF_TRY((copy2d<B, B>(s, (B*)Jb, ldN, Bm, ldN, N, N)));
          Bm = (const B*)Jb;
        }
        KF_TRY(gain_from_inverse_tc(s, p->tc, (int)N, (const float*)Bm, ldN, p->Wi, ldN, (float*)p->tmpN, ldN,
                                    (float*)Jb, ldN, p->status));
      } else {
        KF_TRY((copy2d<V, B>(s, Jb, ldN, Bm, ldN, N, N)));
        KF_TRY(trsm_right<V>(s, true, (int)N, (int)N, Lb, ldN, (const V*)p->Ldinv, nbs, Jb, ldN, p->status));
        KF_TRY(trsm_right<V>(s, false, (int)N, (int)N, Lb, ldN, (const V*)p->Ldinv, nbs, Jb, ldN, p->status));
      }
    }
    // x_{t|T} = x_{t|t} + J_t (x_{t+1|T} - x_{t+1|t})
    KF_TRY(vsub(s, N, p->xs + (t + 1) * N, p->xpred + (t + 1) * N, p->dx));
    if (!fp64sv) {
      KF_TRY(gemv<V>(s, N, N, Jb, ldN, p->dx, p->xfilt + t * N, 1.0, p->xs + t * N));
    } else if (p->refine && p->d.f_kind == KF_F_IDENTITY && p->d.q_kind != KF_COV_DENSE) {
      KF_TRY(gemv<double>(s, N, N, p->J64, ldN, p->dx, p->xfilt + t * N, 1.0, p->xs + t * N));
    } else {
      // x_{t|T} = x_{t|t} + P_{t|t} F^T y with y = P_{t+1|t}^{-1} dx to float64 accuracy
      double* y = p->ysol;
      if (sizeof(V) == 8) {  // float64 Cholesky factor: two triangular solves of the row vector dx
        KF_CUDA_TRY(cudaMemcpyAsync(y, p->dx, N * 8, cudaMemcpyDeviceToDevice, s));
        KF_TRY(trsm_right<double>(s, true, 1, (int)N, (const double*)Lb, ldN, (const double*)p->Ldinv, nbs, y, N,
                                  p->status));
        KF_TRY(trsm_right<double>(s, false, 1, (int)N, (const double*)Lb, ldN, (const double*)p->Ldinv, nbs, y, N,
                                  p->status));
      } else if (p->refine) {  // the float64-accurate inverse
        KF_TRY(gemv<double>(s, N, N, p->rb.X0, ldN, p->dx, nullptr, 1.0, y));
      } else {
        // iterative refinement: float64 residuals r = dx - P y, corrections y += X0 r with the
        // float32-class inverse (each step shrinks the error by |I - X0 P| ~ 1e-5)
        KF_TRY(gemv<float>(s, N, N, p->X0f, ldN, p->dx, nullptr, 1.0, y));
        for (int k = 0; k < 3; ++k) {
          KF_TRY(gemv<double>(s, N, N, p->Pn64, ldN, y, p->dx, -1.0, p->rsol));
          KF_TRY(gemv<float>(s, N, N, p->X0f, ldN, p->rsol, y, 1.0, y));
        }
      }
      if (p->d.f_kind == KF_F_IDENTITY)
        KF_TRY(gemv_f64acc(s, N, N, (const float*)Pt, ldN, y, p->xfilt + t * N, 1.0, p->xs + t * N));
      else  // P_{t|t} F^T y = (F P_{t|t})^T y
        KF_TRY(gemv_t(s, N, N, p->FP64, ldN, y, p->xfilt + t * N, 1.0, p->xs + t * N));
    }
    if ((void*)Jm != (void*)Jb) KF_TRY((copy2d<B, V>(s, Jm, ldN, Jb, ldN, N, N)));
    {
      Prof pr(p, KF_KC_SMOOTH_GEMM);
      KernelTimer kt(p, KF_KC_SMOOTH_GEMM_KERNEL);
      GemmParams<B> w;  // W = J_t D_{t+1}  (D symmetric)
      w.M = (int)N; w.N = (int)N; w.K = (int)N;
      w.A = Jm; w.lda = ldN;
      w.B = Db; w.ldb = ldN;
      w.out = Wb; w.ldo = ldN;
      w.status = p->status;
      KF_TRY(gemm_bulk<B>(p, true, w, p->smooth_slices));
    }
    const B* Ptm1;
    KF_TRY(get_P<B>(p, t - 1, &Ptm1));
    KF_TRY(predict_cov<B>(p, Ptm1, Pn));  // P_{t|t-1}
    {
      Prof pr(p, KF_KC_SMOOTH_GEMM);
      KernelTimer kt(p, KF_KC_SMOOTH_GEMM_KERNEL);
      GemmParams<B> g;  // D_t = P_{t|t} + W J_t^T - P_{t|t-1};  diag(P_{t|T}) out
      g.M = (int)N; g.N = (int)N; g.K = (int)N;
      g.A = Wb; g.lda = ldN;
      g.B = Jm; g.ldb = ldN;
      g.cin = Pt; g.ldcin = ldN; g.beta = B(1);
      g.csub = Pn; g.ldcsub = ldN;
      g.out = Db; g.ldo = ldN;
      if (P_full && t_full == t) {
        g.out2 = (B*)p->tmpN; g.ldo2 = ldN;
      }
      g.diag_out = diagP_smooth ? diagP_smooth + (t - 1) * N : nullptr;
      g.check_diag = 1;
      g.step = (int)t;
      g.sym = 1;
      g.status = p->status;
      KF_TRY(gemm_bulk<B>(p, true, g, p->smooth_slices));
    }
    if (P_full && t_full == t) KF_TRY((copy2d<double, B>(s, P_full, N, (const B*)p->tmpN, ldN, N, N)));
  }
  KF_CUDA_TRY(cudaMemcpyAsync(x_smooth, p->xs + N, (size_t)T * N * 8, cudaMemcpyDeviceToDevice, s));
  return read_status(p, fail_step);
}

kf_status copy_inputs(kf_plan_s* p, const double* F, const int64_t* rp, const int64_t* col, const double* Q,
                      const double* H, const double* R) {
  cudaStream_t s = p->s;
  const int64_t N = p->N, m = p->m;
  if (p->d.f_kind == KF_F_CSR) {
    KF_CUDA_TRY(cudaMemcpyAsync(p->F, F, p->d.f_nnz * 8, cudaMemcpyDeviceToDevice, s));
    KF_CUDA_TRY(cudaMemcpyAsync(p->Frp, rp, (N + 1) * 8, cudaMemcpyDeviceToDevice, s));
    KF_CUDA_TRY(cudaMemcpyAsync(p->Fcol, col, p->d.f_nnz * 8, cudaMemcpyDeviceToDevice, s));
  } else if (p->d.f_kind == KF_F_DENSE) {
    KF_CUDA_TRY(cudaMemcpyAsync(p->F, F, (size_t)N * N * 8, cudaMemcpyDeviceToDevice, s));
    if (p->b == 8)
      KF_TRY((copy2d<double, double>(s, (double*)p->Fb, p->ldN, F, N, N, N)));
    else
      KF_TRY((copy2d<float, double>(s, (float*)p->Fb, p->ldN, F, N, N, N)));
  }
  KF_CUDA_TRY(cudaMemcpyAsync(p->Q, Q, cov_count(p->d.q_kind, N) * 8, cudaMemcpyDeviceToDevice, s));
  KF_CUDA_TRY(cudaMemcpyAsync(p->H, H, (size_t)m * N * 8, cudaMemcpyDeviceToDevice, s));
  KF_CUDA_TRY(cudaMemcpyAsync(p->R, R, cov_count(p->d.r_kind, m) * 8, cudaMemcpyDeviceToDevice, s));
  if (p->b == 8)
    KF_TRY((copy2d<double, double>(s, (double*)p->Hb, p->ldN, H, N, m, N, true)));
  else
    KF_TRY((copy2d<float, double>(s, (float*)p->Hb, p->ldN, H, N, m, N, true)));
  return KF_OK;
}

}  // namespace

// =================================================================== C ABI

extern "C" {

kf_status kf_plan_footprint(const kf_desc* d, uint64_t* workspace_bytes, uint64_t* store_bytes,
                            int32_t* checkpoint_every) {
  KF_TRY(validate(d));
  Sizes z = sizes_for(d);
  int64_t c = 1;
  uint64_t sbytes = 0;
  kf_status st = choose_checkpoint(d, z, &c, &sbytes);
  if (workspace_bytes) *workspace_bytes = z.workspace;
  if (store_bytes) *store_bytes = sbytes;
  if (checkpoint_every) *checkpoint_every = (int32_t)c;
  return st;
}

kf_status kf_plan(kf_plan_t* out, const kf_desc* d) {
  if (!out) return KF_ERR_ARG;
  KF_TRY(validate(d));
  if (d->prec == KF_PREC_MIXED_BF16X3 && !tc_available()) return KF_ERR_UNSUPPORTED;
  Sizes z = sizes_for(d);
  int64_t c = 1;
  uint64_t store_bytes = 0;
  KF_TRY(choose_checkpoint(d, z, &c, &store_bytes));

  kf_plan_s* p = new kf_plan_s();
  p->d = *d;
  p->s = (cudaStream_t)d->stream;
  p->N = d->N; p->m = d->m; p->T = d->T;
  p->ldN = z.ldN; p->ldm = z.ldm;
  p->b = z.b; p->sb = z.sb;
  p->bulk = d->prec == KF_PREC_FP64 ? BULK_F64 : d->prec == KF_PREC_FP32 ? BULK_F32 : BULK_BF16X3;
  p->solve = z.sb == 8 ? 0 : 1;
  p->refine = d->solve_prec == KF_SOLVE_FP64_TC;
  p->mean_refine = d->solve_prec == KF_SOLVE_FP64_MEAN;
  p->smooth_slices = d->split_terms == 6 ? 3 : 2;
  p->slot = z.slot;
  p->ckpt = c;
  const int64_t N = p->N, m = p->m, T = p->T, ldN = p->ldN, ldm = p->ldm;
  const size_t b = p->b, sb = p->sb;
  kf_status st = KF_OK;
  auto A = [&](auto** ptr, size_t bytes) {
    if (st == KF_OK) st = dalloc(p, ptr, bytes);
  };
  A(&p->store, store_bytes - (c > 1 ? (size_t)(c - 1) * p->slot : 0));  // checkpoints (+ the t = 1 slot)
  if (c > 1) A(&p->seg, (size_t)(c - 1) * p->slot);
  p->nck = c > 1 ? T / c + 1 : T + 1;
  A(&p->xpred, (T + 1) * N * 8);
  A(&p->xfilt, (T + 1) * N * 8);
  A(&p->xs, (T + 1) * N * 8);
  A(&p->nu, m * 8);
  A(&p->dx, N * 8);
  A(&p->P, p->slot);
  A(&p->tmpN, p->slot);
  A(&p->Ut, N * ldm * b);
  A(&p->Zb, N * ldm * b);
  A(&p->KV, N * 2 * ldm * b);
  A(&p->VK, N * 2 * ldm * b);
  A(&p->Hb, m * ldN * b);
  A(&p->S, m * m * 8);
  A(&p->S0, m * m * 8);
  A(&p->Sdinv, round_up(m, 64) * 64 * 8);
  A(&p->partials, kSplitsS * m * m * 8);
  A(&p->Sl, m * m * b);
  A(&p->Sldinv, round_up(m, 64) * 64 * b);
  A(&p->S0b, m * m * b);
  const int64_t nbs = sb == 8 ? 64 : 128;
  A(&p->Lb, N * ldN * sb);
  A(&p->Jb, N * ldN * sb);
  A(&p->Ldinv, round_up(N, nbs) * nbs * sb);
  if (sb != b) A(&p->Jm, p->slot);
  if (p->bulk == BULK_BF16X3 && sb == 4) A(&p->Wi, p->slot);
  if (p->mean_refine) A(&p->X0f, p->slot);
  if (p->bulk == BULK_BF16X3 && d->solve_prec != KF_SOLVE_FP32) {
    A(&p->Pn64, N * ldN * 8);
    if (d->f_kind != KF_F_IDENTITY) A(&p->FP64, N * ldN * 8);
    A(&p->ysol, N * 8);
    A(&p->rsol, N * 8);
    A(&p->wsol, N * 8);
  }
  if (p->refine) {
    char* rm = nullptr;
    A(&rm, refine_bytes(N, ldN));
    if (st == KF_OK) refine_layout(p->rb, rm, N, ldN);
    A(&p->J64, N * ldN * 8);
  }
  if (b == 4) {
    A(&p->P64, N * ldN * 8);
    if (d->f_kind != KF_F_IDENTITY) A(&p->W64, N * ldN * 8);
    A(&p->U64, N * ldm * 8);
    A(&p->Z64, N * ldm * 8);
  }
  if (p->bulk == BULK_BF16X3) {
    A(&p->Um, m * ldN * 8);
    A(&p->Linv, m * m * 8);
    A(&p->LinvT, m * m * 8);
    A(&p->ozpart, kOzSplitsS * m * m * 8);
    if (d->joseph_every > 0) {
      A(&p->KV64, N * 2 * ldm * 8);
      A(&p->VK64, N * 2 * ldm * 8);
    }
    auto AS = [&](OzSlices& sl, int64_t rows, int64_t cols) {
      char* mem = nullptr;
      A(&mem, oz_slice_bytes(rows, cols, kOzLevels));
      if (st == KF_OK) oz_slice_layout(sl, mem, rows, cols, kOzLevels);
    };
    AS(p->sP, N, N);
    AS(p->sH, m, N);
    AS(p->sU, m, N);
    AS(p->sUt, N, m);
    AS(p->sZ, N, m);
    AS(p->sK, N, m);
    AS(p->sL, m, m);
    AS(p->sLT, m, m);
    AS(p->sS0, m, m);
    if (d->joseph_every > 0) {
      AS(p->sKV, N, 2 * ldm);
      AS(p->sVK, N, 2 * ldm);
    }
  }
  A(&p->Wb, p->slot);
  A(&p->Db, p->slot);
  A(&p->Pn, p->slot);
  if (d->f_kind == KF_F_CSR) {
    A(&p->F, d->f_nnz * 8);
    A(&p->Fcol, d->f_nnz * 8);
    A(&p->Frp, (N + 1) * 8);
  } else if (d->f_kind == KF_F_DENSE) {
    A(&p->F, N * N * 8);
    A(&p->Fb, p->slot);
  }
  A(&p->Q, cov_count(d->q_kind, N) * 8);
  A(&p->H, m * N * 8);
  A(&p->R, cov_count(d->r_kind, m) * 8);
  A(&p->status, ST_WORDS * sizeof(int));
  if (st == KF_OK && p->bulk == BULK_BF16X3) st = tc_scratch_alloc(p->tc, std::max(N, m), std::max(ldN, 2 * ldm), [&](void** ptr, size_t bytes) {
    return dalloc(p, (char**)ptr, bytes);
  });
  if (st == KF_OK && cudaStreamSynchronize(p->s) != cudaSuccess) st = KF_ERR_CUDA;
  if (st != KF_OK) {
    kf_plan_destroy(p);
    return st;
  }
  *out = p;
  return KF_OK;
}

kf_status kf_filter(kf_plan_t p, const double* F, const int64_t* F_rowptr, const int64_t* F_col,
                    const double* Q, const double* H, const double* R, const double* Y, const double* x0,
                    const double* P0, double* x_filt, double* diagP_filt, int64_t* fail_step) {
  if (fail_step) *fail_step = 0;
  if (!p || !Q || !H || !R || !Y || !x0 || !P0 || !x_filt) return KF_ERR_ARG;
  if (p->d.f_kind != KF_F_IDENTITY && !F) return KF_ERR_ARG;
  if (p->d.f_kind == KF_F_CSR && (!F_rowptr || !F_col)) return KF_ERR_ARG;
  p->filtered = false;
  const int64_t l0 = t_launches;
  kf_status st = copy_inputs(p, F, F_rowptr, F_col, Q, H, R);
  if (st == KF_OK)
    st = p->b == 8 ? run_filter<double>(p, Y, x0, P0, x_filt, diagP_filt, fail_step)
                   : run_filter<float>(p, Y, x0, P0, x_filt, diagP_filt, fail_step);
  p->launches += t_launches - l0;
  p->filtered = st == KF_OK;
  return st;
}

kf_status fis_smooth(kf_plan_t p, double* x_smooth, double* diagP_smooth, double* P_smooth_at, int64_t t_full,
                     int64_t* fail_step) {
  if (fail_step) *fail_step = 0;
  if (!p || !x_smooth) return KF_ERR_ARG;
  if (P_smooth_at && (t_full < 1 || t_full > p->T)) return KF_ERR_ARG;
  if (!p->filtered) return KF_ERR_STATE;
  const int64_t l0 = t_launches;
  kf_status st;
  if (p->b == 8)
    st = run_smoother<double, double>(p, x_smooth, diagP_smooth, P_smooth_at, t_full, fail_step);
  else if (p->sb == 8)
    st = run_smoother<float, double>(p, x_smooth, diagP_smooth, P_smooth_at, t_full, fail_step);
  else
    st = run_smoother<float, float>(p, x_smooth, diagP_smooth, P_smooth_at, t_full, fail_step);
  p->launches += t_launches - l0;
  return st;
}

kf_status kf_solve_host(kf_plan_t p, const double* F, const int64_t* F_rowptr, const int64_t* F_col,
                        const double* Q, const double* H, const double* R, const double* Y, const double* x0,
                        const double* P0, double* x_filt, double* diagP_filt, double* x_smooth,
                        double* diagP_smooth, int64_t* fail_step) {
  if (!p || !Q || !H || !R || !Y || !x0 || !P0) return KF_ERR_ARG;
  const int64_t N = p->N, m = p->m, T = p->T;
  cudaStream_t s = p->s;
  kf_status st = KF_OK;
  auto A = [&](auto** ptr, size_t bytes) {
    if (st == KF_OK && *ptr == nullptr) st = dalloc(p, ptr, bytes);
  };
  A(&p->hY, T * m * 8);
  A(&p->hx0, N * 8);
  A(&p->hP0, N * N * 8);
  A(&p->hQ, cov_count(p->d.q_kind, N) * 8);
  A(&p->hH, m * N * 8);
  A(&p->hR, cov_count(p->d.r_kind, m) * 8);
  A(&p->hxf, T * N * 8);
  A(&p->hdf, T * N * 8);
  A(&p->hxs, T * N * 8);
  A(&p->hds, T * N * 8);
  if (p->d.f_kind == KF_F_CSR) {
    A(&p->hF, p->d.f_nnz * 8);
    A(&p->hFcol, p->d.f_nnz * 8);
    A(&p->hFrp, (N + 1) * 8);
  } else if (p->d.f_kind == KF_F_DENSE) {
    A(&p->hF, N * N * 8);
  }
  KF_TRY(st);
  auto H2D = [&](void* dst, const void* src, size_t bytes) {
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
  };
  KF_CUDA_TRY(H2D(p->hY, Y, T * m * 8));
  KF_CUDA_TRY(H2D(p->hx0, x0, N * 8));
  KF_CUDA_TRY(H2D(p->hP0, P0, N * N * 8));
  KF_CUDA_TRY(H2D(p->hQ, Q, cov_count(p->d.q_kind, N) * 8));
  KF_CUDA_TRY(H2D(p->hH, H, m * N * 8));
  KF_CUDA_TRY(H2D(p->hR, R, cov_count(p->d.r_kind, m) * 8));
  if (p->d.f_kind == KF_F_CSR) {
    if (!F || !F_rowptr || !F_col) return KF_ERR_ARG;
    KF_CUDA_TRY(H2D(p->hF, F, p->d.f_nnz * 8));
    KF_CUDA_TRY(H2D(p->hFcol, F_col, p->d.f_nnz * 8));
    KF_CUDA_TRY(H2D(p->hFrp, F_rowptr, (N + 1) * 8));
  } else if (p->d.f_kind == KF_F_DENSE) {
    if (!F) return KF_ERR_ARG;
    KF_CUDA_TRY(H2D(p->hF, F, N * N * 8));
  }
  KF_TRY(kf_filter(p, p->hF, p->hFrp, p->hFcol, p->hQ, p->hH, p->hR, p->hY, p->hx0, p->hP0, p->hxf, p->hdf,
                   fail_step));
  KF_TRY(fis_smooth(p, p->hxs, p->hds, nullptr, -1, fail_step));
  auto D2H = [&](void* dst, const void* src, size_t bytes) {
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s);
  };
  if (x_filt) KF_CUDA_TRY(D2H(x_filt, p->hxf, T * N * 8));
  if (diagP_filt) KF_CUDA_TRY(D2H(diagP_filt, p->hdf, T * N * 8));
  if (x_smooth) KF_CUDA_TRY(D2H(x_smooth, p->hxs, T * N * 8));
  if (diagP_smooth) KF_CUDA_TRY(D2H(diagP_smooth, p->hds, T * N * 8));
  KF_CUDA_TRY(cudaStreamSynchronize(s));
  return KF_OK;
}

kf_status kf_plan_profile(kf_plan_t p, int32_t enable) {
  if (!p) return KF_ERR_ARG;
  KF_CUDA_TRY(cudaStreamSynchronize(p->s));
  for (auto& mk : p->marks) {
    p->pool.push_back(mk.a);
    p->pool.push_back(mk.b);
  }
  p->marks.clear();
  p->prof = enable != 0;
  return KF_OK;
}

kf_status kf_plan_profile_read(kf_plan_t p, int32_t cls, int64_t* launches, double* total_ms) {
  if (!p || cls < 0 || cls >= KF_KC_COUNT) return KF_ERR_ARG;
  KF_CUDA_TRY(cudaStreamSynchronize(p->s));
  int64_t n = 0;
  double ms = 0.0;
  for (auto& mk : p->marks) {
    if (mk.cls != cls) continue;
    float f = 0.f;
    KF_CUDA_TRY(cudaEventElapsedTime(&f, mk.a, mk.b));
    ms += f;
    ++n;
  }
  if (launches) *launches = n;
  if (total_ms) *total_ms = ms;
  return KF_OK;
}

int64_t kf_plan_launch_count(kf_plan_t p) { return p ? p->launches : 0; }

void kf_plan_destroy(kf_plan_t p) {
  if (!p) return;
  if (p->s) cudaStreamSynchronize(p->s);
  if (p->chol_graph) cudaGraphExecDestroy(p->chol_graph);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  for (void* a : p->allocs) {
    if (arena_owns(a))
      arena_free(a);
    else
      cudaFree(a);
  }
  for (auto& mk : p->marks) {
    cudaEventDestroy(mk.a);
    cudaEventDestroy(mk.b);
  }
  for (auto e : p->pool) cudaEventDestroy(e);
  delete p;
}

const char* kf_strerror(kf_status s) {
  switch (s) {
    case KF_OK: return "ok";
    case KF_ERR_ARG: return "invalid argument";
    case KF_ERR_NOT_PD: return "matrix not positive definite";
    case KF_ERR_BUDGET: return "covariance store does not fit the memory budget";
    case KF_ERR_CUDA: return "CUDA runtime error";
    case KF_ERR_NUMERIC: return "non-finite value or non-positive variance";
    case KF_ERR_TIMEOUT: return "bounded device wait expired";
    case KF_ERR_STATE: return "call order violated (fis_smooth needs a successful kf_filter)";
    case KF_ERR_UNSUPPORTED: return "unsupported by the compiled library";
  }
  return "unknown status";
}

}  // extern "C"
