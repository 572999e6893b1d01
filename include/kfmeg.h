/*
 * kfmeg — Kalman filter + fixed-interval smoother for the dynamic MEG inverse
 * problem (Long et al., Ann. Appl. Stat. 2011), as a C ABI over hand-written
 * sm_103a CUDA kernels.
 *
 * Model (Sec. 2, eqns 1 and 3):   x_t = F x_{t-1} + v_t,  v_t ~ N(0, Q)
 *                                 y_t = H x_t + e_t,      e_t ~ N(0, R)
 * with N sources (state dimension), m sensors and T time steps.  The paper's
 * P (sources), S (sensors) and N (time points) are N, m and T here; its
 * W (state covariance), Sigma_w, Sigma_eps and smoother gain A_k are P, Q, R
 * and J_t.
 *
 * Conventions shared by every entry point unless stated otherwise:
 *  - Array arguments are DEVICE pointers to row-major, contiguous float64
 *    buffers owned by the caller.  The plan owns its workspace and covariance
 *    store and frees them in kf_plan_destroy.
 *  - Inputs are float64 in every precision mode; the mode changes only the
 *    internal arithmetic and the dtype of the stored covariances.
 *  - Work is enqueued on the stream given in the descriptor (a cudaStream_t,
 *    NULL = legacy default stream).  kf_filter and fis_smooth synchronise that
 *    stream once at their end to read the device status word.
 *  - Covariance kinds: KF_COV_SCALAR = one value v (cov = v I),
 *    KF_COV_DIAG = a vector of the diagonal, KF_COV_DENSE = full matrix.
 *  - Errors never fault the GPU: kernels that meet a non-positive pivot or a
 *    non-finite value set a device status word and later kernels skip their
 *    work; the host maps it to a kf_status.
 */
#ifndef KFMEG_H
#define KFMEG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kf_plan_s* kf_plan_t;

typedef enum {
  KF_OK = 0,
  KF_ERR_ARG = 1,          /* bad argument (sizes, kinds, NULL where required)     */
  KF_ERR_NOT_PD = 2,       /* S or P_{t+1|t} not positive definite; see fail_step  */
  KF_ERR_BUDGET = 3,       /* store cannot fit the memory budget even checkpointed */
  KF_ERR_CUDA = 4,         /* a CUDA runtime call failed (incl. out of memory)     */
  KF_ERR_NUMERIC = 5,      /* NaN/Inf in data or a non-positive covariance diagonal */
  KF_ERR_TIMEOUT = 6,      /* a bounded device wait expired                        */
  KF_ERR_STATE = 7,        /* call order violated (fis_smooth before kf_filter)    */
  KF_ERR_UNSUPPORTED = 8   /* combination the compiled library does not provide    */
} kf_status;

typedef enum { KF_F_IDENTITY = 0, KF_F_CSR = 1, KF_F_DENSE = 2 } kf_f_kind;

/* Arithmetic of the bulk N x N products (predict, innovation, update, the
 * smoother's J D J^T) and dtype of the covariance store. */
typedef enum {
  KF_PREC_FP64 = 0,          /* float64 everywhere                                   */
  KF_PREC_FP32 = 1,          /* float32 products, float32 store                      */
  KF_PREC_MIXED_BF16X3 = 2   /* split-bf16 tensor-core products, fp32 accumulate,    */
                             /* float32 store: the smoother's N x N covariance       */
                             /* products as hi*hi + hi*lo + lo*hi (see split_terms), */
                             /* the filter's products with a three-way split         */
} kf_precision;

/* Arithmetic of the smoother-gain solve J_t = P_{t|t} F^T P_{t+1|t}^{-1}
 * (eqn 11: Cholesky of P_{t+1|t} and two triangular solves, or the inverse). */
typedef enum {
  KF_SOLVE_FP64 = 0,         /* float64 Cholesky and triangular solves on the CUDA   */
                             /* cores                                                */
  KF_SOLVE_FP32 = 1,         /* float32 class: float32 factor (split-bf16 tensor-core */
                             /* products in KF_PREC_MIXED_BF16X3)                    */
  KF_SOLVE_FP64_TC = 2,      /* float64 accuracy on the tensor cores (needs          */
                             /* KF_PREC_MIXED_BF16X3): the float32-class inverse of  */
                             /* P_{t+1|t} refined by two Newton steps whose residuals */
                             /* I - P X are exact-slice products (kfx_spd_inverse    */
                             /* mode 2); J_t in float64 for the smoothed mean        */
  KF_SOLVE_FP64_MEAN = 3     /* needs KF_PREC_MIXED_BF16X3: the smoothed mean's solve */
                             /* y = P_{t+1|t}^{-1} d (eqn 12) refined to float64     */
                             /* accuracy (float64 residuals d - P y, the float32-    */
                             /* class inverse as preconditioner, three steps),       */
                             /* x_{t|T} = x_{t|t} + P_{t|t} F^T y; J_t inside the     */
                             /* split-bf16 covariance product of eqn 13 from the     */
                             /* float32-class inverse                                */
} kf_solve_precision;
/* In KF_PREC_MIXED_BF16X3 every float64 solve (FP64, FP64_TC, FP64_MEAN) inverts the same
 * P_{t+1|t} = F P_{t|t} F^T + Q, formed in float64 from the float32 stored P_{t|t}, and their
 * smoothed means agree to float64 rounding times the conditioning. */

typedef enum { KF_COV_SCALAR = 0, KF_COV_DIAG = 1, KF_COV_DENSE = 2 } kf_cov_kind;

typedef struct {
  int64_t N;                 /* sources (state dimension), >= 1                      */
  int64_t m;                 /* sensors, >= 1                                        */
  int64_t T;                 /* time steps, >= 1                                     */
  int32_t f_kind;            /* kf_f_kind                                            */
  int32_t prec;              /* kf_precision                                         */
  int32_t solve_prec;        /* kf_solve_precision                                   */
  int32_t q_kind;            /* kf_cov_kind of Q                                     */
  int32_t r_kind;            /* kf_cov_kind of R                                     */
  int32_t joseph_every;      /* 0 = never; k = Joseph-form covariance update every   */
                             /* k-th step (others use P - K H P, symmetrised)        */
  int64_t f_nnz;             /* non-zeros of F when f_kind == KF_F_CSR               */
  uint64_t mem_budget_bytes; /* cap on plan-owned device memory; 0 = no cap          */
  int32_t checkpoint_every;  /* 0 = chosen from the budget; c > 0 forces keeping     */
                             /* every c-th P_{t|t} and recomputing the rest          */
  int32_t split_terms;       /* KF_PREC_MIXED_BF16X3 only: bf16 products per product */
                             /* in the smoother's covariance GEMMs, 3 (hi/lo split,  */
                             /* default when 0) or 6 (three-way split, float32-class) */
  void* stream;              /* cudaStream_t for all work of this plan               */
} kf_desc;

/* Sizes a plan would allocate for descriptor d, without allocating.
 * workspace_bytes: working buffers; store_bytes: covariance store;
 * checkpoint_every: 1 = every P_{t|t} is stored, c > 1 = every c-th is stored
 * and the others are recomputed forward during fis_smooth.
 * Returns KF_ERR_BUDGET if even checkpointing cannot fit mem_budget_bytes. */
kf_status kf_plan_footprint(const kf_desc* d, uint64_t* workspace_bytes,
                            uint64_t* store_bytes, int32_t* checkpoint_every);

/* Validates d and allocates the workspace and the covariance store on the
 * current CUDA device.  *out is set only on KF_OK. */
kf_status kf_plan(kf_plan_t* out, const kf_desc* d);

/* Forward pass, eqns 6-10 (Sec. 2.2), for t = 1..T:
 *   x_{t|t-1} = F x_{t-1|t-1},  P_{t|t-1} = F P_{t-1|t-1} F^T + Q   (eqns 6-7)
 *   S_t = H P_{t|t-1} H^T + R,  S_t = L L^T (float64 Cholesky)      (eqn 8)
 *   K_t = P_{t|t-1} H^T S_t^{-1}                                     (eqn 8)
 *   x_{t|t} = x_{t|t-1} + K_t (y_t - H x_{t|t-1})                    (eqn 10)
 *   P_{t|t} = (I - K_t H) P_{t|t-1}, stored symmetric                (eqn 10)
 * (x0, P0) describe the state at t = 0; step 1 predicts, then updates with Y[0].
 *   F:        f_kind IDENTITY: NULL; CSR: the f_nnz values; DENSE: N x N.
 *   F_rowptr: CSR only, N+1 int64 offsets; F_col: CSR only, f_nnz int64 columns.
 *   Q: per q_kind (1, N or N x N values); H: m x N; R: per r_kind (1, m or m x m);
 *   Y: T x m (row t-1 is y_t); x0: N; P0: N x N symmetric positive definite.
 *   x_filt: T x N output (row t-1 is x_{t|t}).
 *   diagP_filt: T x N output of diag(P_{t|t}), or NULL.
 *   fail_step: if not NULL, receives the 1-based step of a KF_ERR_NOT_PD /
 *              KF_ERR_NUMERIC failure (0 otherwise).
 * The plan keeps P_{t|t} (or checkpoints of it) and the means for fis_smooth. */
kf_status kf_filter(kf_plan_t p, const double* F, const int64_t* F_rowptr,
                    const int64_t* F_col, const double* Q, const double* H,
                    const double* R, const double* Y, const double* x0,
                    const double* P0, double* x_filt, double* diagP_filt,
                    int64_t* fail_step);

/* Backward pass, eqns 11-13 (Sec. 2.3) in Rauch-Tung-Striebel form, for
 * t = T-1..1, starting from x_{T|T}, P_{T|T} of the last filter step:
 *   J_t = P_{t|t} F^T P_{t+1|t}^{-1}   (Cholesky of P_{t+1|t}, two solves)
 *   x_{t|T} = x_{t|t} + J_t (x_{t+1|T} - x_{t+1|t})
 *   P_{t|T} = P_{t|t} + J_t (P_{t+1|T} - P_{t+1|t}) J_t^T
 * Requires a successful kf_filter on the same plan (else KF_ERR_STATE).
 *   x_smooth:     T x N output (row t-1 is x_{t|T}; row T-1 equals x_{T|T}).
 *   diagP_smooth: T x N output of diag(P_{t|T}), or NULL.
 *   P_smooth_at:  N x N output of the full P_{t_full|T}, or NULL.
 *   t_full:       1-based step for P_smooth_at, or -1.
 *   fail_step:    as for kf_filter (step whose P_{t+1|t} failed), or NULL. */
kf_status fis_smooth(kf_plan_t p, double* x_smooth, double* diagP_smooth,
                     double* P_smooth_at, int64_t t_full, int64_t* fail_step);

/* Minimum-norm estimate, eqn 5 (Sec. 2.1), for all T columns at once:
 *   X[t] = lambda C H^T (lambda H C H^T + R)^{-1} y_t
 * H: m x N; C: N x N (c_kind DENSE) or N (DIAG) or 1 (SCALAR); R per r_kind;
 * Y: T x m; X_out: T x N.  float64 throughout; uses its own temporary device
 * memory.  stream: cudaStream_t.  Returns KF_ERR_NOT_PD if the m x m matrix
 * is not positive definite. */
kf_status mne_solve(const double* H, const double* C, int32_t c_kind,
                    const double* R, int32_t r_kind, const double* Y,
                    int64_t N, int64_t m, int64_t T, double lambda,
                    double* X_out, void* stream);

/* The paper's initialisation (Sec. 2.4, practical considerations): the
 * initial state is the minimum-norm estimate, and the state-noise covariance
 * Sigma_w (Q here) is the sample covariance of the differenced sequence of
 * minimum-norm estimates X[0..T-1] (eqn 5, as mne_solve):
 *   x0_out = X[0]   (the first sample's estimate: no observation exists at t = 0)
 *   d_k    = X[k+1] - X[k],  k = 0..T-2
 *   Q_out  = sum_k (d_k - dbar)(d_k - dbar)^T / (T - 2),  dbar = mean of d_k
 * (unbiased, mean removed; rank <= T - 2, so Q_out is singular when T - 2 < N
 * and goes to kf_filter as a dense Q, where P_{t|t} + Q stays positive
 * definite).  Arguments as for mne_solve, plus:
 *   X_out:  T x N output of the estimates, or NULL (then kept internally);
 *   x0_out: N output; Q_out: N x N output, row-major, exactly symmetric.
 * Needs T >= 3 (KF_ERR_ARG otherwise).  float64 throughout; device pointers;
 * uses its own temporary device memory. */
kf_status mne_init(const double* H, const double* C, int32_t c_kind,
                   const double* R, int32_t r_kind, const double* Y,
                   int64_t N, int64_t m, int64_t T, double lambda,
                   double* X_out, double* x0_out, double* Q_out, void* stream);

/* Host-buffer convenience: copies the HOST inputs to plan-owned device
 * buffers, runs kf_filter then fis_smooth, and copies the HOST outputs back.
 * Argument meaning as for kf_filter / fis_smooth (all pointers here are host
 * pointers; pinned memory makes the copies asynchronous).  Outputs that are
 * NULL are not copied. */
kf_status kf_solve_host(kf_plan_t p, const double* F, const int64_t* F_rowptr,
                        const int64_t* F_col, const double* Q, const double* H,
                        const double* R, const double* Y, const double* x0,
                        const double* P0, double* x_filt, double* diagP_filt,
                        double* x_smooth, double* diagP_smooth, int64_t* fail_step);

/* Per-kernel-class device timing with CUDA events on the plan's stream.
 * kf_plan_profile(p, 1) starts recording (and clears totals); 0 stops.
 * kf_plan_profile_read returns, for kernel class `cls` (see kf_kernel_class),
 * the number of launches and their summed device time in milliseconds
 * (the stream is synchronised first). */
typedef enum {
  KF_KC_FILTER_UPDATE = 0,   /* P_{t|t} = P - K U (and Joseph) product            */
  KF_KC_INNOVATION = 1,      /* U^T = P H^T                                        */
  KF_KC_SMOOTH_GEMM = 2,     /* W = J D and P_{t|T} = P_{t|t} + W J^T              */
  KF_KC_SMOOTH_SOLVE = 3,    /* Cholesky of P_{t+1|t} and the two solves           */
  KF_KC_PREDICT = 4,         /* F P F^T + Q                                        */
  KF_KC_SOLVE_FACTOR = 5,    /* inside SMOOTH_SOLVE: Cholesky (+ inverse) of       */
                             /* P_{t+1|t}                                          */
  KF_KC_SOLVE_GAIN = 6,      /* inside SMOOTH_SOLVE: forming J_t from the factor   */
  KF_KC_SMOOTH_GEMM_KERNEL = 7, /* inside SMOOTH_GEMM, mixed mode: the tensor-core */
                             /* kernel launches alone (one mark per launch)        */
  KF_KC_SOLVE_REFINE = 8,    /* inside SOLVE_GAIN, KF_SOLVE_FP64_TC: the Newton      */
                             /* refinement of the inverse of P_{t+1|t}             */
  KF_KC_REFINE_EXACT_KERNEL = 9, /* inside SOLVE_REFINE: the exact-slice residual  */
                             /* kernel launches alone (I - P X_0, then I - P X_1)  */
  KF_KC_COUNT = 10
} kf_kernel_class;
kf_status kf_plan_profile(kf_plan_t p, int32_t enable);
kf_status kf_plan_profile_read(kf_plan_t p, int32_t cls, int64_t* launches,
                               double* total_ms);

/* Number of kernels this plan has launched since creation (all classes). */
int64_t kf_plan_launch_count(kf_plan_t p);

/* Device-memory arena for plans (a runtime facility of the library; the paper
 * has no counterpart).  kf_arena_reserve allocates `bytes` once on the current
 * device; from then on kf_plan takes its buffers from that reservation
 * (first fit, 256-byte aligned, falling back to cudaMalloc when the arena is
 * full) and kf_plan_destroy returns them, so a server that creates and
 * destroys a plan per request makes no cudaMalloc / cudaFree calls, whose
 * device-wide synchronisation would stall the other requests' streams.
 * Thread-safe.  KF_ERR_STATE if an arena is already reserved.
 * kf_arena_release frees it (KF_ERR_STATE while plans still hold blocks).
 * kf_arena_stats: reserved bytes, bytes held by plans, largest free block. */
kf_status kf_arena_reserve(uint64_t bytes);
kf_status kf_arena_release(void);
kf_status kf_arena_stats(uint64_t* reserved, uint64_t* in_use, uint64_t* largest_free);

void kf_plan_destroy(kf_plan_t p);
const char* kf_strerror(kf_status s);

#ifdef __cplusplus
}
#endif
#endif /* KFMEG_H */
