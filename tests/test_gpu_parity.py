"""GPU Kalman filter + fixed-interval smoother vs the CPU float64 oracle,
through the C ABI, on seeded synthetic problems.

Tolerances: float64 path <= 1e-10 relative on means (per time step, 2-norm)
and on diag P (elementwise); float32 bulk paths <= 1e-4 on means and <= 1e-3
on diag P.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import kf_oracle as ko  # noqa: E402
from paper_1107_4192_gb300 import binding as B  # noqa: E402
from paper_1107_4192_gb300 import solver, synth  # noqa: E402
from tests.helpers import diag_of, oracle_dense, rel_err_elementwise, rel_err_per_step, run_oracle  # noqa: E402

TOL64 = 1e-10
TOL_MEAN32, TOL_DIAG32 = 1e-4, 1e-3


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1107_4192_gb300 import build
    build.build()
    B.lib()


def check(out, ref, tol_mean, tol_diag):
    assert rel_err_per_step(out["x_filt"], ref["x_filt"]) <= tol_mean
    assert rel_err_elementwise(out["diagP_filt"], diag_of(ref["P_filt"])) <= tol_diag
    assert rel_err_per_step(out["x_smooth"], ref["x_smooth"]) <= tol_mean
    assert rel_err_elementwise(out["diagP_smooth"], diag_of(ref["P_smooth"])) <= tol_diag


def test_config0_fp64():
    """N=384, m=64, T=40 random walk, float64 throughout."""
    prob = synth.config0()
    check(solver.run(prob, prec=B.KF_PREC_FP64), run_oracle(prob), TOL64, TOL64)


@pytest.mark.parametrize("N,m,T", [(1, 1, 1), (7, 3, 2), (129, 65, 5), (200, 70, 3), (257, 130, 4), (70, 300, 3)])
def test_ragged_sizes_fp64(N, m, T):
    prob = synth.random_walk_problem(N, m, T, seed=N + m + T)
    check(solver.run(prob, prec=B.KF_PREC_FP64), run_oracle(prob), TOL64, TOL64)


def test_general_dense_inputs_fp64():
    """Non-symmetric sparse F, dense Q, R, P0, non-zero x0."""
    prob = synth.random_dense_problem(150, 13, 9, seed=3)
    check(solver.run(prob, prec=B.KF_PREC_FP64), run_oracle(prob), TOL64, TOL64)


def test_mesh_coupling_fp64():
    prob = synth.mesh_problem(324, 30, 12, seed=4)
    check(solver.run(prob, prec=B.KF_PREC_FP64), run_oracle(prob), TOL64, TOL64)


@pytest.mark.parametrize("solve", [B.KF_SOLVE_FP64, B.KF_SOLVE_FP32])
@pytest.mark.parametrize("mesh", [False, True])
def test_fp32_paths(solve, mesh):
    prob = synth.mesh_problem(324, 30, 12, seed=4) if mesh else synth.random_walk_problem(384, 64, 20, seed=0)
    check(solver.run(prob, prec=B.KF_PREC_FP32, solve_prec=solve), run_oracle(prob), TOL_MEAN32, TOL_DIAG32)


@pytest.mark.parametrize("solve", [B.KF_SOLVE_FP64, B.KF_SOLVE_FP32, B.KF_SOLVE_FP64_TC])
@pytest.mark.parametrize("mesh", [False, True])
def test_mixed_bf16x3_paths(solve, mesh):
    """Split-bf16 tensor-core products with float32 accumulation, Joseph form every 4 steps."""
    prob = synth.mesh_problem(324, 30, 12, seed=4) if mesh else synth.random_walk_problem(384, 64, 20, seed=0)
    out = solver.run(prob, prec=B.KF_PREC_MIXED_BF16X3, solve_prec=solve, joseph_every=4)
    check(out, run_oracle(prob), TOL_MEAN32, TOL_DIAG32)


@pytest.mark.parametrize("solve", [B.KF_SOLVE_FP32, B.KF_SOLVE_FP64_TC, B.KF_SOLVE_FP64_MEAN])
@pytest.mark.parametrize("N,m,T", [(129, 20, 4), (257, 70, 5), (600, 64, 4), (200, 306, 5), (512, 306, 6)])
def test_mixed_ragged_sizes(N, m, T, solve):
    prob = synth.random_walk_problem(N, m, T, seed=N + m)
    out = solver.run(prob, prec=B.KF_PREC_MIXED_BF16X3, solve_prec=solve, joseph_every=2)
    check(out, run_oracle(prob), TOL_MEAN32, TOL_DIAG32)


def test_mixed_six_term_smoother_products():
    prob = synth.mesh_problem(324, 30, 12, seed=4)
    out = solver.run(prob, prec=B.KF_PREC_MIXED_BF16X3, solve_prec=B.KF_SOLVE_FP32, joseph_every=4, split_terms=6)
    check(out, run_oracle(prob), TOL_MEAN32, TOL_DIAG32)


def test_joseph_every_k_fp64():
    prob = synth.random_dense_problem(130, 20, 10, seed=9)
    check(solver.run(prob, prec=B.KF_PREC_FP64, joseph_every=3), run_oracle(prob), TOL64, TOL64)


@pytest.mark.parametrize("prec", [B.KF_PREC_FP64, B.KF_PREC_FP32])
def test_checkpoint_recompute_is_bitwise_identical(prec):
    prob = synth.mesh_problem(324, 30, 17, seed=8)
    full = solver.run(prob, prec=prec)
    for c in (2, 3, 5, 17):
        part = solver.run(prob, prec=prec, checkpoint_every=c)
        for k in full:
            assert np.array_equal(full[k], part[k]), (c, k)


@pytest.mark.parametrize("solve", [B.KF_SOLVE_FP32, B.KF_SOLVE_FP64_TC])
@pytest.mark.parametrize("mesh", [False, True])
@pytest.mark.parametrize("c", [2, 5])
def test_mixed_checkpoint_recompute(mesh, c, solve):
    """Mixed path with only every c-th P_{t|t} kept: the skipped steps are recomputed during the
    smoother from float32 checkpoints (the float64 working covariance restarts from a float32
    value), so results differ from the full store by rounding only; both stay within the mixed
    tolerances of the oracle."""
    prob = synth.mesh_problem(324, 30, 17, seed=8, identity_F=not mesh)
    kw = dict(prec=B.KF_PREC_MIXED_BF16X3, solve_prec=solve, joseph_every=4)
    ref = run_oracle(prob)
    full = solver.run(prob, **kw)
    part = solver.run(prob, checkpoint_every=c, **kw)
    check(part, ref, TOL_MEAN32, TOL_DIAG32)
    # the filter pass is the same launch sequence either way
    assert np.array_equal(full["x_filt"], part["x_filt"])
    assert rel_err_per_step(part["x_smooth"], full["x_smooth"]) <= 1e-5


@pytest.mark.parametrize("prec,solve,tm,td", [
    (B.KF_PREC_FP64, B.KF_SOLVE_FP64, TOL64, TOL64),
    (B.KF_PREC_FP32, B.KF_SOLVE_FP64, TOL_MEAN32, TOL_DIAG32),
    (B.KF_PREC_MIXED_BF16X3, B.KF_SOLVE_FP32, TOL_MEAN32, TOL_DIAG32),
    (B.KF_PREC_MIXED_BF16X3, B.KF_SOLVE_FP64, TOL_MEAN32, TOL_DIAG32),
    (B.KF_PREC_MIXED_BF16X3, B.KF_SOLVE_FP64_TC, TOL_MEAN32, TOL_DIAG32),
    (B.KF_PREC_MIXED_BF16X3, B.KF_SOLVE_FP64_MEAN, TOL_MEAN32, TOL_DIAG32)])
@pytest.mark.parametrize("N,m,T", [(200, 20, 8), (257, 70, 5)])
def test_dense_F(prec, solve, tm, td, N, m, T):
    """General dense, non-symmetric F passed as a dense N x N matrix (KF_F_DENSE), dense Q, R, P0."""
    prob = synth.dense_dynamics_problem(N, m, T, seed=N + T)
    out = solver.run(prob, prec=prec, solve_prec=solve, joseph_every=3, dense_F=True)
    check(out, run_oracle(prob), tm, td)


def test_dense_F_equals_compressed_rows_fp64():
    """The same F given densely and as compressed rows with every entry present: same result to
    float64 rounding."""
    prob = synth.dense_dynamics_problem(150, 13, 6, seed=2)
    a = solver.run(prob, prec=B.KF_PREC_FP64, dense_F=True)
    b = solver.run(prob, prec=B.KF_PREC_FP64)
    for k in a:
        assert rel_err_per_step(a[k], b[k]) <= 1e-12, k


@pytest.fixture(scope="module")
def long_epoch():
    prob = synth.mesh_problem(1024, 306, 300, seed=11, identity_F=True)
    return prob, run_oracle(prob)


@pytest.mark.parametrize("solve", [B.KF_SOLVE_FP32, B.KF_SOLVE_FP64_TC, B.KF_SOLVE_FP64_MEAN])
def test_mixed_long_epoch_T300(long_epoch, solve):
    """Mixed path over a 300-step epoch (Joseph form every 16 steps, float32 store), the
    configuration of the N = 8196 benchmark at N = 1024: rounding errors must not build up
    through the filter's random walk or the smoother's recursions beyond the mixed tolerances."""
    prob, ref = long_epoch
    out = solver.run(prob, prec=B.KF_PREC_MIXED_BF16X3, solve_prec=solve, joseph_every=16)
    errs = dict(x_filt=rel_err_per_step(out["x_filt"], ref["x_filt"]),
                x_smooth=rel_err_per_step(out["x_smooth"], ref["x_smooth"]),
                diagP_filt=rel_err_elementwise(out["diagP_filt"], diag_of(ref["P_filt"])),
                diagP_smooth=rel_err_elementwise(out["diagP_smooth"], diag_of(ref["P_smooth"])))
    print(f"mixed (solve {solve}) N=1024 m=306 T=300 errors vs oracle:", errs)
    check(out, ref, TOL_MEAN32, TOL_DIAG32)


@pytest.mark.parametrize("solve", [B.KF_SOLVE_FP64_TC, B.KF_SOLVE_FP64_MEAN])
@pytest.mark.parametrize("fkind", ["identity", "mesh", "dense"])
def test_fp64_accurate_solves_match_the_cuda_core_solve(solve, fkind):
    """With the same mixed filter (float64-class, so filtered means and stored P_{t|t} are the
    same launch sequence) every float64 solve inverts the same float64 P_{t+1|t} = F P_{t|t} F^T + Q:
    the smoothed means of the float64-accurate tensor-core solves equal those of the float64
    CUDA-core solve (Cholesky + two triangular solves) to float64 rounding times the conditioning,
    far below the float32-class solve's difference."""
    prob = {"dense": lambda: synth.dense_dynamics_problem(384, 40, 12, seed=5),
            "mesh": lambda: synth.mesh_problem(324, 40, 12, seed=6),
            "identity": lambda: synth.mesh_problem(600, 64, 12, seed=7, identity_F=True)}[fkind]()
    kw = dict(prec=B.KF_PREC_MIXED_BF16X3, joseph_every=4, dense_F=fkind == "dense")
    ref = solver.run(prob, solve_prec=B.KF_SOLVE_FP64, **kw)
    out = solver.run(prob, solve_prec=solve, **kw)
    f32 = solver.run(prob, solve_prec=B.KF_SOLVE_FP32, **kw)
    assert np.array_equal(out["x_filt"], ref["x_filt"])
    e = rel_err_per_step(out["x_smooth"], ref["x_smooth"])
    e32 = rel_err_per_step(f32["x_smooth"], ref["x_smooth"])
    print(f"solve {solve} F {fkind}: smoothed means vs float64 solve {e:.2e} (float32-class solve {e32:.2e})")
    assert e <= 1e-10
    assert rel_err_elementwise(out["diagP_smooth"], ref["diagP_smooth"]) <= TOL_DIAG32


def test_full_smoothed_covariance_output():
    prob = synth.random_dense_problem(90, 11, 6, seed=12)
    ref = run_oracle(prob)
    for t_full in (1, 3, 6):
        out = solver.run(prob, prec=B.KF_PREC_FP64, t_full=t_full)
        P = out["P_smooth_at"]
        R = ref["P_smooth"][t_full - 1]
        assert np.array_equal(P, P.T)
        assert np.linalg.norm(P - R) <= TOL64 * np.linalg.norm(R)


def test_first_step_equals_mne_closed_form():
    """x_{1|1} with F = I, x0 = 0 equals eqn 5 with C = P0 + Q; and = P0 when Q = 0."""
    prob = synth.random_walk_problem(300, 40, 2, seed=21)
    for q in (0.01, 0.0):
        prob.Q = np.array(q)
        out = solver.run(prob, prec=B.KF_PREC_FP64) if q > 0 else None
        d = solver.upload(prob)
        with solver.Plan.for_inputs(d, prob.N, prob.m, prob.T) as plan:
            if q == 0.0:
                # Q = 0 makes P_{2|1} singular for the smoother; the filter alone is fine
                xf, _ = plan.filter(d)
                x1 = xf[0].cpu().numpy()
            else:
                x1 = out["x_filt"][0]
        C = (1.0 + q) * np.eye(prob.N)
        ref = ko.mne_solve(prob.H, C, np.eye(prob.m), prob.Y[:1])[0]
        assert np.linalg.norm(x1 - ref) <= 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("c_kind", [B.KF_COV_SCALAR, B.KF_COV_DIAG, B.KF_COV_DENSE])
@pytest.mark.parametrize("lam", [0.5, 3.0])
def test_mne_solve(c_kind, lam):
    rng = np.random.default_rng(5)
    N, m, T = 230, 37, 9
    H = synth.lead_field(rng, m, N)
    Y = rng.standard_normal((T, m))
    Rv = rng.uniform(0.5, 2, m)
    Cv = {0: np.array([0.7]), 1: rng.uniform(0.5, 2, N)}.get(c_kind)
    if c_kind == 2:
        A = rng.standard_normal((N, N)) / np.sqrt(N)
        Cv = 0.5 * np.eye(N) + A @ A.T
    Cd = ko.dense_cov(c_kind, Cv, N)
    ref = ko.mne_solve(H, Cd, np.diag(Rv), Y, lam)
    X = torch.empty(T, N, dtype=torch.float64, device="cuda")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float64)).cuda()
    B.mne_solve(t(H), t(Cv), c_kind, t(Rv), B.KF_COV_DIAG, t(Y), N, m, T, lam, X)
    assert rel_err_per_step(X.cpu().numpy(), ref) <= 1e-11


@pytest.mark.parametrize("c_kind", [0, 1, 2])
@pytest.mark.parametrize("N,m,T", [(230, 37, 9), (129, 20, 3)])
def test_mne_init(c_kind, N, m, T):
    """Sec. 2.4 initialisation (x0 and Q from the minimum-norm estimates) against the oracle;
    then used as x0 and dense Q of a float64 filter + smoother run, also against the oracle."""
    rng = np.random.default_rng(6 + c_kind)
    H = synth.lead_field(rng, m, N)
    Y = rng.standard_normal((T, m))
    Rv = rng.uniform(0.5, 2, m)
    Cv = {0: np.array([0.7]), 1: rng.uniform(0.5, 2, N)}.get(c_kind)
    if c_kind == 2:
        A = rng.standard_normal((N, N)) / np.sqrt(N)
        Cv = 0.5 * np.eye(N) + A @ A.T
    Cd = ko.dense_cov(c_kind, Cv, N)
    x0_ref, Q_ref, X_ref = ko.mne_init(H, Cd, np.diag(Rv), Y, 1.5)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float64)).cuda()
    x0 = torch.empty(N, dtype=torch.float64, device="cuda")
    Q = torch.empty(N, N, dtype=torch.float64, device="cuda")
    X = torch.empty(T, N, dtype=torch.float64, device="cuda")
    B.mne_init(t(H), t(Cv), c_kind, t(Rv), B.KF_COV_DIAG, t(Y), N, m, T, 1.5, X, x0, Q)
    assert rel_err_per_step(X.cpu().numpy(), X_ref) <= 1e-11
    assert np.linalg.norm(x0.cpu().numpy() - x0_ref) <= 1e-11 * np.linalg.norm(x0_ref)
    Qg = Q.cpu().numpy()
    assert np.array_equal(Qg, Qg.T)
    assert np.linalg.norm(Qg - Q_ref) <= 1e-10 * np.linalg.norm(Q_ref)
    # without X_out
    Q2 = torch.empty(N, N, dtype=torch.float64, device="cuda")
    B.mne_init(t(H), t(Cv), c_kind, t(Rv), B.KF_COV_DIAG, t(Y), N, m, T, 1.5, None, x0, Q2)
    assert torch.equal(Q, Q2)


def test_mne_init_feeds_the_filter():
    """x0 and dense Q from mne_init drive a float64 KF + FIS on the GPU, checked against the
    oracle run from the oracle's own initialisation (the paper's pipeline, Sec. 2.4)."""
    prob = synth.mesh_problem(200, 30, 12, seed=9)
    F, _, H, R, P0 = oracle_dense(prob)
    x0_ref, Q_ref, _ = ko.mne_init(H, np.eye(prob.N), R, prob.Y, 1.0)
    ref = ko.kf_fis(F, Q_ref, H, R, prob.Y, x0_ref, P0)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float64)).cuda()
    x0 = torch.empty(prob.N, dtype=torch.float64, device="cuda")
    Q = torch.empty(prob.N, prob.N, dtype=torch.float64, device="cuda")
    B.mne_init(t(prob.H), t(np.array([1.0])), 0, t(prob.R), B.KF_COV_DIAG, t(prob.Y), prob.N, prob.m, prob.T,
               1.0, None, x0, Q)
    prob.x0 = x0.cpu().numpy()
    prob.q_kind, prob.Q = 2, Q.cpu().numpy()
    out = solver.run(prob, prec=B.KF_PREC_FP64)
    assert rel_err_per_step(out["x_filt"], ref["x_filt"]) <= 1e-9
    assert rel_err_per_step(out["x_smooth"], ref["x_smooth"]) <= 1e-9


def test_not_pd_innovation_is_reported():
    """R = 0 with a rank-deficient H: S_1 is singular -> KF_ERR_NOT_PD at step 1."""
    prob = synth.random_walk_problem(40, 6, 3, seed=1)
    prob.H[3:] = 0.0
    prob.R = np.array(0.0)
    d = solver.upload(prob)
    with solver.Plan.for_inputs(d, prob.N, prob.m, prob.T) as plan:
        x = torch.empty(prob.T, prob.N, dtype=torch.float64, device="cuda")
        st, step = B.kf_filter(plan.handle, d.F, d.F_rowptr, d.F_col, d.Q, d.H, d.R, d.Y, d.x0, d.P0, x,
                               raise_on_error=False)
        assert st == B.KF_ERR_NOT_PD and step == 1
        st, _ = B.fis_smooth(plan.handle, x, raise_on_error=False)
        assert st == B.KF_ERR_STATE


def test_nan_in_data_is_reported():
    prob = synth.random_walk_problem(50, 8, 6, seed=2)
    prob.Y[2, 4] = np.nan
    d = solver.upload(prob)
    with solver.Plan.for_inputs(d, prob.N, prob.m, prob.T) as plan:
        x = torch.empty(prob.T, prob.N, dtype=torch.float64, device="cuda")
        st, step = B.kf_filter(plan.handle, d.F, d.F_rowptr, d.F_col, d.Q, d.H, d.R, d.Y, d.x0, d.P0, x,
                               raise_on_error=False)
        assert st == B.KF_ERR_NUMERIC and step == 3


def test_smooth_before_filter_is_state_error():
    with solver.Plan(10, 3, 4) as plan:
        x = torch.empty(4, 10, dtype=torch.float64, device="cuda")
        st, _ = B.fis_smooth(plan.handle, x, raise_on_error=False)
        assert st == B.KF_ERR_STATE


def test_host_buffer_entry_matches_device_path():
    prob = synth.mesh_problem(324, 30, 7, seed=6)
    dev = solver.run(prob, prec=B.KF_PREC_FP64)
    h = solver.host_inputs(prob)
    outs = {k: np.empty((prob.T, prob.N)) for k in ("x_filt", "diagP_filt", "x_smooth", "diagP_smooth")}
    with solver.Plan(prob.N, prob.m, prob.T, f_kind=h["f_kind"], f_nnz=h["f_nnz"], q_kind=h["q_kind"],
                     r_kind=h["r_kind"]) as plan:
        B.kf_solve_host(plan.handle, h["F"], h["F_rowptr"], h["F_col"], h["Q"], h["H"], h["R"], h["Y"], h["x0"],
                        h["P0"], outs["x_filt"], outs["diagP_filt"], outs["x_smooth"], outs["diagP_smooth"])
    for k in outs:
        assert np.array_equal(outs[k], dev[k]), k
