"""Pins of the CPU FP64 oracle against what the paper and the mathematics fix.

Each check here uses a route independent of the oracle's own recursion:
a stacked least-squares solve of the regularised criterion (eqn 4), the
brute-force joint Gaussian posterior, the scalar Riccati closed form,
the information-form filter, structural invariants and special cases.
"""
import numpy as np
import pytest

from oracle import kf_oracle as ko
from paper_1107_4192_gb300 import synth
from tests.helpers import oracle_dense, rel_err_per_step

RTOL = 1e-10


def eqn4_minimiser(H, R, y, mu, C):
    """argmin ||y - Hx||^2_R + ||x - mu||^2_C as an ordinary least-squares problem.

    Whitening both terms stacks the criterion into min ||A x - b||_2 with
    A = [Lr^{-1} H ; Lc^{-1}], b = [Lr^{-1} y ; Lc^{-1} mu]; the minimiser
    and its covariance (A^T A)^{-1} are the posterior mean and covariance.
    """
    Lr = np.linalg.cholesky(R)
    Lc = np.linalg.cholesky(C)
    A = np.vstack([np.linalg.solve(Lr, H), np.linalg.solve(Lc, np.eye(C.shape[0]))])
    b = np.concatenate([np.linalg.solve(Lr, y), np.linalg.solve(Lc, mu)])
    x, *_ = np.linalg.lstsq(A, b, rcond=None)
    return x, np.linalg.inv(A.T @ A)


# ------------------------------------------------------------- MNE pins

@pytest.mark.parametrize("with_q", [True, False])
def test_first_step_equals_mne_closed_form(with_q):
    """With F = I, x0 = 0: x_{1|1} = C H^T (H C H^T + R)^{-1} y_1, C = P0 + Q (eqn 5)."""
    prob = synth.random_walk_problem(40, 12, 3, seed=11)
    F, Q, H, R, P0 = oracle_dense(prob)
    if not with_q:
        Q = np.zeros_like(Q)
    out = ko.kalman_filter(F, Q, H, R, prob.Y, prob.x0, P0)
    C = P0 + Q
    x_ls, P_ls = eqn4_minimiser(H, R, prob.Y[0], np.zeros(prob.N), C)
    assert np.linalg.norm(out["x_filt"][0] - x_ls) <= 1e-12 * np.linalg.norm(x_ls)
    assert np.abs(out["P_filt"][0] - P_ls).max() <= 1e-12 * np.abs(P_ls).max()
    # the oracle's eqn-5 routine gives the same x with lambda * C = C
    x_mne = ko.mne_solve(H, C, R, prob.Y[:1], lam=1.0)[0]
    assert np.linalg.norm(x_mne - x_ls) <= 1e-12 * np.linalg.norm(x_ls)


def test_kf_step_is_regularised_ls_with_predicted_prior():
    """Each KF step is eqn 4 with mu = F x_{t-1|t-1} and C = P_{t|t-1} (Sec. 2.2)."""
    prob = synth.random_dense_problem(24, 7, 5, seed=5)
    F, Q, H, R, P0 = oracle_dense(prob)
    out = ko.kalman_filter(F, Q, H, R, prob.Y, prob.x0, P0)
    x_prev, P_prev = prob.x0, P0
    for t in range(prob.T):
        mu = F @ x_prev
        C = F @ P_prev @ F.T + Q
        x_ls, P_ls = eqn4_minimiser(H, R, prob.Y[t], mu, C)
        assert np.linalg.norm(out["x_filt"][t] - x_ls) <= 1e-11 * np.linalg.norm(x_ls)
        assert np.abs(out["P_filt"][t] - P_ls).max() <= 1e-11 * np.abs(P_ls).max()
        x_prev, P_prev = x_ls, P_ls


@pytest.mark.parametrize("lam", [0.5, 1.0, 3.0])
def test_mne_solve_matches_least_squares(lam):
    """Eqn 5 for every t equals the eqn-4 minimiser with mu = 0 and C := lam * C."""
    rng = np.random.default_rng(3)
    N, m, T = 30, 9, 4
    H = synth.lead_field(rng, m, N)
    C = np.diag(rng.uniform(0.5, 2.0, N))
    R = np.diag(rng.uniform(0.5, 2.0, m))
    Y = rng.standard_normal((T, m))
    X = ko.mne_solve(H, C, R, Y, lam=lam)
    for t in range(T):
        x_ls, _ = eqn4_minimiser(H, R, Y[t], np.zeros(N), lam * C)
        assert np.linalg.norm(X[t] - x_ls) <= 1e-12 * np.linalg.norm(x_ls)


def _running_sample_cov(samples):
    """Unbiased sample covariance accumulated one sample at a time (Welford's update)."""
    n = 0
    mean = np.zeros(samples.shape[1])
    m2 = np.zeros((samples.shape[1], samples.shape[1]))
    for s in samples:
        n += 1
        delta = s - mean
        mean = mean + delta / n
        m2 = m2 + np.outer(delta, s - mean)
    return m2 / (n - 1)


def test_mne_init_recovers_known_increments():
    """Sec. 2.4 initialisation: with H = I, a tiny R and an exact random walk as data, the
    minimum-norm estimates are the walk itself, so x0 is its first sample and Q is the sample
    covariance of its known increments (accumulated by a different route)."""
    rng = np.random.default_rng(11)
    N, T = 6, 40
    steps = rng.standard_normal((T - 1, N)) @ np.diag([0.5, 1.0, 2.0, 0.3, 1.5, 0.8])
    walk = np.vstack([rng.standard_normal(N), np.zeros((T - 1, N))])
    walk[1:] = walk[0] + np.cumsum(steps, axis=0)
    x0, Q, X = ko.mne_init(np.eye(N), np.eye(N), 1e-13 * np.eye(N), walk, lam=1.0)
    assert np.allclose(X, walk, rtol=0, atol=1e-9)
    assert np.allclose(x0, walk[0], rtol=0, atol=1e-9)
    ref = _running_sample_cov(steps)
    assert np.linalg.norm(Q - ref) <= 1e-9 * np.linalg.norm(ref)


def test_mne_init_structure_and_shift_invariance():
    """Q is symmetric, positive semidefinite, of rank <= T - 2, and unchanged when every
    observation moves by the same H c (the estimates then move by one constant vector)."""
    rng = np.random.default_rng(12)
    N, m, T = 25, 8, 7
    H = synth.lead_field(rng, m, N)
    C = np.diag(rng.uniform(0.5, 2.0, N))
    R = np.diag(rng.uniform(0.5, 2.0, m))
    Y = rng.standard_normal((T, m))
    x0, Q, X = ko.mne_init(H, C, R, Y, lam=2.0)
    assert np.array_equal(Q, Q.T)
    ev = np.linalg.eigvalsh(Q)
    assert ev.min() >= -1e-12 * ev.max()
    assert np.sum(ev > 1e-10 * ev.max()) <= T - 2
    assert np.array_equal(x0, X[0])
    c = rng.standard_normal(N)
    _, Q2, _ = ko.mne_init(H, C, R, Y + H @ c, lam=2.0)
    assert np.linalg.norm(Q2 - Q) <= 1e-10 * np.linalg.norm(Q)


# ------------------------------------------------- brute-force posterior

def _tiny_general(seed=7, N=4, m=3, T=6):
    return synth.random_dense_problem(N, m, T, seed=seed)


@pytest.mark.parametrize("seed,N,m,T", [(7, 4, 3, 6), (8, 5, 2, 5), (9, 3, 3, 8)])
def test_smoother_equals_batch_posterior(seed, N, m, T):
    prob = _tiny_general(seed, N, m, T)
    F, Q, H, R, P0 = oracle_dense(prob)
    out = ko.kf_fis(F, Q, H, R, prob.Y, prob.x0, P0)
    mean, cov = ko.batch_posterior(F, Q, H, R, prob.Y, prob.x0, P0)
    assert rel_err_per_step(out["x_smooth"], mean) <= RTOL
    assert rel_err_per_step(out["P_smooth"], cov) <= RTOL


@pytest.mark.parametrize("seed,N,m,T", [(7, 4, 3, 6), (10, 6, 2, 4)])
def test_filter_equals_partial_batch_posterior(seed, N, m, T):
    prob = _tiny_general(seed, N, m, T)
    F, Q, H, R, P0 = oracle_dense(prob)
    out = ko.kalman_filter(F, Q, H, R, prob.Y, prob.x0, P0)
    for t in range(1, T + 1):
        mean, cov = ko.batch_posterior(F, Q, H, R, prob.Y, prob.x0, P0, upto=t)
        assert np.linalg.norm(out["x_filt"][t - 1] - mean[t - 1]) <= RTOL * np.linalg.norm(mean[t - 1])
        assert np.linalg.norm(out["P_filt"][t - 1] - cov[t - 1]) <= RTOL * np.linalg.norm(cov[t - 1])
        # the prediction one step ahead is the same posterior's next block
        if t < T:
            assert np.linalg.norm(out["x_pred"][t] - mean[t]) <= RTOL * max(np.linalg.norm(mean[t]), 1e-300)


def test_batch_posterior_prior_blocks_brute_force():
    """With no data the posterior is the prior: Sigma_t = F^t P0 F^tT + sum F^k Q F^kT."""
    prob = _tiny_general(12, 3, 2, 4)
    F, Q, H, R, P0 = oracle_dense(prob)
    mean, cov = ko.batch_posterior(F, Q, 0 * H, R, prob.Y, prob.x0, P0)
    for t in range(1, 5):
        Ft = np.linalg.matrix_power(F, t)
        S = Ft @ P0 @ Ft.T + sum(np.linalg.matrix_power(F, k) @ Q @ np.linalg.matrix_power(F, k).T
                                 for k in range(t))
        assert np.allclose(cov[t - 1], S, rtol=1e-12, atol=1e-14)
        assert np.allclose(mean[t - 1], Ft @ prob.x0, rtol=1e-12, atol=1e-14)


# --------------------------------------------------------- closed forms

@pytest.mark.parametrize("q,h,r", [(0.01, 1.0, 1.0), (0.5, 2.0, 0.3), (1e-3, 0.5, 4.0)])
def test_scalar_riccati_steady_state(q, h, r):
    a, p = ko.scalar_riccati_fixed_point(q, h, r)
    # independent check of the closed form: it satisfies the fixed-point equation
    assert abs(a - (q + a * r / (h * h * a + r))) <= 1e-14 * a
    F, Q, H, R = np.eye(1), q * np.eye(1), h * np.eye(1), r * np.eye(1)
    T = 4000
    Y = np.zeros((T, 1))
    out = ko.kalman_filter(F, Q, H, R, Y, np.zeros(1), np.eye(1))
    assert abs(out["P_filt"][-1, 0, 0] - p) <= 1e-12 * p
    assert abs(out["P_pred"][-1, 0, 0] - a) <= 1e-12 * a


def test_information_filter_agrees():
    prob = synth.random_dense_problem(16, 5, 8, seed=21)
    F, Q, H, R, P0 = oracle_dense(prob)
    out = ko.kalman_filter(F, Q, H, R, prob.Y, prob.x0, P0)
    xs, Ps = ko.information_filter(F, Q, H, R, prob.Y, prob.x0, P0)
    assert rel_err_per_step(out["x_filt"], xs) <= RTOL
    assert rel_err_per_step(out["P_filt"], Ps) <= RTOL


# -------------------------------------------------------------- structure

def test_structure_symmetry_psd_loewner():
    prob = synth.random_dense_problem(12, 4, 10, seed=31)
    F, Q, H, R, P0 = oracle_dense(prob)
    out = ko.kf_fis(F, Q, H, R, prob.Y, prob.x0, P0)
    for t in range(prob.T):
        Pp, Pf, Ps = out["P_pred"][t], out["P_filt"][t], out["P_smooth"][t]
        for P in (Pp, Pf, Ps):
            assert np.abs(P - P.T).max() <= 1e-14 * np.abs(P).max()
            assert np.linalg.eigvalsh(P).min() >= -1e-12 * np.abs(P).max()
        # P_{t|T} <= P_{t|t} <= P_{t|t-1} in the Loewner order
        assert np.linalg.eigvalsh(Pf - Ps).min() >= -1e-12 * np.abs(Pf).max()
        assert np.linalg.eigvalsh(Pp - Pf).min() >= -1e-12 * np.abs(Pp).max()
    assert np.array_equal(out["x_smooth"][-1], out["x_filt"][-1])
    assert np.array_equal(out["P_smooth"][-1], out["P_filt"][-1])


def test_special_case_no_observation_is_pure_prediction():
    prob = synth.random_dense_problem(6, 3, 5, seed=41)
    F, Q, H, R, P0 = oracle_dense(prob)
    out = ko.kf_fis(F, Q, 0 * H, R, prob.Y, prob.x0, P0)
    x, P = prob.x0, P0
    for t in range(prob.T):
        x, P = F @ x, F @ P @ F.T + Q
        assert np.allclose(out["x_filt"][t], x, rtol=1e-12, atol=1e-14)
        assert np.allclose(out["P_filt"][t], P, rtol=1e-12, atol=1e-14)
    # the smoother cannot improve on nothing: filtered = predicted, smoothed = filtered means
    assert np.allclose(out["x_smooth"], out["x_filt"], rtol=1e-10, atol=1e-12)


def test_special_case_exact_observation_tracks_data():
    N, T = 5, 6
    rng = np.random.default_rng(2)
    Y = rng.standard_normal((T, N))
    out = ko.kf_fis(np.eye(N), 0.1 * np.eye(N), np.eye(N), 1e-12 * np.eye(N), Y,
                    np.zeros(N), np.eye(N))
    assert np.abs(out["x_filt"] - Y).max() <= 1e-9
    assert np.abs(out["x_smooth"] - Y).max() <= 1e-9


def test_permutation_equivariance():
    prob = synth.random_dense_problem(10, 4, 6, seed=51)
    F, Q, H, R, P0 = oracle_dense(prob)
    out = ko.kf_fis(F, Q, H, R, prob.Y, prob.x0, P0)
    p = np.random.default_rng(0).permutation(prob.N)
    Pm = np.eye(prob.N)[p]
    out2 = ko.kf_fis(Pm @ F @ Pm.T, Pm @ Q @ Pm.T, H @ Pm.T, R, prob.Y, Pm @ prob.x0, Pm @ P0 @ Pm.T)
    assert np.allclose(out2["x_smooth"], out["x_smooth"][:, p], rtol=1e-11, atol=1e-13)
    assert np.allclose(out2["P_smooth"], out["P_smooth"][:, p][:, :, p], rtol=1e-11, atol=1e-13)


def test_not_pd_innovation_raises():
    """R = 0 with a rank-deficient H makes S singular: the oracle refuses (no jitter)."""
    N, m = 4, 3
    H = np.zeros((m, N))
    H[0, 0] = 1.0
    with pytest.raises(np.linalg.LinAlgError):
        ko.kalman_filter(np.eye(N), 0 * np.eye(N), H, 0 * np.eye(m), np.zeros((2, m)),
                         np.zeros(N), np.eye(N))


def test_csr_densify_brute_force():
    prob = synth.mesh_problem(40, 5, 2, seed=1)
    F = ko.dense_from_csr(prob.N, prob.F.rowptr, prob.F.col, prob.F.val)
    for i in range(prob.N):
        for j in range(prob.N):
            mask = (prob.F.col[prob.F.rowptr[i]:prob.F.rowptr[i + 1]] == j)
            expect = prob.F.val[prob.F.rowptr[i]:prob.F.rowptr[i + 1]][mask].sum()
            assert F[i, j] == expect
