"""CPU FP64 oracle for the Kalman filter + fixed-interval smoother.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import or call
this module: only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` use it.  It shares no code with the CUDA
library (no kernels, helpers, tables or pre/post-processing).

Everything here is plain numpy in float64, written step by step in the
order the paper states the method, with library primitives (matmul,
Cholesky, triangular solve) as the only building blocks.

Notation follows the paper, renamed as in the project's interface:
the paper's W (state covariance) is P here, Sigma_w is Q, Sigma_eps is R,
J_k (source vector) is x_t and the smoother gain A_k is J_t.

Readings of the paper that the oracle fixes (the paper's text is garbled
or silent at these points):

* Eqn 7 prints W_{k|k-1} = W_{k-1|k-1} + Sigma_w without F.  That is the
  F = I special case; with the general state model of eqn 3 the predicted
  covariance is F P F^T + Q.
* Initial condition: (x0, P0) describe the state at t = 0, Q is a separate
  input, and step t = 1 predicts and then updates with y_1.
* Eqn 9's broken lines are the same update as eqn 10, which is used.
* Eqns 11-13 carry typos; the standard Rauch-Tung-Striebel recursion the
  paper cites is used: J_t = P_{t|t} F^T P_{t+1|t}^{-1},
  x_{t|T} = x_{t|t} + J_t (x_{t+1|T} - x_{t+1|t}),
  P_{t|T} = P_{t|t} + J_t (P_{t+1|T} - P_{t+1|t}) J_t^T, for t = T-1..1,
  starting from the filter's last step.
* The covariance update of eqn 10 (I - K H) P is computed in Joseph form
  and symmetrised; both are equal in exact arithmetic.
* Initialisation (Sec. 2.4): the initial state "J_0^MNE" is read as the
  minimum-norm estimate of the first sample, and Sigma_w as the unbiased
  sample covariance (mean removed, divisor T - 2) of the T - 1 differences
  of consecutive minimum-norm estimates.

Parity pins (checked by the CPU test-suite, not by this module): the MNE
closed form of eqn 5 solved as the regularised least squares of eqn 4,
the brute-force joint Gaussian posterior, the scalar Riccati fixed point,
an information-form filter, symmetry / PSD / Loewner ordering and special
cases; for mne_init, the sample covariance of known random-walk increments
(accumulated one sample at a time) and invariance to a constant shift.
Every function here is pinned by at least one of them.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


# ------------------------------------------------------------ input forms

def dense_cov(kind: int, value, n: int) -> np.ndarray:
    """Covariance given as 0 = scalar * I, 1 = diagonal vector, 2 = dense."""
    if kind == 0:
        return float(np.asarray(value, dtype=np.float64).reshape(-1)[0]) * np.eye(n)
    if kind == 1:
        return np.diag(np.asarray(value, dtype=np.float64))
    return np.array(value, dtype=np.float64, copy=True)


def dense_from_csr(n: int, rowptr, col, val) -> np.ndarray:
    """The state transition F of eqn 3 from compressed-row arrays."""
    F = np.zeros((n, n))
    for i in range(n):
        for k in range(int(rowptr[i]), int(rowptr[i + 1])):
            F[i, int(col[k])] += float(val[k])
    return F


def symmetrise(A: np.ndarray) -> np.ndarray:
    return 0.5 * (A + A.T)


# ------------------------------------------------------------- Kalman filter

def kf_predict(F, Q, x, P):
    """Eqn 6 (mean) and eqn 7 read as F P F^T + Q (covariance)."""
    x_pred = F @ x
    P_pred = F @ P @ F.T + Q
    return x_pred, symmetrise(P_pred)


def kf_update(H, R, y, x_pred, P_pred):
    """Eqns 8 and 10: gain via Cholesky of S = H P H^T + R, Joseph-form covariance."""
    S = H @ P_pred @ H.T + R
    L = np.linalg.cholesky(S)                       # raises LinAlgError if S is not PD
    PHt = P_pred @ H.T
    # K = P H^T S^{-1}  <=>  K^T = S^{-1} H P = L^{-T} L^{-1} (P H^T)^T
    Z = sla.solve_triangular(L, PHt.T, lower=True)
    K = sla.solve_triangular(L.T, Z, lower=False).T
    innov = y - H @ x_pred
    x = x_pred + K @ innov
    A = np.eye(P_pred.shape[0]) - K @ H
    P = A @ P_pred @ A.T + K @ R @ K.T
    return x, symmetrise(P), K, S


def kalman_filter(F, Q, H, R, Y, x0, P0):
    """Forward pass, t = 1..T.  Returns arrays indexed [t-1] for t = 1..T.

    x_pred[t-1] = x_{t|t-1}, P_pred[t-1] = P_{t|t-1},
    x_filt[t-1] = x_{t|t},   P_filt[t-1] = P_{t|t}.
    """
    T = Y.shape[0]
    x, P = np.asarray(x0, float), np.asarray(P0, float)
    out = {k: [] for k in ("x_pred", "P_pred", "x_filt", "P_filt")}
    for t in range(T):
        xp, Pp = kf_predict(F, Q, x, P)
        x, P, _, _ = kf_update(H, R, Y[t], xp, Pp)
        out["x_pred"].append(xp)
        out["P_pred"].append(Pp)
        out["x_filt"].append(x)
        out["P_filt"].append(P)
    return {k: np.asarray(v) for k, v in out.items()}


# ----------------------------------------------- fixed-interval smoother

def rts_smoother(F, filt):
    """Eqns 11-13 (standard RTS form), t = T-1..1 from (x_{T|T}, P_{T|T})."""
    xf, Pf, xp, Pp = filt["x_filt"], filt["P_filt"], filt["x_pred"], filt["P_pred"]
    T = xf.shape[0]
    xs = np.empty_like(xf)
    Ps = np.empty_like(Pf)
    xs[T - 1], Ps[T - 1] = xf[T - 1], Pf[T - 1]
    for t in range(T - 2, -1, -1):
        # J_t = P_{t|t} F^T P_{t+1|t}^{-1}, by Cholesky of P_{t+1|t}:
        # J^T = L^{-T} L^{-1} (F P_{t|t})
        L = np.linalg.cholesky(Pp[t + 1])
        Z = sla.solve_triangular(L, F @ Pf[t], lower=True)
        J = sla.solve_triangular(L.T, Z, lower=False).T
        xs[t] = xf[t] + J @ (xs[t + 1] - xp[t + 1])
        Ps[t] = symmetrise(Pf[t] + J @ (Ps[t + 1] - Pp[t + 1]) @ J.T)
    return xs, Ps


def kf_fis(F, Q, H, R, Y, x0, P0):
    """Kalman filter followed by the fixed-interval smoother."""
    filt = kalman_filter(F, Q, H, R, Y, x0, P0)
    xs, Ps = rts_smoother(F, filt)
    filt["x_smooth"], filt["P_smooth"] = xs, Ps
    return filt


# ------------------------------------------------------- static solver (MNE)

def mne_solve(H, C, R, Y, lam=1.0):
    """Eqn 5: x_t = lam C H^T (lam H C H^T + R)^{-1} y_t for every t (rows of Y)."""
    G = lam * (H @ C @ H.T) + R
    L = np.linalg.cholesky(G)
    Z = sla.solve_triangular(L, Y.T, lower=True)
    W = sla.solve_triangular(L.T, Z, lower=False)
    return (lam * (C @ H.T) @ W).T


def mne_init(H, C, R, Y, lam=1.0):
    """The paper's initialisation (Sec. 2.4): the initial state is the minimum-norm
    estimate and Sigma_w (Q) is the sample covariance of the differenced sequence
    of minimum-norm estimates.  Readings: the initial state is the first sample's
    estimate (no observation exists at t = 0); the sample covariance removes the
    mean of the differences and divides by (number of differences - 1)."""
    X = mne_solve(H, C, R, Y, lam)
    d = X[1:] - X[:-1]
    dc = d - d.mean(axis=0)
    Q = dc.T @ dc / (d.shape[0] - 1)
    return X[0].copy(), symmetrise(Q), X


# ------------------------------------- second, independent recursion

def information_filter(F, Q, H, R, Y, x0, P0):
    """The same posterior propagated in information form (inverse covariances).

    Prediction in covariance form, update as P^{-1} <- P^{-1} + H^T R^{-1} H and
    P^{-1} x <- P^{-1} x_pred + H^T R^{-1} y.  Used to cross-check the filter.
    """
    T = Y.shape[0]
    x, P = np.asarray(x0, float), np.asarray(P0, float)
    Rinv = np.linalg.inv(R)
    HtRiH = H.T @ Rinv @ H
    xs, Ps = [], []
    for t in range(T):
        xp = F @ x
        Pp = F @ P @ F.T + Q
        Lam_p = np.linalg.inv(Pp)
        Lam = Lam_p + HtRiH
        eta = Lam_p @ xp + H.T @ Rinv @ Y[t]
        P = np.linalg.inv(Lam)
        x = P @ eta
        P = symmetrise(P)
        xs.append(x)
        Ps.append(P)
    return np.asarray(xs), np.asarray(Ps)


# ------------------------------------------------- brute-force posterior

def batch_posterior(F, Q, H, R, Y, x0, P0, upto=None):
    """Joint Gaussian posterior of (x_1..x_T) given y_1..y_upto, by brute force.

    Prior: x_t = F^t x0 + sum of propagated noises, so
    E[x_t] = F^t x0 and Cov(x_s, x_t) = F^{t-s} Sigma_s (s <= t), with
    Sigma_t = F Sigma_{t-1} F^T + Q, Sigma_0 = P0.  Observations
    y_t = H x_t + e_t for t <= upto.  Conditioning a dense Gaussian gives
    means (T x N) and covariance blocks (T x N x N) of p(x_t | y_1..y_upto).
    Only for tiny N*T.
    """
    T = Y.shape[0]
    N = F.shape[0]
    m = H.shape[0]
    upto = T if upto is None else upto
    mu = np.zeros(T * N)
    Sig = np.zeros((T, N, N))
    xm, S = np.asarray(x0, float), np.asarray(P0, float)
    for t in range(T):
        xm = F @ xm
        S = F @ S @ F.T + Q
        mu[t * N:(t + 1) * N] = xm
        Sig[t] = S
    C = np.zeros((T * N, T * N))
    for s in range(T):
        blk = Sig[s]
        for t in range(s, T):
            C[t * N:(t + 1) * N, s * N:(s + 1) * N] = blk
            C[s * N:(s + 1) * N, t * N:(t + 1) * N] = blk.T
            blk = F @ blk
    G = np.zeros((upto * m, T * N))
    for t in range(upto):
        G[t * m:(t + 1) * m, t * N:(t + 1) * N] = H
    Rb = np.kron(np.eye(upto), R)
    yv = Y[:upto].reshape(-1)
    Sy = G @ C @ G.T + Rb
    gain = np.linalg.solve(Sy, G @ C).T          # C G^T Sy^{-1}
    post_mu = mu + gain @ (yv - G @ mu)
    post_C = C - gain @ G @ C
    means = post_mu.reshape(T, N)
    covs = np.stack([post_C[t * N:(t + 1) * N, t * N:(t + 1) * N] for t in range(T)])
    return means, covs


# ---------------------------------------------------- closed forms

def scalar_riccati_fixed_point(q: float, h: float, r: float):
    """Steady state of the scalar random walk (F = 1): returns (p_pred, p_filt).

    With a = p_pred, the fixed point of a = q + a r / (h^2 a + r) solves
    h^2 a^2 - q h^2 a - q r = 0, whose positive root is taken.
    """
    a = 0.5 * (q + np.sqrt(q * q + 4.0 * q * r / (h * h)))
    return a, a - q
