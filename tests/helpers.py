"""Shared test helpers: feeding a synthetic problem to the oracle and error metrics."""
import numpy as np

from oracle import kf_oracle as ko


def oracle_dense(prob):
    """Dense (F, Q, H, R, P0) for the oracle, built by the oracle's own helpers."""
    if prob.F is None:
        F = np.eye(prob.N)
    else:
        F = ko.dense_from_csr(prob.N, prob.F.rowptr, prob.F.col, prob.F.val)
    Q = ko.dense_cov(prob.q_kind, prob.Q, prob.N)
    R = ko.dense_cov(prob.r_kind, prob.R, prob.m)
    P0 = prob.P0 if prob.P0 is not None else prob.p0_scale * np.eye(prob.N)
    return F, Q, prob.H, R, np.asarray(P0, float)


def run_oracle(prob, T=None):
    F, Q, H, R, P0 = oracle_dense(prob)
    Y = prob.Y if T is None else prob.Y[:T]
    return ko.kf_fis(F, Q, H, R, Y, prob.x0, P0)


def rel_err_per_step(a, b):
    """max over t of ||a_t - b_t||_2 / ||b_t||_2 (rows are time steps)."""
    a = np.asarray(a).reshape(a.shape[0], -1)
    b = np.asarray(b).reshape(b.shape[0], -1)
    num = np.linalg.norm(a - b, axis=1)
    den = np.maximum(np.linalg.norm(b, axis=1), 1e-300)
    return float(np.max(num / den))


def rel_err_elementwise(a, b):
    """max over entries of |a - b| / |b|."""
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)))


def diag_of(Ps):
    return np.stack([np.diag(P) for P in Ps])
