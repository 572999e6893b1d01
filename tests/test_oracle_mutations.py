"""Plant plausible mistakes in a copy of the oracle and check that the pins catch them.

Each mutation is a textual edit of the oracle's source (a dropped term, a
flipped sign, a wrong index, a transposed operand).  The mutated module is
executed in a fresh namespace on the CPU; the real oracle is untouched.
A mutation that no pin detects would mean the pins do not constrain that
part of the oracle.
"""
import inspect
import types

import numpy as np
import pytest

from oracle import kf_oracle as ko
from paper_1107_4192_gb300 import synth
from tests.helpers import oracle_dense, rel_err_per_step
from tests.test_oracle import eqn4_minimiser

MUTATIONS = [
    ("drop Q in predict", "P_pred = F @ P @ F.T + Q", "P_pred = F @ P @ F.T"),
    ("transpose F in predict", "P_pred = F @ P @ F.T + Q", "P_pred = F.T @ P @ F + Q"),
    ("predict mean without F", "x_pred = F @ x", "x_pred = x"),
    ("drop R in S", "S = H @ P_pred @ H.T + R", "S = H @ P_pred @ H.T"),
    ("sign of innovation", "x = x_pred + K @ innov", "x = x_pred - K @ innov"),
    ("drop K R K^T in Joseph", "P = A @ P_pred @ A.T + K @ R @ K.T", "P = A @ P_pred @ A.T"),
    ("smoother gain without F", "Z = sla.solve_triangular(L, F @ Pf[t], lower=True)",
     "Z = sla.solve_triangular(L, Pf[t], lower=True)"),
    ("smoother gain wrong index", "L = np.linalg.cholesky(Pp[t + 1])", "L = np.linalg.cholesky(Pp[t])"),
    ("smoother mean wrong index", "xs[t] = xf[t] + J @ (xs[t + 1] - xp[t + 1])",
     "xs[t] = xf[t] + J @ (xs[t + 1] - xp[t])"),
    ("smoother cov transposed gain", "Ps[t] = symmetrise(Pf[t] + J @ (Ps[t + 1] - Pp[t + 1]) @ J.T)",
     "Ps[t] = symmetrise(Pf[t] + J.T @ (Ps[t + 1] - Pp[t + 1]) @ J)"),
    ("smoother cov sign", "Ps[t] = symmetrise(Pf[t] + J @ (Ps[t + 1] - Pp[t + 1]) @ J.T)",
     "Ps[t] = symmetrise(Pf[t] - J @ (Ps[t + 1] - Pp[t + 1]) @ J.T)"),
    ("posterior cross-cov transposed", "blk = F @ blk", "blk = F.T @ blk"),
    ("mne missing lambda in G", "G = lam * (H @ C @ H.T) + R", "G = (H @ C @ H.T) + R"),
    ("init covariance divisor n", "Q = dc.T @ dc / (d.shape[0] - 1)", "Q = dc.T @ dc / d.shape[0]"),
    ("init covariance without mean removal", "dc = d - d.mean(axis=0)", "dc = d"),
    ("init state from the last estimate", "return X[0].copy(), symmetrise(Q), X", "return X[-1].copy(), symmetrise(Q), X"),
]


def _load_mutant(old, new):
    src = inspect.getsource(ko)
    assert src.count(old) >= 1, old
    mod = types.ModuleType("kf_oracle_mutant")
    exec(compile(src.replace(old, new), "kf_oracle_mutant", "exec"), mod.__dict__)
    return mod


def _pins_pass(mod) -> bool:
    """The subset of pins used to decide on a mutant (all hold for the real oracle)."""
    prob = synth.random_dense_problem(4, 3, 6, seed=7)
    F, Q, H, R, P0 = oracle_dense(prob)
    try:
        out = mod.kf_fis(F, Q, H, R, prob.Y, prob.x0, P0)
    except np.linalg.LinAlgError:
        return False
    # recursion vs the brute-force joint posterior (both taken from the mutant)
    mmean, mcov = mod.batch_posterior(F, Q, H, R, prob.Y, prob.x0, P0)
    ok = rel_err_per_step(out["x_smooth"], mmean) <= 1e-10
    ok &= rel_err_per_step(out["P_smooth"], mcov) <= 1e-10
    # the brute-force posterior with no data against explicit matrix powers
    pmean, pcov = mod.batch_posterior(F, Q, 0 * H, R, prob.Y, prob.x0, P0)
    for t in range(1, prob.T + 1):
        Fp = [np.linalg.matrix_power(F, k) for k in range(t + 1)]
        S = Fp[t] @ P0 @ Fp[t].T + sum(Fp[k] @ Q @ Fp[k].T for k in range(t))
        ok &= np.allclose(pcov[t - 1], S, rtol=1e-12, atol=1e-14)
        ok &= np.allclose(pmean[t - 1], Fp[t] @ prob.x0, rtol=1e-12, atol=1e-14)
    # eqn 5 pin
    rng = np.random.default_rng(3)
    Hm = synth.lead_field(rng, 5, 12)
    C = np.diag(rng.uniform(0.5, 2, 12))
    Rm = np.eye(5)
    Y = rng.standard_normal((2, 5))
    lam = 3.0
    ref = np.stack([eqn4_minimiser(Hm, Rm, y, np.zeros(12), lam * C)[0] for y in Y])
    ok &= np.allclose(mod.mne_solve(Hm, C, Rm, Y, lam), ref, rtol=1e-12, atol=1e-14)
    # initialisation pin: known random-walk increments (see test_oracle)
    from tests.test_oracle import _running_sample_cov
    rng = np.random.default_rng(11)
    steps = rng.standard_normal((20, 4))
    walk = np.vstack([rng.standard_normal(4), np.zeros((20, 4))])
    walk[1:] = walk[0] + np.cumsum(steps, axis=0)
    x0, Qi, _ = mod.mne_init(np.eye(4), np.eye(4), 1e-13 * np.eye(4), walk, lam=1.0)
    ok &= np.allclose(x0, walk[0], rtol=0, atol=1e-9)
    ok &= np.allclose(Qi, _running_sample_cov(steps), rtol=1e-9, atol=1e-12)
    return bool(ok)


def test_real_oracle_passes_mutation_pins():
    assert _pins_pass(ko)


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_mutant_is_caught(name, old, new):
    assert not _pins_pass(_load_mutant(old, new)), f"mutation not detected: {name}"
