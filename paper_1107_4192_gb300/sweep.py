"""Synthetic SNR / lambda sweep of the paper's simulation (Sec. 4.1): mean-squared
error of the MNE, Kalman filter and fixed-interval smoother estimates against
the true sources, as a function of the signal-to-noise ratio.

Workload (a synthetic stand-in; the paper's subject lead field and cortex are
not available): a two-hemisphere mesh of N sources, a lead field H (m x N),
Gaussian-smoothed source patches carrying 10-20 Hz sinusoids under a 0.4 Hz
envelope at 600 Hz (T samples), and white sensor noise scaled to the target
SNR.  SNR (eqn 14, garbled in print) is read as
    SNR = sum_t ||H x_t||^2 / (m T sigma^2).
For each (SNR, lambda):
  - MNE: eqn 5 with C = I (mne_solve);
  - the paper's initialisation (Sec. 2.4): x0 and Q from the minimum-norm
    estimates (mne_init);
  - KF + FIS (eqns 6-13) with F = I, R = sigma^2 I (the noise level is known,
    as the paper's empty-room covariance), P0 = lambda I, Q from mne_init.
MSE is reported over all sources and over the active ones (peak amplitude
above 1% of the largest), relative to the mean power of the true sources there.

Only the noise scaling, the MSE bookkeeping and the driving loop run here;
every estimate comes from the library's CUDA path.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import binding as B
from . import solver, synth


def noise_variance(H: np.ndarray, X: np.ndarray, snr: float) -> float:
    """sigma^2 that gives sum_t ||H x_t||^2 / (m T sigma^2) = snr."""
    m, T = H.shape[0], X.shape[0]
    return float(np.sum((X @ H.T) ** 2) / (m * T * snr))


def snr_of(H: np.ndarray, X: np.ndarray, sigma2: float) -> float:
    """The eqn-14 reading: signal power at the sensors over m T sigma^2."""
    m, T = H.shape[0], X.shape[0]
    return float(np.sum((X @ H.T) ** 2) / (m * T * sigma2))


def relative_mse(est: np.ndarray, truth: np.ndarray, mask: np.ndarray | None = None) -> float:
    """sum (est - truth)^2 / sum truth^2 over all samples of the selected sources."""
    if mask is not None:
        est, truth = est[:, mask], truth[:, mask]
    return float(np.sum((est - truth) ** 2) / np.sum(truth ** 2))


def make_workload(N: int, m: int, T: int, seed: int):
    rng = np.random.default_rng(seed)
    neigh = synth.hemisphere_mesh(N)
    H = synth.lead_field(rng, m, N)
    X = synth.patch_sources(rng, neigh, T)
    noise = rng.standard_normal((T, m))
    return H, X, noise


def run_point(H, X, noise, snr: float, lam: float, prec: int, torch):
    """One (SNR, lambda) point on the GPU; returns the three relative MSEs (all, active)."""
    N, m, T = H.shape[1], H.shape[0], X.shape[0]
    sigma2 = noise_variance(H, X, snr)
    Y = X @ H.T + np.sqrt(sigma2) * noise
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float64)).cuda()
    dH, dY, dC, dR = t(H), t(Y), t(np.array([1.0])), t(np.array([sigma2]))
    Xm = torch.empty(T, N, dtype=torch.float64, device="cuda")
    x0 = torch.empty(N, dtype=torch.float64, device="cuda")
    Q = torch.empty(N, N, dtype=torch.float64, device="cuda")
    B.mne_init(dH, dC, B.KF_COV_SCALAR, dR, B.KF_COV_SCALAR, dY, N, m, T, lam, Xm, x0, Q)
    prob = synth.Problem(N, m, T, H, Y, x0.cpu().numpy(), lam, B.KF_COV_DENSE, Q.cpu().numpy(),
                         B.KF_COV_SCALAR, np.array(sigma2), name="sweep")
    del Q
    out = solver.run(prob, prec=prec, solve_prec=B.KF_SOLVE_FP32 if prec != B.KF_PREC_FP64 else B.KF_SOLVE_FP64,
                     joseph_every=16 if prec == B.KF_PREC_MIXED_BF16X3 else 0)
    mne = Xm.cpu().numpy()
    active = np.max(np.abs(X), axis=0) > 0.01 * np.max(np.abs(X))
    res = {}
    for name, est in (("mne", mne), ("kf", out["x_filt"]), ("fis", out["x_smooth"])):
        res[name] = relative_mse(est, X)
        res[name + "_active"] = relative_mse(est, X, active)
    return res


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--N", type=int, default=5124)
    ap.add_argument("--m", type=int, default=306)
    ap.add_argument("--T", type=int, default=120)
    ap.add_argument("--snrs", type=int, default=20, help="SNRs equispaced in [0.1, 2]")
    ap.add_argument("--lambdas", type=str, default="0.5,1,3")
    ap.add_argument("--prec", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--seed", type=int, default=14)
    args = ap.parse_args(argv)
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("the sweep runs on the GPU path; no CUDA device")
    B.lib()
    prec = B.KF_PREC_MIXED_BF16X3 if args.prec == "mixed" else B.KF_PREC_FP64
    H, X, noise = make_workload(args.N, args.m, args.T, args.seed)
    for lam in [float(v) for v in args.lambdas.split(",")]:
        for snr in np.linspace(0.1, 2.0, args.snrs):
            t0 = time.perf_counter()
            res = run_point(H, X, noise, float(snr), lam, prec, torch)
            res.update({"snr": float(snr), "lambda": lam, "N": args.N, "m": args.m, "T": args.T,
                        "prec": args.prec, "seconds": time.perf_counter() - t0})
            print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
