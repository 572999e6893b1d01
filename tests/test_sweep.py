"""SNR sweep of the paper's simulation: host-side bookkeeping (CPU) and a small
sweep through the GPU path."""
import numpy as np
import pytest

from paper_1107_4192_gb300 import sweep


def test_noise_variance_inverts_the_snr_reading():
    rng = np.random.default_rng(1)
    H = rng.standard_normal((7, 20))
    X = rng.standard_normal((11, 20))
    for snr in (0.1, 1.0, 2.0):
        s2 = sweep.noise_variance(H, X, snr)
        assert abs(sweep.snr_of(H, X, s2) - snr) <= 1e-12 * snr
        # by hand: signal power at the sensors over m T sigma^2
        power = sum(float(np.dot(H @ x, H @ x)) for x in X)
        assert abs(power / (7 * 11 * s2) - snr) <= 1e-12 * snr


def test_relative_mse():
    truth = np.array([[1.0, 0.0], [0.0, 2.0]])
    est = np.array([[1.5, 0.0], [0.0, 2.0]])
    assert sweep.relative_mse(est, truth) == pytest.approx(0.25 / 5.0)
    assert sweep.relative_mse(est, truth, np.array([False, True])) == 0.0


def test_workload_shapes():
    H, X, noise = sweep.make_workload(300, 40, 25, seed=3)
    assert H.shape == (40, 300) and X.shape == (25, 300) and noise.shape == (25, 40)
    assert np.count_nonzero(np.max(np.abs(X), axis=0)) > 0


@pytest.mark.gpu
def test_small_sweep_on_the_gpu():
    """The smoother uses all the data, so its error is below the filter's; more SNR, less error."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1107_4192_gb300 import binding as B
    H, X, noise = sweep.make_workload(320, 60, 40, seed=5)
    lo = sweep.run_point(H, X, noise, 0.5, 1.0, B.KF_PREC_FP64, torch)
    hi = sweep.run_point(H, X, noise, 2.0, 1.0, B.KF_PREC_FP64, torch)
    for r in (lo, hi):
        assert all(np.isfinite(v) for v in r.values())
        assert r["fis"] < r["kf"]
    for k in ("mne", "kf", "fis"):
        assert hi[k] < lo[k]
