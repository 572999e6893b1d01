"""Parity at the benchmark's full size: N = 8196 sources, m = 306 sensors, the
same inputs and launch configuration as bench.py, on a prefix of the time
axis (the oracle needs about a minute per time step at this size).

 - mixed path (split-bf16 tensor-core products, float32 solve) and the float64
   GPU path against the CPU float64 oracle on the first 2 steps;
 - mixed path against the float64 GPU path (itself oracle-checked at smaller
   sizes) on the first 5 steps, Joseph form every 2 steps;
 - properties that hold at any size: x_{T|T} equals the filter's, diag P_{t|T}
   <= diag P_{t|t}, exact symmetry of the returned full smoothed covariance.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1107_4192_gb300 import binding as B  # noqa: E402
from paper_1107_4192_gb300 import solver, synth  # noqa: E402
from tests.helpers import diag_of, rel_err_elementwise, rel_err_per_step, run_oracle  # noqa: E402

MIXED = dict(prec=B.KF_PREC_MIXED_BF16X3, solve_prec=B.KF_SOLVE_FP32)
MIXED64 = dict(prec=B.KF_PREC_MIXED_BF16X3, solve_prec=B.KF_SOLVE_FP64_TC)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1107_4192_gb300 import build
    build.build()
    B.lib()


@pytest.fixture(scope="module")
def oracle_T2():
    return run_oracle(synth.config2(T=2))


@pytest.mark.parametrize("mode", ["mixed", "mixed_fp64tc", "mixed_fp64mean", "fp64"])
def test_fullsize_vs_oracle_prefix(oracle_T2, mode):
    prob = synth.config2(T=2)
    kw = {"mixed": MIXED, "mixed_fp64tc": MIXED64, "fp64": dict(prec=B.KF_PREC_FP64),
          "mixed_fp64mean": dict(prec=B.KF_PREC_MIXED_BF16X3, solve_prec=B.KF_SOLVE_FP64_MEAN)}[mode]
    out = solver.run(prob, **kw)
    ref = oracle_T2
    tm, td = (1e-4, 1e-3) if mode.startswith("mixed") else (1e-10, 1e-10)
    assert rel_err_per_step(out["x_filt"], ref["x_filt"]) <= tm
    assert rel_err_per_step(out["x_smooth"], ref["x_smooth"]) <= tm
    assert rel_err_elementwise(out["diagP_filt"], diag_of(ref["P_filt"])) <= td
    assert rel_err_elementwise(out["diagP_smooth"], diag_of(ref["P_smooth"])) <= td


def test_fullsize_mixed_vs_fp64_gpu():
    prob = synth.config2(T=5)
    ref = solver.run(prob, prec=B.KF_PREC_FP64)
    for split in (0, 6):
        out = solver.run(prob, joseph_every=2, split_terms=split, **MIXED)
        assert rel_err_per_step(out["x_filt"], ref["x_filt"]) <= 1e-4
        assert rel_err_per_step(out["x_smooth"], ref["x_smooth"]) <= 1e-4
        assert rel_err_elementwise(out["diagP_filt"], ref["diagP_filt"]) <= 1e-3
        assert rel_err_elementwise(out["diagP_smooth"], ref["diagP_smooth"]) <= 1e-3


def test_fullsize_properties():
    prob = synth.config2(T=4)
    out = solver.run(prob, t_full=2, **MIXED)
    assert np.array_equal(out["x_smooth"][-1], out["x_filt"][-1])
    assert np.all(out["diagP_smooth"] <= out["diagP_filt"] * (1 + 1e-5))
    assert np.all(out["diagP_smooth"] > 0)
    P = out["P_smooth_at"]
    assert np.array_equal(P, P.T)
    assert np.allclose(np.diag(P), out["diagP_smooth"][1], rtol=0, atol=0)


@pytest.mark.skipif(not __import__("os").environ.get("KFMEG_LONG"),
                    reason="a whole float64 epoch at N = 8196 takes about 13 minutes; set KFMEG_LONG=1")
def test_full_epoch_mixed_vs_fp64_gpu():
    """The whole benchmark epoch (N = 8196, m = 306, T = 300, Joseph every 16 steps) on the mixed
    path with the float64-accurate solve, against the float64 GPU path (oracle-checked at smaller
    sizes and on the first steps at this size), within the mixed tolerances; prints both epoch
    times (the float64 one is the plain-float64 baseline measured over the whole epoch)."""
    import time
    prob = synth.config2()
    t0 = time.perf_counter()
    ref = solver.run(prob, prec=B.KF_PREC_FP64)
    torch.cuda.synchronize()
    t_fp64 = time.perf_counter() - t0
    t0 = time.perf_counter()
    out = solver.run(prob, joseph_every=16, **MIXED64)
    torch.cuda.synchronize()
    t_mix = time.perf_counter() - t0
    e = {"x_filt": rel_err_per_step(out["x_filt"], ref["x_filt"]),
         "x_smooth": rel_err_per_step(out["x_smooth"], ref["x_smooth"]),
         "diagP_filt": rel_err_elementwise(out["diagP_filt"], ref["diagP_filt"]),
         "diagP_smooth": rel_err_elementwise(out["diagP_smooth"], ref["diagP_smooth"])}
    print(f"N=8196 m=306 T=300: float64 epoch {t_fp64:.1f} s ({prob.T / t_fp64:.3f} timesteps/s), mixed "
          f"float64-accurate solve {t_mix:.1f} s (including upload and plan); errors vs float64 GPU path: {e}")
    assert e["x_filt"] <= 1e-4 and e["x_smooth"] <= 1e-4
    assert e["diagP_filt"] <= 1e-3 and e["diagP_smooth"] <= 1e-3
