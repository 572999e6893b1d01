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
