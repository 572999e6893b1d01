"""The allocation-free solve entry point (kfx_posv_right_static) against the
allocating one (kfx_posv_right), through the C ABI.

The static variant serves callers that cannot allocate device memory when the
solve runs; its scratch is a fixed device array shared by all calls, so two
calls in a row must not depend on what the previous call left behind.  This
file is named to be collected last.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1107_4192_gb300 import binding as B  # noqa: E402

DT = {0: torch.float64, 1: torch.float32}
TOL = {0: (1e-13, 1e-11), 1: (1e-5, 1e-4)}  # (factor, solution), as in the kernel tests


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1107_4192_gb300 import build
    build.build()
    B.lib()


def _spd(n, seed):
    rng = np.random.default_rng(seed)
    Qm, _ = np.linalg.qr(rng.standard_normal((n, n)))
    return (Qm * np.geomspace(1.0, 50.0, n)) @ Qm.T


def _solve(fn, dtype, A, Bm):
    n, M = A.shape[0], Bm.shape[0]
    dA = torch.from_numpy(A).to("cuda", DT[dtype])
    dB = torch.from_numpy(Bm).to("cuda", DT[dtype])
    st, fi = fn(dtype, n, dA, n, M, dB, n)
    return st, fi, np.tril(dA.double().cpu().numpy()), dB.double().cpu().numpy()


@pytest.mark.parametrize("dtype", [0, 1])
def test_static_matches_allocating_twice_in_a_row(dtype):
    for call, (n, M) in enumerate([(300, 257), (129, 40)]):  # two calls in a row, different sizes
        A = _spd(n, 10 * call + dtype)
        Bm = np.random.default_rng(call).standard_normal((M, n))
        st0, fi0, L0, X0 = _solve(B.kfx_posv_right, dtype, A, Bm)
        st1, fi1, L1, X1 = _solve(B.kfx_posv_right_static, dtype, A, Bm)
        assert st0 == st1 == 0 and fi0 == fi1 == -1
        tl, tx = TOL[dtype]
        assert np.abs(L1 - L0).max() <= tl * np.abs(L0).max()
        assert np.linalg.norm(X1 - X0) <= tx * np.linalg.norm(X0)


@pytest.mark.parametrize("dtype", [0, 1])
def test_static_reports_bad_pivot_then_recovers(dtype):
    n = 150
    A = _spd(n, 3)
    A[97, :] = 0.0
    A[:, 97] = 0.0
    st, fi, _, _ = _solve(B.kfx_posv_right_static, dtype, A, np.zeros((1, n)))
    assert st == B.KF_ERR_NOT_PD and fi == 97
    # the status word is cleared by the next call
    st, fi, L, _ = _solve(B.kfx_posv_right_static, dtype, _spd(n, 4), np.zeros((1, n)))
    assert st == 0 and fi == -1


def test_static_rejects_sizes_above_the_limit():
    n = 4097
    dA = torch.zeros(1, dtype=torch.float64, device="cuda")
    st, fi = B.kfx_posv_right_static(0, n, dA, n, 0, None, n)
    assert st == B.KF_ERR_ARG and fi == -1


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("n", [4096, 4000])
def test_static_at_the_size_limit(dtype, n):
    """n = 4096 fills the fixed scratch exactly (the diagonal-block inverses of both dtypes come to
    the whole array); 4000 leaves a ragged last block.  Small M keeps the solve cheap."""
    rng = np.random.default_rng(n + dtype)
    G = rng.standard_normal((n, n))
    A = G @ G.T / n + np.eye(n)
    Bm = rng.standard_normal((3, n))
    st0, fi0, L0, X0 = _solve(B.kfx_posv_right, dtype, A, Bm)
    st1, fi1, L1, X1 = _solve(B.kfx_posv_right_static, dtype, A, Bm)
    assert st0 == st1 == 0 and fi0 == fi1 == -1
    tl, tx = TOL[dtype]
    assert np.abs(L1 - L0).max() <= tl * np.abs(L0).max()
    assert np.linalg.norm(X1 - X0) <= tx * np.linalg.norm(X0)
