"""The exact-slice tensor-core product and the float64-accurate inverse built on it, through the
C ABI (include/kfmeg_kernels.h).

 - kfx_gemm_exact against an independent numpy restatement of the slicing scheme (integer slices
   below each row's largest magnitude, exact integer level sums, one rounding at the end): the
   GPU must reproduce it to a few units in the last place, which pins the slicing, the exact
   accumulation and the scaling;
 - the same product against the true product of the float64 inputs (computed in extended
   precision) within the scheme's error bound;
 - kfx_spd_inverse (float32-class factor refined to float64 accuracy) against the float64
   CUDA-core solve (kfx_posv_right, itself checked against numpy) at N in {257, 1024, 2048}:
   the smoother-gain inverse of eqn 11 at float64 accuracy.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1107_4192_gb300 import binding as B  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1107_4192_gb300 import build
    build.build()
    B.lib()


def rne_shift(a, s):
    """a / 2^s rounded to nearest, ties to even, for int64 arrays."""
    return (a + (1 << (s - 1)) - 1 + ((a >> s) & 1)) >> s


def slices_ref(X, S):
    """Row exponents e (max |X[r]| < 2^e) and integer slices q_p with
    X[r] ~= 2^(e_r - 7) sum_p 2^(-8p) q_p[r]: the signed base-256 digits (rounded to nearest,
    ties to even) of X rounded to the grid 2^(e_r - 7 - 8(S - 1))."""
    X = np.asarray(X, np.float64)
    mx = np.abs(X).max(axis=1)
    e = np.where(mx > 0, np.frexp(mx)[1], 0).astype(np.int64)
    Xi = np.rint(np.ldexp(X, (7 + 8 * (S - 1) - e)[:, None])).astype(np.int64)
    qs = []
    for p in range(S):
        sp = 8 * (S - 1 - p)
        q = rne_shift(Xi, sp) if sp > 0 else Xi.copy()
        assert np.abs(q).max(initial=0) <= 128
        Xi = Xi - (q << sp)
        qs.append(q)
    return e, qs


def exact_sliced_product(A, Bm, L):
    """Correctly rounded value of the sliced product keeping slice levels < L."""
    ea, qa = slices_ref(A, L)
    eb, qb = slices_ref(Bm, L)
    M, N = A.shape[0], Bm.shape[0]
    total = np.zeros((M, N), dtype=object)
    for lvl in range(L):
        V = sum(qa[a] @ qb[lvl - a].T for a in range(lvl + 1))  # exact int64
        total = total + V.astype(object) * (1 << (8 * (L - 1 - lvl)))
    out = np.empty((M, N))
    for i in range(M):
        for j in range(N):
            out[i, j] = math.ldexp(float(total[i, j]), int(ea[i] + eb[j]) - 14 - 8 * (L - 1))
    return out, ea, eb


@pytest.mark.parametrize("levels", [4, 5, 6, 7])
@pytest.mark.parametrize("M,N,K", [(130, 70, 300), (256, 192, 1024), (1, 1, 1), (129, 65, 33), (70, 130, 3000)])
def test_exact_product_matches_the_scheme(levels, M, N, K):
    rng = np.random.default_rng(M + N + K + levels)
    A = rng.standard_normal((M, K)) * np.exp(rng.uniform(-4, 4, (M, 1))) * np.exp(rng.uniform(-3, 3, (M, K)))
    Bm = rng.standard_normal((N, K)) * np.exp(rng.uniform(-4, 4, (N, 1)))
    ref, ea, eb = exact_sliced_product(A, Bm, levels)
    C = torch.zeros(M, N, dtype=torch.float64, device="cuda")
    B.kfx_gemm_exact(levels, M, N, K, 1.0, torch.from_numpy(A).cuda(), K, torch.from_numpy(Bm).cuda(), K, 0.0, 0.0,
                     C, N)
    got = C.cpu().numpy()
    # two roundings (the 64-bit level sums to float64) against one: a few ulp of the tile scale
    scale = np.ldexp(1.0, (ea[:, None] + eb[None, :]).astype(np.int64))
    assert np.all(np.abs(got - ref) <= 2.0 ** -50 * scale * max(1, K) ** 0.0 + 4 * np.spacing(np.abs(ref)))


@pytest.mark.parametrize("levels", [4, 5, 6, 7])
def test_exact_product_accuracy_and_epilogue(levels):
    """Against the true product (extended precision); alpha, beta and the delta on the diagonal."""
    rng = np.random.default_rng(7 + levels)
    M, N, K = 200, 200, 700
    A = rng.standard_normal((M, K))
    Bm = rng.standard_normal((N, K))
    C0 = rng.standard_normal((M, N))
    true = (A.astype(np.longdouble) @ Bm.astype(np.longdouble).T).astype(np.longdouble)
    ref = (-0.5 * true + 2.0 * C0.astype(np.longdouble) + np.eye(M, dtype=np.longdouble) * 3.0).astype(np.float64)
    C = torch.from_numpy(C0.copy()).cuda()
    B.kfx_gemm_exact(levels, M, N, K, -0.5, torch.from_numpy(A).cuda(), K, torch.from_numpy(Bm).cuda(), K, 2.0, 3.0,
                     C, N)
    got = C.cpu().numpy()
    bound = 2.0 ** (5 - 8 * levels) * K * np.abs(A).max(1)[:, None] * np.abs(Bm).max(1)[None, :] * 0.5
    err = np.abs(got - ref)
    print(f"levels {levels}: max error / bound = {(err / bound).max():.3f}")
    assert np.all(err <= bound + 4 * np.spacing(np.abs(ref)))


def test_exact_product_float32_operands():
    rng = np.random.default_rng(3)
    M, N, K = 150, 90, 260
    A = rng.standard_normal((M, K)).astype(np.float32)
    Bm = rng.standard_normal((N, K)).astype(np.float32)
    ref, _, _ = exact_sliced_product(A.astype(np.float64), Bm.astype(np.float64), 7)
    C = torch.zeros(M, N, dtype=torch.float64, device="cuda")
    B.kfx_gemm_exact(7, M, N, K, 1.0, torch.from_numpy(A).cuda(), K, torch.from_numpy(Bm).cuda(), K, 0.0, 0.0, C, N)
    assert np.abs(C.cpu().numpy() - ref).max() <= 1e-13 * np.abs(ref).max()


def spd32(n, cond, seed):
    """float32 SPD matrix with eigenvalues spread geometrically over [1/cond, 1] (the range of a
    smoother prediction P_{t+1|t} = P_{t|t} + Q with Q = 1e-2 I and P0 = I has cond <= ~100)."""
    rng = np.random.default_rng(seed)
    Qm, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = (Qm * np.geomspace(1.0 / cond, 1.0, n)) @ Qm.T
    A = 0.5 * (A + A.T)
    return A.astype(np.float32)


@pytest.mark.parametrize("n,cond", [(257, 100.0), (1024, 100.0), (2048, 100.0), (4096, 100.0), (1024, 1000.0)])
def test_refined_inverse_is_float64_accurate(n, cond):
    A = spd32(n, cond, n)
    dA = torch.from_numpy(A).cuda()
    # float64 CUDA-core reference: Cholesky + two triangular solves with B = I
    A64 = torch.from_numpy(A.astype(np.float64)).cuda()
    X64 = torch.eye(n, dtype=torch.float64, device="cuda")
    st, _ = B.kfx_posv_right(0, n, A64, n, n, X64, n)
    assert st == 0
    X64 = X64.cpu().numpy()
    Xnp = np.linalg.inv(A.astype(np.float64))
    assert np.linalg.norm(X64 - Xnp) <= 1e-12 * np.linalg.norm(Xnp) * cond / 100
    errs = {}
    for mode in (1, 2):
        X = torch.zeros(n, n, dtype=torch.float64, device="cuda")
        st, fi = B.kfx_spd_inverse(mode, n, dA, n, X, n)
        assert st == 0 and fi == -1
        Xg = X.cpu().numpy()
        errs[mode] = np.linalg.norm(Xg - X64) / np.linalg.norm(X64)
    print(f"n {n} cond {cond:g}: float32-class {errs[1]:.2e}, refined {errs[2]:.2e} (vs float64 solve)")
    assert errs[1] <= 1e-3
    assert errs[2] <= 1e-12 * cond / 100


def test_refined_inverse_reports_not_pd():
    n = 300
    A = spd32(n, 50.0, 1).astype(np.float64)
    A[150, :] = 0.0
    A[:, 150] = 0.0
    X = torch.zeros(n, n, dtype=torch.float64, device="cuda")
    st, fi = B.kfx_spd_inverse(2, n, torch.from_numpy(A.astype(np.float32)).cuda(), n, X, n)
    assert st == B.KF_ERR_NOT_PD and fi == 150


def test_exact_product_non_finite_rows_give_nan():
    """A NaN or infinity in a row of A makes that output row NaN (and no other)."""
    rng = np.random.default_rng(11)
    M, N, K = 40, 30, 50
    A = rng.standard_normal((M, K))
    Bm = rng.standard_normal((N, K))
    A[3, 7] = np.nan
    A[9, 0] = np.inf
    C = torch.zeros(M, N, dtype=torch.float64, device="cuda")
    B.kfx_gemm_exact(5, M, N, K, 1.0, torch.from_numpy(A).cuda(), K, torch.from_numpy(Bm).cuda(), K, 0.0, 0.0, C, N)
    got = C.cpu().numpy()
    bad = np.zeros(M, bool)
    bad[[3, 9]] = True
    assert np.all(np.isnan(got[bad])) and np.all(np.isfinite(got[~bad]))


def test_exact_product_wait_limit_timeout_then_recovery():
    """Failure detection of the exact-slice pipeline without a fault: with the pipeline waits
    limited to 1 ns the gate, MMA, TMA and epilogue roles stop at their first unmet wait, the
    kernel waits for what it already issued, frees its tensor memory and the entry point returns
    KF_ERR_TIMEOUT; with the default limit restored the same call matches the scheme."""
    rng = np.random.default_rng(11)
    M, N, K = 256, 128, 2048
    A = rng.standard_normal((M, K))
    Bm = rng.standard_normal((N, K))
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(Bm).cuda()
    C = torch.zeros(M, N, dtype=torch.float64, device="cuda")
    prev = B.kfx_tc_wait_limit(1)
    try:
        for _ in range(2):
            with pytest.raises(B.KfError) as e:
                B.kfx_gemm_exact(7, M, N, K, 1.0, dA, K, dB, K, 0.0, 0.0, C, N)
            assert e.value.status == B.KF_ERR_TIMEOUT
    finally:
        B.kfx_tc_wait_limit(0)
    assert prev == 2_000_000_000
    B.kfx_gemm_exact(7, M, N, K, 1.0, dA, K, dB, K, 0.0, 0.0, C, N)
    ref, ea, eb = exact_sliced_product(A, Bm, 7)
    scale = np.ldexp(1.0, (ea[:, None] + eb[None, :]).astype(np.int64))
    assert np.all(np.abs(C.cpu().numpy() - ref) <= 2.0 ** -50 * scale + 4 * np.spacing(np.abs(ref)))
