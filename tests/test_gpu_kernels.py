"""Kernel-level GPU checks through the C ABI (include/kfmeg_kernels.h) against
plain float64 references of the same operation, on ragged shapes that span
several tiles and partial tails."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1107_4192_gb300 import binding as B  # noqa: E402
from paper_1107_4192_gb300 import synth  # noqa: E402

DT = {0: torch.float64, 1: torch.float32}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1107_4192_gb300 import build
    build.build()
    B.lib()


def _dev(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", DT[dt])


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("transB", [0, 1])
@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (7, 5, 3), (129, 65, 200), (300, 130, 77), (64, 64, 0),
                                   (256, 260, 128), (520, 132, 1028)])
def test_gemm(dtype, transB, M, N, K):
    rng = np.random.default_rng(M * 1000 + N * 10 + K)
    A = rng.standard_normal((M, K))
    Bm = rng.standard_normal((N, K)) if transB else rng.standard_normal((K, N))
    C0 = rng.standard_normal((M, N))
    alpha, beta = -0.7, 1.3
    ref = alpha * A @ (Bm.T if transB else Bm) + beta * C0
    dA, dB, dC = _dev(A, dtype), _dev(Bm, dtype), _dev(C0, dtype)
    B.kfx_gemm(dtype, transB, 0, M, N, K, alpha, dA, max(K, 1), dB, (K if transB else N) or 1, beta, dC, N)
    got = dC.double().cpu().numpy()
    tol = 1e-13 if dtype == 0 else 2e-5
    assert np.linalg.norm(got - ref) <= tol * max(np.linalg.norm(ref), 1e-300) * max(1, np.sqrt(K) / 4)


@pytest.mark.parametrize("transB", [0, 1])
@pytest.mark.parametrize("M,N", [(1000, 128), (77, 64), (3000, 96)])
def test_gemm_in_place_rows(transB, M, N):
    """C = C B (or C B^T) with the output overwriting A: the row transform that
    the blocked solves apply in place (N <= 128)."""
    rng = np.random.default_rng(M + N + transB)
    A = rng.standard_normal((M, N))
    Bm = rng.standard_normal((N, N))
    ref = A @ (Bm.T if transB else Bm)
    dA, dB = _dev(A, 1), _dev(Bm, 1)
    B.kfx_gemm(1, transB, 0, M, N, N, 1.0, dA, N, dB, N, 0.0, dA, N)
    got = dA.double().cpu().numpy()
    assert np.linalg.norm(got - ref) <= 2e-5 * np.linalg.norm(ref) * max(1, np.sqrt(N) / 4)


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("n,K", [(1, 3), (63, 64), (130, 20), (257, 129)])
def test_gemm_symmetric_mirror(dtype, n, K):
    rng = np.random.default_rng(n + K)
    A = rng.standard_normal((n, K))
    Bm = rng.standard_normal((n, K))
    S0 = rng.standard_normal((n, n))
    S0 = S0 + S0.T
    ref = A @ Bm.T + S0
    dC = _dev(S0, dtype)
    B.kfx_gemm(dtype, 1, 1, n, n, K, 1.0, _dev(A, dtype), K, _dev(Bm, dtype), K, 1.0, dC, n)
    got = dC.double().cpu().numpy()
    assert np.array_equal(got, got.T), "mirror must give an exactly symmetric result"
    low = np.tril(np.ones((n, n), bool))
    tol = 1e-13 if dtype == 0 else 2e-5
    assert np.abs(got - ref)[low].max() <= tol * np.abs(ref).max() * max(1, np.sqrt(K) / 4)


def _spd(n, seed, cond=50.0):
    rng = np.random.default_rng(seed)
    Qm, _ = np.linalg.qr(rng.standard_normal((n, n)))
    ev = np.geomspace(1.0, cond, n)
    return (Qm * ev) @ Qm.T


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("n,M", [(1, 4), (5, 3), (64, 70), (65, 65), (129, 31), (300, 257)])
def test_cholesky_and_right_solve(dtype, n, M):
    A = _spd(n, n * 7 + M)
    rng = np.random.default_rng(n)
    Bm = rng.standard_normal((M, n))
    dA, dB = _dev(A, dtype), _dev(Bm, dtype)
    st, fi = B.kfx_posv_right(dtype, n, dA, n, M, dB, n)
    assert st == 0 and fi == -1
    L = np.tril(dA.double().cpu().numpy())
    Lref = np.linalg.cholesky(A)
    X = dB.double().cpu().numpy()
    Xref = np.linalg.solve(A, Bm.T).T
    if dtype == 0:
        assert np.abs(L - Lref).max() <= 1e-13 * np.abs(Lref).max()
        assert np.linalg.norm(X - Xref) <= 1e-11 * np.linalg.norm(Xref)
    else:
        assert np.abs(L - Lref).max() <= 1e-5 * np.abs(Lref).max()
        assert np.linalg.norm(X - Xref) <= 1e-4 * np.linalg.norm(Xref)


@pytest.mark.parametrize("dtype", [0, 1])
def test_cholesky_reports_first_bad_pivot(dtype):
    n = 150
    A = _spd(n, 3)
    A[97, :] = 0.0
    A[:, 97] = 0.0  # pivot 97 becomes 0 (all earlier ones stay positive)
    dA = _dev(A, dtype)
    st, fi = B.kfx_posv_right(dtype, n, dA, n, 0, None, n)
    assert st == B.KF_ERR_NOT_PD and fi == 97


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("q_kind", [-1, 0, 1, 2])
def test_spmm_fpft(dtype, q_kind):
    N = 324
    neigh = synth.hemisphere_mesh(N)
    F = synth.mesh_coupling(neigh)
    rng = np.random.default_rng(1)
    Fd = np.zeros((N, N))
    for i in range(N):
        Fd[i, F.col[F.rowptr[i]:F.rowptr[i + 1]]] = F.val[F.rowptr[i]:F.rowptr[i + 1]]
    Fd[Fd != 0] *= rng.uniform(0.5, 1.0, size=(Fd != 0).sum())  # non-symmetric values
    vals = np.concatenate([Fd[i, F.col[F.rowptr[i]:F.rowptr[i + 1]]] for i in range(N)])
    A = rng.standard_normal((N, N))
    P = A @ A.T / N
    Q = {-1: None, 0: np.array([0.3]), 1: rng.uniform(0.1, 1, N), 2: P * 0.1}[q_kind]
    Qd = {-1: 0, 0: 0.3 * np.eye(N), 1: np.diag(Q) if q_kind == 1 else 0, 2: Q}[q_kind]
    ref = Fd @ P @ Fd.T + Qd
    ld = 384
    Pp = np.zeros((N, ld))
    Pp[:, :N] = P
    out = torch.zeros(N, ld, dtype=DT[dtype], device="cuda")
    tQ = None if Q is None else torch.from_numpy(np.ascontiguousarray(Q, np.float64)).cuda()
    B.kfx_spmm_fpft(dtype, N, torch.from_numpy(F.rowptr).cuda(), torch.from_numpy(F.col).cuda(),
                    torch.from_numpy(vals).cuda(), _dev(Pp, dtype), ld, out, ld, q_kind, tQ)
    got = out.double().cpu().numpy()[:, :N]
    tol = 1e-14 if dtype == 0 else 1e-6
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max()


def test_split_bf16():
    rng = np.random.default_rng(0)
    rows, cols, ld = 37, 100, 128
    A = rng.standard_normal((rows, cols)).astype(np.float32) * np.exp(rng.uniform(-5, 5, (rows, cols))).astype(np.float32)
    dA = torch.from_numpy(A).cuda()
    hi = torch.full((rows, ld), 7.0, dtype=torch.bfloat16, device="cuda")
    lo = torch.full((rows, ld), 7.0, dtype=torch.bfloat16, device="cuda")
    B.kfx_split_bf16(rows, cols, dA, cols, hi, lo, ld)
    h = hi.float().cpu().numpy()
    lw = lo.float().cpu().numpy()
    assert np.array_equal(h[:, :cols], torch.from_numpy(A).bfloat16().float().numpy())
    assert np.all(h[:, cols:] == 0) and np.all(lw[:, cols:] == 0)
    rel = np.abs(h[:, :cols] + lw[:, :cols] - A) / np.abs(A)
    assert rel.max() <= 2.0 ** -16


def _split_ref(X):
    """float64 values of the bf16 hi/lo planes of float32 X (round to nearest even)."""
    t = torch.from_numpy(np.ascontiguousarray(X, np.float32))
    hi = t.bfloat16().float()
    lo = (t - hi).bfloat16().float()
    return hi.double().numpy(), lo.double().numpy()


@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (256, 256, 128), (130, 300, 200), (385, 129, 640), (1, 1, 1)])
def test_tc_bf16x3_gemm(M, N, K):
    """tcgen05 split-bf16 product vs the exact float64 value of the same three bf16 products."""
    rng = np.random.default_rng(M + 7 * N + 13 * K)
    A = rng.standard_normal((M, K)).astype(np.float32)
    Bm = rng.standard_normal((N, K)).astype(np.float32)
    C0 = rng.standard_normal((M, N)).astype(np.float32)
    ah, al = _split_ref(A)
    bh, bl = _split_ref(Bm)
    exact = ah @ bh.T + ah @ bl.T + al @ bh.T
    ref = -1.5 * exact + 0.5 * C0.astype(np.float64)
    dC = torch.from_numpy(C0).cuda()
    B.kfx_gemm(2, 1, 0, M, N, K, -1.5, torch.from_numpy(A).cuda(), K, torch.from_numpy(Bm).cuda(), K, 0.5, dC, N)
    got = dC.double().cpu().numpy()
    # only the float32 accumulation order differs from `exact`
    assert np.abs(got - ref).max() <= 1e-5 * max(1.0, np.sqrt(K)) * np.abs(ref).max()
    # and the product is float32-accurate against the float64 product of the inputs
    full = -1.5 * A.astype(np.float64) @ Bm.astype(np.float64).T + 0.5 * C0
    assert np.linalg.norm(got - full) <= 1e-4 * np.linalg.norm(full)


@pytest.mark.parametrize("n,K", [(300, 64), (513, 320)])
def test_tc_bf16x3_symmetric(n, K):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, K)).astype(np.float32)
    Bm = rng.standard_normal((n, K)).astype(np.float32)
    S0 = rng.standard_normal((n, n)).astype(np.float32)
    S0 = S0 + S0.T
    dC = torch.from_numpy(S0).cuda()
    B.kfx_gemm(2, 1, 1, n, n, K, 1.0, torch.from_numpy(A).cuda(), K, torch.from_numpy(Bm).cuda(), K, 1.0, dC, n)
    got = dC.double().cpu().numpy()
    assert np.array_equal(got, got.T)
    ref = A.astype(np.float64) @ Bm.astype(np.float64).T + S0
    low = np.tril(np.ones((n, n), bool))
    assert np.abs(got - ref)[low].max() <= 1e-4 * np.abs(ref).max()


def _split3_ref(X):
    t = torch.from_numpy(np.ascontiguousarray(X, np.float32))
    out = []
    for _ in range(3):
        h = t.bfloat16().float()
        out.append(h.double().numpy())
        t = t - h
    return out


@pytest.mark.parametrize("transB", [1, 0])
@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (300, 257, 130), (70, 513, 384)])
def test_tc_bf16x6_gemm(transB, M, N, K):
    """Three-way split (six bf16 products): exact emulation, and float32-class accuracy."""
    rng = np.random.default_rng(M + N + K + transB)
    A = rng.standard_normal((M, K)).astype(np.float32)
    Bm = (rng.standard_normal((N, K)) if transB else rng.standard_normal((K, N))).astype(np.float32)
    Bnk = Bm if transB else Bm.T
    a = _split3_ref(A)
    b = _split3_ref(Bnk)
    exact = sum(a[i] @ b[j].T for i in range(3) for j in range(3) if i + j < 3)
    dC = torch.zeros(M, N, dtype=torch.float32, device="cuda")
    B.kfx_gemm(3, transB, 0, M, N, K, 1.0, torch.from_numpy(A).cuda(), K, torch.from_numpy(np.ascontiguousarray(Bm)).cuda(),
               K if transB else N, 0.0, dC, N)
    got = dC.double().cpu().numpy()
    assert np.abs(got - exact).max() <= 4e-6 * max(1.0, np.sqrt(K)) * np.abs(exact).max()
    # six products carry 24 bits of each operand and partial sums are promoted to float32
    # registers every 64-wide k-tile, so the product is float32-class (rounding ~6e-8)
    full = A.astype(np.float64) @ Bnk.astype(np.float64).T
    assert np.linalg.norm(got - full) <= 2e-6 * np.linalg.norm(full)


@pytest.mark.parametrize("dtype", [2, 3])
def test_tc_accumulation_bias(dtype):
    """Same-sign data, K = 8192: the tensor cores' float32 accumulation truncates, so the kernel
    promotes partial sums to float32 registers every k-tile.  The relative bias must stay small and
    independent of K (without promotion it grew to about -4.5e-5 at this K)."""
    rng = np.random.default_rng(0)
    rows = []
    for K in (512, 8192):
        A = rng.random((256, K)).astype(np.float32)
        Bm = rng.random((256, K)).astype(np.float32)
        ref = A.astype(np.float64) @ Bm.astype(np.float64).T
        dC = torch.zeros(256, 256, dtype=torch.float32, device="cuda")
        B.kfx_gemm(dtype, 1, 0, 256, 256, K, 1.0, torch.from_numpy(A).cuda(), K, torch.from_numpy(Bm).cuda(), K,
                   0.0, dC, 256)
        e = (dC.double().cpu().numpy() - ref) / ref
        rows.append((K, float(e.mean()), float(np.abs(e).max())))
        print(f"dtype {dtype} K {K}: mean relative error {e.mean():+.2e}, max {np.abs(e).max():.2e}")
    for K, mean, mx in rows:
        assert abs(mean) < 1e-6 and mx < 3e-6, (K, mean, mx)


def test_tc_wait_limit_timeout_then_recovery():
    """Failure detection of the tensor-core pipeline without a fault: with the pipeline waits
    limited to 1 ns the first waits run out, the kernel stops issuing, waits for the copies it
    already issued, frees its tensor memory and the entry point returns KF_ERR_TIMEOUT; with the
    default limit restored the same call succeeds and is correct."""
    rng = np.random.default_rng(3)
    M, N, K = 256, 256, 4096
    A = rng.standard_normal((M, K)).astype(np.float32)
    Bm = rng.standard_normal((N, K)).astype(np.float32)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(Bm).cuda()
    dC = torch.zeros(M, N, dtype=torch.float32, device="cuda")
    prev = B.kfx_tc_wait_limit(1)
    try:
        for _ in range(2):
            with pytest.raises(B.KfError) as e:
                B.kfx_gemm(3, 1, 0, M, N, K, 1.0, dA, K, dB, K, 0.0, dC, N)
            assert e.value.status == B.KF_ERR_TIMEOUT
    finally:
        B.kfx_tc_wait_limit(0)
    assert prev == 2_000_000_000
    B.kfx_gemm(3, 1, 0, M, N, K, 1.0, dA, K, dB, K, 0.0, dC, N)
    full = A.astype(np.float64) @ Bm.astype(np.float64).T
    assert np.linalg.norm(dC.double().cpu().numpy() - full) <= 2e-6 * np.linalg.norm(full)
