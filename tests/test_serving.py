"""Continuous-batching server: admission by footprint (host logic, CPU) and
identical results alone and in the mix (GPU)."""
import numpy as np
import pytest

from paper_1107_4192_gb300 import binding as B
from paper_1107_4192_gb300 import serve, synth


@pytest.fixture(scope="module")
def built():
    from paper_1107_4192_gb300 import build
    build.build()
    B.lib()


def test_admission_footprint_rule():
    assert serve.admission_footprint(8196, 400) == 2 * 8196 ** 2 * 400 * 4
    assert serve.admission_footprint(8196, 400) > 160e9  # must run in recompute mode
    assert serve.admission_footprint(1024, 50) < 1e9


def test_charge_full_checkpointed_and_rejected(built):
    prob = synth.random_walk_problem(512, 32, 40, seed=1)
    req = serve.Request(0, 0.0, prob)
    st, full, c = serve.plan_bytes(prob, req, 0)
    assert st == 0 and c == 1
    srv = serve.Server(budget_bytes=10 * full, max_slots=2)
    charge, budget = srv._charge(prob, req)
    assert charge >= full and budget == 0                      # full store fits
    srv = serve.Server(budget_bytes=int(0.7 * full) + serve.input_bytes(prob), max_slots=2)
    charge, budget = srv._charge(prob, req)
    assert charge is not None and charge > 0 and budget > 0    # admitted with checkpoints
    assert serve.plan_bytes(prob, req, budget)[2] > 1
    srv = serve.Server(budget_bytes=serve.input_bytes(prob) + 1000, max_slots=2)
    assert srv._charge(prob, req)[0] == -1                      # can never fit


def _requests(prec):
    probs = [synth.random_walk_problem(256, 32, 7, seed=1), synth.mesh_problem(324, 40, 6, seed=2),
             synth.random_walk_problem(384, 64, 9, seed=3), synth.mesh_problem(200, 20, 5, seed=4)]
    return [serve.Request(i, 0.01 * i, p, prec=prec, solve_prec=B.KF_SOLVE_FP32, joseph_every=4)
            for i, p in enumerate(probs)]


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [B.KF_PREC_MIXED_BF16X3, B.KF_PREC_FP64])
def test_alone_equals_mix(built, prec):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    alone = serve.Server(max_slots=1, keep_outputs=True).run(_requests(prec))
    mix = serve.Server(max_slots=4, keep_outputs=True).run(_requests(prec))
    for a, b in zip(alone, mix):
        assert a.status == b.status == "ok"
        for k in a.outputs:
            assert np.array_equal(a.outputs[k], b.outputs[k]), (a.rid, k)


@pytest.mark.gpu
def test_recompute_mode_under_a_small_budget(built):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    probs = [synth.mesh_problem(324, 40, 12, seed=5), synth.random_walk_problem(256, 32, 10, seed=6)]
    reqs = [serve.Request(i, 0.0, p, prec=B.KF_PREC_FP64) for i, p in enumerate(probs)]
    full = serve.Server(max_slots=2, keep_outputs=True).run(reqs)
    st, fb, _ = serve.plan_bytes(probs[0], reqs[0], 0)
    # the largest budget (in 2% steps below the full footprint) that forces checkpointing
    budget = next(int(f * fb) for f in np.arange(0.98, 0.3, -0.02)
                  if serve.plan_bytes(probs[0], reqs[0], int(f * fb))[0] == 0
                  and serve.plan_bytes(probs[0], reqs[0], int(f * fb))[2] > 1)
    tight = serve.Server(budget_bytes=budget + serve.input_bytes(probs[0]), max_slots=2,
                         keep_outputs=True).run(reqs)
    assert tight[0].checkpoint_every > 1
    for a, b in zip(full, tight):
        assert b.status == "ok"
        for k in a.outputs:  # float64 recomputation repeats the forward pass exactly
            assert np.array_equal(a.outputs[k], b.outputs[k]), k
    s = serve.summarize(tight)
    assert s["completed"] == 2 and s["recompute_requests"] >= 1


@pytest.mark.gpu
def test_mid_size_concurrent_equals_alone(built):
    """Six 1024..1536-wide epochs at once: wide enough that the solve runs its
    small products and leaves on the CUDA cores while other plans' kernels
    share the GPU, so a product whose CTAs read what a sibling CTA writes
    would show up here as a difference (or a failed factorisation)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    probs = [synth.mesh_problem(N, m, 10, seed=50 + i, identity_F=(i % 2 == 0))
             for i, (N, m) in enumerate([(1024, 64), (1152, 128), (1280, 64), (1408, 128), (1536, 64), (1024, 128)])]
    reqs = lambda: [serve.Request(i, 0.0, p, prec=B.KF_PREC_MIXED_BF16X3, solve_prec=B.KF_SOLVE_FP32)
                    for i, p in enumerate(probs)]
    alone = serve.Server(max_slots=1, keep_outputs=True).run(reqs())
    mix = serve.Server(max_slots=6, keep_outputs=True).run(reqs())
    for a, b in zip(alone, mix):
        assert a.status == b.status == "ok", (a.status, b.status)
        for k in a.outputs:
            assert np.array_equal(a.outputs[k], b.outputs[k]), (a.rid, k)


@pytest.mark.gpu
def test_arena_backs_plans_without_allocation(built):
    """Plans created after kf_arena_reserve take their buffers from the arena (in_use grows by the
    plan's footprint), return them on destroy (coalesced back to one free block), and compute
    the same result as a plan from cudaMalloc."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1107_4192_gb300 import solver
    prob = synth.mesh_problem(324, 40, 6, seed=2)
    ref = solver.run(prob, prec=B.KF_PREC_MIXED_BF16X3, solve_prec=B.KF_SOLVE_FP32, joseph_every=4)
    size = 4 * 10 ** 9
    B.kf_arena_reserve(size)
    try:
        r, u, f = B.kf_arena_stats()
        assert r > 0.99 * size and u == 0 and f == r
        out = solver.run(prob, prec=B.KF_PREC_MIXED_BF16X3, solve_prec=B.KF_SOLVE_FP32, joseph_every=4)
        d = solver.upload(prob)
        plan = solver.Plan.for_inputs(d, prob.N, prob.m, prob.T, prec=B.KF_PREC_MIXED_BF16X3,
                                      solve_prec=B.KF_SOLVE_FP32, joseph_every=4)
        _, u1, _ = B.kf_arena_stats()
        st, w, s, _ = B.kf_plan_footprint(plan.desc)
        assert u1 >= 0.9 * (w + s)
        plan.close()
        r2, u2, f2 = B.kf_arena_stats()
        assert u2 == 0 and f2 == r2
    finally:
        B.kf_arena_release()
    for k in ref:
        assert np.array_equal(ref[k], out[k]), k


@pytest.mark.parametrize("identity_F", [True, False])
def test_lazy_problem_charges_like_the_built_one(built, identity_F):
    lazy = serve.LazyProblem(600, 40, 30, identity_F=identity_F, seed=7)
    prob = lazy.build()
    assert (prob.N, prob.m, prob.T, prob.q_kind, prob.r_kind) == (600, 40, 30, lazy.q_kind, lazy.r_kind)
    assert (prob.F is None) == identity_F and (identity_F or prob.F.nnz == lazy.nnz)
    assert serve.input_bytes(lazy) == serve.input_bytes(prob)
    req = serve.Request(0, 0.0, lazy)
    for budget in (0, serve.input_bytes(prob) + 2 * 600 * 600 * 4 * 8):
        assert serve.plan_bytes(lazy, req, budget) == serve.plan_bytes(prob, req, budget)


def test_request_solve_default_follows_the_precision():
    p = synth.random_walk_problem(64, 8, 3, seed=1)
    assert serve.Request(0, 0.0, p).solve_prec == B.KF_SOLVE_FP64_MEAN
    assert serve.Request(0, 0.0, p, prec=B.KF_PREC_FP64).solve_prec == B.KF_SOLVE_FP32
    assert serve.Request(0, 0.0, p, solve_prec=B.KF_SOLVE_FP64_TC).solve_prec == B.KF_SOLVE_FP64_TC


def test_admission_window_and_progress(monkeypatch):
    """Requests still waiting when the admission window closes are reported as not admitted; the
    admitted ones finish; progress sees the results while the run goes on (fake worker, no GPU)."""
    import time as _time

    def fake_worker(self, req, res, budget, t0):
        _time.sleep(0.05)
        res.finished_s = _time.perf_counter() - t0
        with self._cv:
            self._in_use -= res.charged_bytes
            self._active -= 1
            self._cv.notify_all()

    monkeypatch.setattr(serve.Server, "_worker", fake_worker)
    monkeypatch.setattr(serve, "plan_bytes", lambda prob, req, budget: (0, 1000, 1))
    reqs = [serve.Request(i, 0.0 if i < 3 else 5.0, serve.LazyProblem(64, 8, 3, identity_F=True, seed=i))
            for i in range(6)]
    seen = []
    res = serve.Server(budget_bytes=10 ** 9, max_slots=1, use_arena=False).run(
        reqs, admit_until_s=0.12, progress=lambda rs: seen.append(sum(r.finished_s > 0 for r in rs)),
        progress_every_s=0.0)
    done = [r for r in res if r.status == "ok"]
    late = [r for r in res if r.status.startswith("not admitted")]
    assert 1 <= len(done) <= 3 and len(done) + len(late) == 6
    assert all(r.rid >= len(done) for r in late) and all(r.finished_s > 0 for r in done)
    assert seen and max(seen) <= len(done)
    summary = serve.summarize(res, 1.0)
    assert summary["completed"] == len(done) and summary["not_admitted"] == len(late)


def test_charge_respects_the_arena_largest_free_block(built, monkeypatch):
    """With plans in the arena, admission is bounded by its largest free block, not by the free
    total: a fragmented arena puts a request in recompute mode or makes it wait."""
    prob = synth.random_walk_problem(512, 32, 40, seed=1)
    req = serve.Request(0, 0.0, prob)
    full = serve.plan_bytes(prob, req, 0)[1]
    srv = serve.Server(budget_bytes=10 * full, max_slots=2)
    srv._arena_active = True
    monkeypatch.setattr(B, "kf_arena_stats", lambda: (10 * full, 0, 10 * full))
    charge, budget = srv._charge(prob, req)
    assert budget == 0 and charge >= full                       # contiguous space: full store
    monkeypatch.setattr(B, "kf_arena_stats", lambda: (10 * full, 0, int(0.7 * full)))
    charge, budget = srv._charge(prob, req)
    assert charge is not None and 0 < budget <= int(0.7 * full)  # fragmented: checkpointed
    assert serve.plan_bytes(prob, req, budget)[1] <= int(0.7 * full)
    monkeypatch.setattr(B, "kf_arena_stats", lambda: (10 * full, 0, 1000))
    assert srv._charge(prob, req)[0] is None                      # nothing fits now: wait
