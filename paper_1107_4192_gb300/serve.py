"""Continuous-batching server for filter + smoother requests (epochs).

Requests (MEG epochs of different N, m, T) arrive over time.  The scheduler
admits a waiting request as soon as a slot is free and its device footprint
fits the memory budget, then runs it on its own CUDA stream from a worker
thread, so the kernels of concurrently admitted epochs overlap on the GPU.
Each admitted epoch keeps its filter state and covariance store on the device
for the whole request.

Admission charges a request 2 N^2 T 4 bytes (predicted and filtered float32
covariances for every step) plus the plan's workspace.  When that does not
fit but the plan can run within the free memory by keeping only checkpoints
of P_{t|t} and recomputing the rest forward during the smoother, the request
is admitted in that mode, charged what its plan actually allocates.  A request
that cannot fit even so into the whole budget is rejected.

Every epoch's computation is independent of the others (own plan, own
stream, deterministic kernels), so a result is bitwise the same alone and in
the mix.

Plans take their device memory from an arena the server reserves once
(kf_arena_reserve, the size of the budget): creating and destroying a plan
per request then makes no cudaMalloc / cudaFree call, whose device-wide
synchronisation would stall the other requests' streams.

Only marshalling and scheduling happen here; all arithmetic runs in the
library's CUDA kernels.
"""
from __future__ import annotations

import threading
import time
from dataclasses import dataclass, field
from typing import Dict, List, Optional

import numpy as np

from . import binding as B
from . import solver


@dataclass
class Request:
    rid: int
    arrival_s: float
    problem: object                     # synth.Problem, or a LazyProblem (built when admitted)
    prec: int = B.KF_PREC_MIXED_BF16X3
    solve_prec: Optional[int] = None    # None: float64-accurate smoothed mean on the mixed path, else float32
    joseph_every: int = 16

    def __post_init__(self):
        if self.solve_prec is None:
            self.solve_prec = B.KF_SOLVE_FP64_MEAN if self.prec == B.KF_PREC_MIXED_BF16X3 else B.KF_SOLVE_FP32


@dataclass
class Result:
    rid: int
    N: int
    m: int
    T: int
    arrival_s: float
    admitted_s: float = 0.0
    finished_s: float = 0.0
    charged_bytes: int = 0
    checkpoint_every: int = 1
    status: str = "ok"
    outputs: Optional[Dict[str, np.ndarray]] = None

    @property
    def latency_s(self):
        return self.finished_s - self.arrival_s

    @property
    def queue_s(self):
        return self.admitted_s - self.arrival_s


def admission_footprint(N: int, T: int) -> int:
    """2 N^2 T float32 words: the admission rule for one epoch."""
    return 2 * N * N * T * 4


def input_bytes(prob) -> int:
    """Device bytes of one request's float64 inputs (P0 dense, H, Y, x0, F, Q, R)."""
    N, m, T = prob.N, prob.m, prob.T
    b = 8 * (N * N + m * N + T * m + N)
    if prob.F is not None:
        b += 16 * prob.F.nnz + 8 * (N + 1)
    b += 8 * (1 if prob.q_kind == 0 else N if prob.q_kind == 1 else N * N)
    b += 8 * (1 if prob.r_kind == 0 else m if prob.r_kind == 1 else m * m)
    return b


@dataclass
class LazyProblem:
    """A request's shape, with its synthetic inputs built only when it is admitted (the inputs of
    a served request arrive with it; building them is the stand-in for receiving them)."""
    N: int
    m: int
    T: int
    identity_F: bool
    seed: int
    q_kind: int = 0
    r_kind: int = 1

    @property
    def f_kind(self):
        return B.KF_F_IDENTITY if self.identity_F else B.KF_F_CSR

    @property
    def nnz(self):
        return 0 if self.identity_F else _mesh_nnz(self.N)

    @property
    def F(self):
        return None if self.identity_F else _NnzOnly(self.nnz)

    def build(self):
        from . import synth
        return synth.mesh_problem(self.N, self.m, self.T, seed=self.seed, identity_F=self.identity_F)


@dataclass
class _NnzOnly:
    nnz: int


_NNZ = {}


def _mesh_nnz(N):
    if N not in _NNZ:
        from . import synth
        _NNZ[N] = synth.mesh_coupling(synth.hemisphere_mesh(N)).nnz
    return _NNZ[N]


def _kinds(prob):
    """(f_kind, nnz, q_kind, r_kind) of a problem, without building its arrays."""
    if prob.F is None:
        return B.KF_F_IDENTITY, 0, prob.q_kind, prob.r_kind
    return B.KF_F_CSR, prob.F.nnz, prob.q_kind, prob.r_kind


def plan_bytes(prob, req: Request, budget: int):
    """(status, bytes, checkpoint_every) of the plan this request would allocate within `budget`."""
    f_kind, nnz, q_kind, r_kind = _kinds(prob)
    d = B.make_desc(prob.N, prob.m, prob.T, f_kind, req.prec, req.solve_prec, q_kind, r_kind,
                    req.joseph_every, nnz, budget, 0, 0, 0)
    st, w, s, c = B.kf_plan_footprint(d)
    return st, w + s, c


class Server:
    """Admits requests as slots and memory free up; runs each on its own stream."""

    def __init__(self, budget_bytes: int = 160 * 10 ** 9, max_slots: int = 4, keep_outputs: bool = False,
                 device: str = "cuda", use_arena: bool = True):
        self.budget = int(budget_bytes)
        self.max_slots = max_slots
        self.keep_outputs = keep_outputs
        self.device = device
        self.use_arena = use_arena
        self._lock = threading.Lock()
        self._cv = threading.Condition(self._lock)
        self._in_use = 0
        self._active = 0
        self._arena_active = False

    def _charge(self, prob, req):
        """(bytes to reserve now, plan budget): bytes None = wait, -1 = never fits."""
        inputs = input_bytes(prob)
        free = self.budget - self._in_use - inputs
        if self._arena_active:
            # plans take their memory from the arena, whose free space the blocks of finished plans
            # can leave fragmented: a plan whose bytes fit in the largest free block always fits
            free = min(free, B.kf_arena_stats()[2])
        need_full = admission_footprint(prob.N, prob.T)
        st, full_bytes, c = plan_bytes(prob, req, 0)
        if max(need_full, full_bytes) <= free:
            return max(need_full, full_bytes) + inputs, 0
        if free > 0:
            st, ck_bytes, c = plan_bytes(prob, req, free)
            if st == B.KF_OK:
                return ck_bytes + inputs, free
        st, _, _ = plan_bytes(prob, req, self.budget - inputs)
        return (-1, 0) if st != B.KF_OK else (None, 0)

    def _worker(self, req: Request, res: Result, budget: int, t0: float):
        import torch
        prob = req.problem
        try:
            if isinstance(prob, LazyProblem):
                prob = prob.build()
            stream = torch.cuda.Stream()
            with torch.cuda.stream(stream):
                d = solver.upload(prob, self.device)
                plan = solver.Plan.for_inputs(d, prob.N, prob.m, prob.T, prec=req.prec, solve_prec=req.solve_prec,
                                              joseph_every=req.joseph_every, mem_budget_bytes=budget,
                                              stream=stream.cuda_stream)
                try:
                    res.checkpoint_every = B.kf_plan_footprint(plan.desc)[3]
                    xf, df = plan.filter(d)
                    xs, ds, _ = plan.smooth()
                    out = {"x_filt": xf.cpu().numpy(), "diagP_filt": df.cpu().numpy(),
                           "x_smooth": xs.cpu().numpy(), "diagP_smooth": ds.cpu().numpy()}
                    if self.keep_outputs:
                        res.outputs = out
                finally:
                    plan.close()
                stream.synchronize()
        except Exception as e:  # reported per request; the server keeps serving
            res.status = f"error: {e}"
        res.finished_s = time.perf_counter() - t0
        with self._cv:
            self._in_use -= res.charged_bytes
            self._active -= 1
            self._cv.notify_all()

    def run(self, requests: List[Request], time_scale: float = 1.0, admit_until_s: Optional[float] = None,
            progress=None, progress_every_s: float = 30.0) -> List[Result]:
        """Serves requests arriving at arrival_s * time_scale seconds after the start.  With
        admit_until_s, requests still waiting at that time are not admitted (status "not admitted")
        and the run ends when the admitted ones finish; progress(results) is called about every
        progress_every_s seconds."""
        reqs = sorted(requests, key=lambda r: r.arrival_s)
        results = {r.rid: Result(r.rid, r.problem.N, r.problem.m, r.problem.T, r.arrival_s * time_scale)
                   for r in reqs}
        threads = []
        arena = False
        if self.use_arena:
            # plans sub-allocate from one reservation; fall back to cudaMalloc if it cannot be made
            try:
                B.kf_arena_reserve(self.budget)
                arena = True
            except B.KfError:
                arena = False
        self._arena_active = arena
        t0 = time.perf_counter()
        pending: List[Request] = []
        i = 0
        last_progress = 0.0
        with self._cv:
            while i < len(reqs) or pending:
                now = time.perf_counter() - t0
                if progress is not None and now - last_progress >= progress_every_s:
                    last_progress = now
                    progress([results[r.rid] for r in reqs])
                if admit_until_s is not None and now >= admit_until_s:
                    for req in pending + reqs[i:]:
                        res = results[req.rid]
                        res.status = "not admitted: admission window closed"
                        res.admitted_s = res.finished_s = now
                    pending, i = [], len(reqs)
                    break
                while i < len(reqs) and reqs[i].arrival_s * time_scale <= now:
                    pending.append(reqs[i])
                    i += 1
                admitted_any = False
                for req in list(pending):          # first come, first served, skipping what does not fit
                    if self._active >= self.max_slots:
                        break
                    charge, budget = self._charge(req.problem, req)
                    if charge is None:
                        continue
                    pending.remove(req)
                    res = results[req.rid]
                    if charge < 0:
                        res.status = "rejected: does not fit the memory budget"
                        res.admitted_s = res.finished_s = now
                        continue
                    res.charged_bytes = charge
                    res.admitted_s = now
                    self._in_use += charge
                    self._active += 1
                    th = threading.Thread(target=self._worker, args=(req, res, budget, t0), daemon=True)
                    threads.append(th)
                    th.start()
                    admitted_any = True
                if admitted_any:
                    continue
                next_arrival = reqs[i].arrival_s * time_scale - now if i < len(reqs) else None
                timeout = 0.05 if next_arrival is None else max(0.0, min(next_arrival, 0.05))
                self._cv.wait(timeout=timeout)
        for th in threads:
            th.join()
        if arena:
            self._arena_active = False
            B.kf_arena_release()
        return [results[r.rid] for r in reqs]


def summarize(results: List[Result], wall_s: Optional[float] = None) -> dict:
    ok = [r for r in results if r.status == "ok"]
    lat = np.array([r.latency_s for r in ok]) if ok else np.zeros(1)
    steps = sum(r.T for r in ok)
    wall = wall_s if wall_s is not None else (max(r.finished_s for r in ok) - min(r.arrival_s for r in results)
                                              if ok else 0.0)
    return {"requests": len(results), "completed": len(ok),
            "rejected": sum(r.status.startswith("rejected") for r in results),
            "not_admitted": sum(r.status.startswith("not admitted") for r in results),
            "errors": sum(r.status.startswith("error") for r in results),
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "mean_queue_s": float(np.mean([r.queue_s for r in ok])) if ok else 0.0,
            "timesteps": int(steps), "wall_s": float(wall),
            "timesteps_per_s": float(steps / wall) if wall > 0 else 0.0,
            "recompute_requests": sum(r.checkpoint_every > 1 for r in ok),
            "error_messages": sorted({r.status for r in results if r.status.startswith("error")})[:4]}


def run_batch(problems, max_slots: int = 8, budget_bytes: int = 160 * 10 ** 9, prec=B.KF_PREC_MIXED_BF16X3,
              solve_prec=B.KF_SOLVE_FP32, keep_outputs: bool = False):
    """Many uneven epochs at once: all arrive at t = 0 and run concurrently, max_slots at a time."""
    reqs = [Request(i, 0.0, p, prec=prec, solve_prec=solve_prec) for i, p in enumerate(problems)]
    server = Server(budget_bytes, max_slots, keep_outputs)
    t0 = time.perf_counter()
    res = server.run(reqs)
    wall = time.perf_counter() - t0
    return res, summarize(res, wall)


def main(argv=None):
    """Replays the seeded Poisson request stream of the serving workload (20 req/s; N in {1024, 2048,
    5124, 8196}, m = 306, T ~ U{50..400}; F = I or mesh coupling by request parity) through the
    continuous-batching server with admission by footprint against the budget, and writes the
    summary (p50/p99 latency, timesteps/s, recompute count) as JSON."""
    import argparse
    import json

    import torch

    from . import build, synth
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--rate", type=float, default=20.0)
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--budget-gb", type=float, default=160.0)
    ap.add_argument("--out", default="")
    ap.add_argument("--admit-window-s", type=float, default=None,
                    help="admit no request after this many seconds (the rest are reported as not admitted)")
    args = ap.parse_args(argv)
    build.build()
    B.lib()
    torch.cuda.init()
    arrivals = synth.serving_arrivals(args.requests, args.rate, seed=4)
    reqs = [Request(i, t, LazyProblem(N, m, T, identity_F=(i % 2 == 0), seed=4000 + i))
            for i, (t, N, m, T) in enumerate(arrivals)]

    def progress(results):
        done = [r for r in results if r.finished_s > 0]
        if args.out and done:
            part = summarize(done, time.perf_counter() - t0)
            part["finished_so_far"] = len(done)
            with open(args.out + ".partial", "w") as f:
                f.write(json.dumps(part) + "\n")

    t0 = time.perf_counter()
    res = Server(int(args.budget_gb * 1e9), max_slots=args.slots).run(reqs, admit_until_s=args.admit_window_s,
                                                                        progress=progress)
    wall = time.perf_counter() - t0
    out = summarize(res, wall)
    by_n = {}
    for r in res:
        if r.status == "ok":
            by_n.setdefault(r.N, []).append(r.latency_s)
    out["p50_latency_s_by_N"] = {int(n): float(np.percentile(v, 50)) for n, v in sorted(by_n.items())}
    if args.admit_window_s is not None:
        out["admit_window_s"] = args.admit_window_s
    out["workload"] = (f"{args.requests} requests, Poisson arrivals at {args.rate} req/s over "
                       f"{arrivals[-1][0]:.1f} s, {args.slots} slots, budget {args.budget_gb} GB, mixed path "
                       f"(split-bf16 products, float64-class filter, float64-accurate smoothed-mean solve)")
    line = json.dumps(out)
    print(line, flush=True)
    if args.out:
        with open(args.out, "w") as f:
            f.write(line + "\n")


if __name__ == "__main__":
    main()
