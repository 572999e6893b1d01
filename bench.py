"""Throughput of the Kalman filter + fixed-interval smoother on one GB300.

Workload: N = 8196 sources, m = 306 sensors, T = 300 time steps, random-walk
dynamics (F = I), Q = 1e-2 I, R = diag U(0.5, 2), P0 = I, synthetic lead field
and patch sources (seed 2).  One step = one whole epoch: the forward filter
over all T steps and the backward smoother over T - 1 steps.  The metric is
KF+FIS timesteps/s (T per epoch), with algorithmic TFLOP/s beside it.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
               [--prec mixed|fp32|fp64] [--solve fp64tc|fp64mean|fp32|fp64]

Multi-GPU (torchrun): every rank runs its own independent epoch (replicas;
the recursion in t is sequential and the epochs share nothing), the timed
region is bracketed by a barrier and device synchronisation, and the
slowest rank's time is used.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "KF+FIS timesteps/s & TFLOP/s at N=8196,m=306 vs FP64 plain; serve p50/p99"
N_SRC, M_SENS, T_STEPS = 8196, 306, 300


def flops_per_timestep(N, m):
    """Operation count of one filter step plus one smoother step in the method's standard form
    (the count the paper's cost discussion and the scope table use; an "equivalent" rate).

    filter:   U^T = P H^T (2mN^2), S = H U^T (2m^2N), Cholesky of S (m^3/3),
              K = U^T S^{-1} (2m^2N), P - K U (2mN^2)
    smoother: Cholesky of P_{t+1|t} (N^3/3), two triangular solves with N
              right-hand sides (2N^3), W = J D (2N^3), P + W J^T on the lower
              triangle (N^2 (N+1)), mean (2N^2)
    """
    filt = 4 * m * N * N + 4 * m * m * N + m ** 3 / 3
    smooth = N ** 3 / 3 + 2 * N ** 3 + 2 * N ** 3 + N * N * (N + 1) + 2 * N * N
    return filt + smooth, smooth, filt


def executed_flops_per_timestep(N, m, joseph_every, refine_iters=0):
    """Flops the F = I path with a scalar Q actually executes per time step (each split-bf16
    product counted once, as one product of its float32 or float64 operands).

    filter:   U^T = P H^T (2mN^2), S = H U^T (2m^2N), Cholesky of S (m^3/3), Z = U^T L^{-T}
              (m^2N), P - Z Z^T on the lower triangle (mN^2); every k-th step the Joseph form
              instead: K = Z L^{-1} (m^2N), V = U^T - K S/2 (2m^2N), rank-2m product (2mN^2)
    smoother: Cholesky of P_{t+1|t} (N^3/3), triangular inverse W = L^{-1} (N^3/3),
              W^T W with J = I - Q W^T W in its epilogue (N^3/3, lower triangle), W = J D
              (2N^3), P + W J^T (N^3, lower triangle), mean (2N^2); each refinement iteration
              of the inverse: residual I - P X (2N^3) and correction X + X R (N^3, symmetric)
    """
    filt = 2 * m * N * N + 2 * m * m * N + m ** 3 / 3 + m * m * N + m * N * N
    if joseph_every:
        filt += (3 * m * m * N + m * N * N) / joseph_every
    smooth = N ** 3 + 2 * N ** 3 + N ** 3 + 2 * N * N + refine_iters * 3 * N ** 3
    return filt + smooth


def smoother_gemm_flops_per_launch(N):
    """Average algorithmic flops of one smoother product launch (W = J D, then W J^T lower)."""
    return (2 * N ** 3 + N * N * (N + 1)) / 2


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
        "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.file = None

    def __enter__(self):
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"], stdout=self.file,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        self.file.flush()

    def summary(self):
        rows = []
        try:
            with open(self.file.name) as f:
                for line in f:
                    parts = [x.strip() for x in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
        finally:
            os.unlink(self.file.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        power = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(power) if power else None}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="mixed", choices=["mixed", "fp32", "fp64"])
    ap.add_argument("--solve", default="fp64tc", choices=["fp32", "fp64", "fp64tc", "fp64mean"],
                    help="smoother-gain solve: fp64tc = float64-accurate on the tensor cores (float32-class "
                         "factor + Newton steps with exact-slice residuals; the workload's float64 smoother "
                         "solve), fp64mean = the smoothed mean's solve refined to float64 accuracy, fp32 = "
                         "float32 class, fp64 = float64 on the CUDA cores")
    ap.add_argument("--no-solve-variants", action="store_true",
                    help="skip the whole-epoch rates of the other tensor-core solve modes")
    ap.add_argument("--T", type=int, default=T_STEPS, help="time steps per epoch (the workload uses 300)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-plain", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--serve-requests", type=int, default=12,
                    help="requests of the Poisson serving stream to replay (0 = skip)")
    ap.add_argument("--batch-epochs", type=int, default=64, help="uneven epochs of the batched workload (0 = skip)")
    ap.add_argument("--config1-prefix", type=int, default=10,
                    help="time steps of the N=5124 mesh epoch run in float64 and float32 (0 = skip the config 1 leg)")
    ap.add_argument("--no-config2-mesh", action="store_true",
                    help="skip the N=8196 mesh-F epoch that runs with checkpoint recomputation under 160 GB")
    return ap.parse_args()


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_oracle_timestep(prob, T_sample=2):
    """Times the CPU oracle as it stands: T_sample filter steps then one smoother step."""
    from oracle import kf_oracle as ko
    N = prob.N
    F = np.eye(N)
    Q = ko.dense_cov(prob.q_kind, prob.Q, N)
    R = ko.dense_cov(prob.r_kind, prob.R, prob.m)
    P0 = prob.p0_scale * np.eye(N)
    t0 = time.perf_counter()
    filt = ko.kalman_filter(F, Q, prob.H, R, prob.Y[:T_sample], prob.x0, P0)
    t1 = time.perf_counter()
    ko.rts_smoother(F, filt)
    t2 = time.perf_counter()
    per_step = (t1 - t0) / T_sample + (t2 - t1) / (T_sample - 1)
    return per_step, f"{T_sample} filter steps + {T_sample - 1} smoother step of the N={N}, m={prob.m} workload " \
                     f"(float64 numpy oracle); rate = 1 / (filter step + smoother step)"


_CFG0_ORACLE = """
import sys, time
import numpy as np
sys.path.insert(0, {root!r})
from oracle import kf_oracle as ko
from paper_1107_4192_gb300 import synth
p = synth.config0()
F = np.eye(p.N)
Q = ko.dense_cov(p.q_kind, p.Q, p.N)
R = ko.dense_cov(p.r_kind, p.R, p.m)
P0 = p.p0_scale * np.eye(p.N)
ts = []
for _ in range(3):
    t0 = time.perf_counter()
    ko.kf_fis(F, Q, p.H, R, p.Y, p.x0, P0)
    ts.append(time.perf_counter() - t0)
print(sorted(ts)[1])
"""


def config0_sample(B, solver, synth, torch):
    """Config 0 (N = 384, m = 64, T = 40) in full: the float64 GPU path through the public API
    (plan, upload, filter, smoother, download) and the CPU oracle on one core and on all host
    cores, each the median of 3 runs."""
    prob = synth.config0()
    solver.run(prob, prec=B.KF_PREC_FP64)
    ts = []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        solver.run(prob, prec=B.KF_PREC_FP64)
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
    out = {"workload": "N384_m64_T40 (config 0)", "unit": "timesteps/s",
           "gpu_fp64_api": prob.T / sorted(ts)[1]}
    root = os.path.dirname(os.path.abspath(__file__))
    single = {k: "1" for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS")}
    for name, extra in (("cpu_oracle_1core", single), ("cpu_oracle_all_cores", {})):
        env = {k: v for k, v in os.environ.items() if k not in single}
        env.update(extra)
        r = subprocess.run([sys.executable, "-c", _CFG0_ORACLE.format(root=root)], capture_output=True, text=True,
                           env=env, timeout=600)
        out[name] = prob.T / float(r.stdout.strip().splitlines()[-1]) if r.returncode == 0 else None
    out["host_cores"] = os.cpu_count()
    return out


def host_threads():
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        n = max((i.get("num_threads", 0) for i in info), default=0)
        if n:
            return n
    except Exception:
        pass
    return os.cpu_count() or 1


def run_reference(args, world, rank):
    """The oracle timed on the host cores, same workload and metric (rank 0 only)."""
    if rank != 0:
        return
    from paper_1107_4192_gb300 import synth
    prob = synth.config2(T=2)
    for _ in range(args.warmup):
        cpu_oracle_timestep(prob)
    times = [cpu_oracle_timestep(prob)[0] for _ in range(args.steps)]
    sample = (f"per step: 2 filter steps + 1 smoother step of the N={N_SRC}, m={M_SENS} workload (float64 numpy "
              f"oracle); rate = 1 / (filter step + smoother step)")
    per = float(np.mean(times))
    value = 1.0 / per
    line = {"metric": METRIC, "value": value, "unit": "timesteps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": prob.name.replace("T2", f"T{T_STEPS}"), "N": N_SRC, "m": M_SENS, "T": T_STEPS},
            "cpu_baseline": {"value": value, "unit": "timesteps/s", "cores": host_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "timesteps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    import torch
    import torch.distributed as dist

    from paper_1107_4192_gb300 import binding as B
    from paper_1107_4192_gb300 import build, solver, synth

    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    build.build()
    B.lib()
    prec = {"mixed": B.KF_PREC_MIXED_BF16X3, "fp32": B.KF_PREC_FP32, "fp64": B.KF_PREC_FP64}[args.prec]
    solve = {"fp32": B.KF_SOLVE_FP32, "fp64": B.KF_SOLVE_FP64, "fp64tc": B.KF_SOLVE_FP64_TC,
             "fp64mean": B.KF_SOLVE_FP64_MEAN}[args.solve]
    T = args.T
    prob = synth.config2(T=T)
    d = solver.upload(prob)
    stream = torch.cuda.current_stream()
    plan = solver.Plan.for_inputs(d, prob.N, prob.m, T, prec=prec, solve_prec=solve,
                                  joseph_every=16 if args.prec == "mixed" else 0, stream=stream.cuda_stream)
    outs = {k: torch.empty(T, prob.N, dtype=torch.float64, device="cuda") for k in ("xf", "df", "xs", "ds")}

    def epoch():
        B.kf_filter(plan.handle, d.F, d.F_rowptr, d.F_col, d.Q, d.H, d.R, d.Y, d.x0, d.P0, outs["xf"], outs["df"])
        B.fis_smooth(plan.handle, outs["xs"], outs["ds"])

    for _ in range(args.warmup):
        epoch()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    B.kf_plan_profile(plan.handle, True)
    launches0 = B.kf_plan_launch_count(plan.handle)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            epoch()
        ev1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    launches = B.kf_plan_launch_count(plan.handle) - launches0
    prof = {c: B.kf_plan_profile_read(plan.handle, c) for c in range(10)}
    B.kf_plan_profile(plan.handle, False)
    if world > 1:
        t = torch.tensor([elapsed], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed = float(t.item())
    clocks = clk.summary()

    # end to end through the host-buffer entry point (inputs from pinned host memory, outputs back)
    h = solver.host_inputs(prob)
    pin = lambda a: None if a is None else torch.from_numpy(a).pin_memory()
    hin = {k: pin(h[k]) for k in ("F", "F_rowptr", "F_col", "Q", "H", "R", "Y", "x0", "P0")}
    hout = {k: torch.empty(T, prob.N, dtype=torch.float64).pin_memory() for k in ("xf", "df", "xs", "ds")}
    h2d = sum(v.numel() * v.element_size() for v in hin.values() if v is not None)
    d2h = sum(v.numel() * v.element_size() for v in hout.values())
    e2e_steps = max(1, args.e2e_steps)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        B.kf_solve_host(plan.handle, hin["F"], hin["F_rowptr"], hin["F_col"], hin["Q"], hin["H"], hin["R"], hin["Y"],
                        hin["x0"], hin["P0"], hout["xf"], hout["df"], hout["xs"], hout["ds"])
    e2e_time = (time.perf_counter() - t0) / e2e_steps
    if world > 1:
        t = torch.tensor([e2e_time], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_time = float(t.item())
    plan.close()

    N, m = prob.N, prob.m
    total_f, smooth_f, filt_f = flops_per_timestep(N, m)
    value = world * args.steps * T / elapsed
    ms_per_step = elapsed / args.steps * 1e3
    peaks, peak_src = load_peaks()

    # Roofline of the smoother's N x N covariance products (W = J D and P + W J^T): in the mixed
    # mode these are the tcgen05 split-bf16 kernel launches timed alone (class 7); otherwise the
    # phase of the same two products on the CUDA cores.  `achieved` counts each product once
    # (its algorithmic flops); the bf16 operations the tensor cores issue are three per product,
    # reported separately as the tensor-pipe fraction.
    if args.prec == "mixed" and prof[7][0] > 0:
        n_l, ms_l = prof[7]
        kname = "tc_gemm_kernel<256,2> (split-bf16 W = J D, P + W J^T)"
        roof = {"bound": "tensor", "peak": peaks["bf16_tflops_sustained"], "unit": "TFLOP/s",
                "peak_note": "bf16_tflops_sustained (measured), the dtype the tensor cores multiply in"}
    else:
        n_l, ms_l = prof[2]
        kname = "gemm_simt (W = J D, P + W J^T)"
        alu = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        roof = {"bound": "alu", "peak": alu if args.prec == "fp32" else 1.25, "unit": "TFLOP/s",
                "peak_note": "152 SMs x 128 FP32 lanes x 2 x max SM clock" if args.prec == "fp32" else
                "FP64 nominal 1.25 TFLOP/s"}
    avg_s = ms_l / 1e3 / max(n_l, 1)
    achieved = smoother_gemm_flops_per_launch(N) / avg_s / 1e12
    # DRAM bytes of one launch of that kernel at N = 8196 (dram__bytes_read.sum + dram__bytes_write.sum,
    # one ncu --set full capture of W = J D at t = 2 of the T = 3 run: 2.556e9 read + 0.280e9 written)
    traffic = 2.836e9 if args.prec == "mixed" and prof[7][0] > 0 and N == 8196 else None
    roof.update({"kernel": kname, "achieved": achieved, "frac": achieved / roof["peak"], "traffic": traffic,
                 "peak_source": peak_src, "launches": n_l, "avg_launch_ms": avg_s * 1e3,
                 "work_per_launch": f"(2 N^3 + N^2 (N+1)) / 2 flops, N = {N}"})
    if roof["bound"] == "tensor":
        roof["tensor_pipe_frac"] = 3 * achieved / roof["peak"]
        roof["tensor_pipe_note"] = "three bf16 products issued per split-bf16 product: 3 x achieved / peak"
    # the smoother-gain solve: Cholesky + triangular inverse of P_{t+1|t} (2 N^3 / 3 per step)
    # against the same measured bf16 peak (its large products run on the tensor cores)
    solve_ms = prof[5][1] / max(prof[5][0], 1)
    roof_solve = {"phase": "solve_factor (Cholesky + inverse of P_{t+1|t})", "bound": "tensor",
                  "achieved": (2 * N ** 3 / 3) / (solve_ms / 1e3) / 1e12 if solve_ms > 0 else None,
                  "peak": peaks["bf16_tflops_sustained"], "unit": "TFLOP/s", "peak_source": peak_src,
                  "ms_per_step": solve_ms, "work_per_step": f"2 N^3 / 3 flops, N = {N}"}
    if roof_solve["achieved"] is not None:
        roof_solve["frac"] = roof_solve["achieved"] / roof_solve["peak"]
    names = {0: "filter_update", 1: "innovation", 2: "smoother_gemm", 3: "smoother_solve", 4: "predict",
             5: "solve_factor", 6: "solve_gain", 7: "smoother_gemm_kernel", 8: "solve_refine",
             9: "refine_exact_kernel"}
    roof_smoother = roof
    # With the float64-accurate solve the dominant kernel is the exact-slice residual product
    # (I - P X_0 with 5 slice levels = 15 bf16 products, then I - P X_1 with 7 levels = 28), each
    # launch timed alone (class 9).  Its tensor work is the bf16 products it issues; the float64
    # product it delivers (2 N^3 per launch) is reported beside it against the float64 peak.
    if prof[9][0] > 0 and prof[9][1] > prof[7][1]:
        n_x, ms_x = prof[9]
        pairs_per_step, launches_per_step = 15 + 28, 2
        steps_x = n_x / launches_per_step
        issued = pairs_per_step * 2 * N ** 3 * steps_x
        t_x = ms_x / 1e3
        roof = {"bound": "tensor", "kernel": "oz_gemm_kernel<5>, oz_gemm_kernel<7> (exact-slice I - P X)",
                "achieved": issued / t_x / 1e12, "peak": peaks["bf16_tflops_sustained"], "unit": "TFLOP/s",
                "peak_source": peak_src,
                "peak_note": "bf16_tflops_sustained (measured): the products are bf16 slice products",
                # DRAM bytes of one oz_gemm_kernel<7> launch at N = 8196 (dram__bytes_read.sum +
                # dram__bytes_write.sum, one ncu capture of the T = 3 run: 38.14e9 read + 0.56e9
                # written); the 5-level launch streams 5/7 of the slice planes
                "traffic": 38.70e9 if N == 8196 else None,
                "traffic_note": "per oz_gemm_kernel<7> launch; the operand planes are re-read from DRAM by "
                                "every 8-row-tile group (20x the 1.9 GB of planes), at 23% of HBM bandwidth",
                "launches": n_x, "avg_launch_ms": ms_x / max(n_x, 1),
                "work_per_launch": f"(15 or 28) x 2 N^3 bf16 flops, N = {N} (levels 5 and 7)",
                "fp64_equivalent_tflops": launches_per_step * 2 * N ** 3 * steps_x / t_x / 1e12,
                "fp64_equivalent_note": "2 N^3 float64-accurate flops per launch, vs 1.25 TFLOP/s nominal "
                                        "float64 of this GPU",
                "mma_shape_note": "per k-step and A slice, one 128 x (64 run) x 16 MMA per run of up to four "
                                  "slice levels whose TMEM accumulators are adjacent (13.5 MMAs per k-step at "
                                  "7 levels); probe: N = 64 runs at 67% of the bf16 rate, N = 256 at 100%"}
        roof["frac"] = roof["achieved"] / roof["peak"]

    line = {"metric": METRIC, "value": value, "unit": "timesteps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": {"mixed": "bf16x3+f32+f64", "fp32": "f32", "fp64": "f64"}[args.prec] +
                     ("" if args.prec == "fp64" else f"/solve-{args.solve}"),
            "data": "synthetic",
            "config": {"workload": prob.name, "N": N, "m": m, "T": T, "F": "identity", "precision": args.prec,
                       "solve": args.solve if args.prec != "fp64" else "fp64",
                       "joseph_every": 16 if args.prec == "mixed" else 0,
                       "parallelism": f"replicas{world}",
                       "l2": "working set > L2 (covariance store of T N x N matrices)"},
            "tflops": value * executed_flops_per_timestep(N, m, 16 if args.prec == "mixed" else 0,
                                                          2 if args.solve == "fp64tc" else 0) / 1e12,
            "tflops_note": "flops the path executes (each split-bf16 product counted once)",
            "tflops_equivalent": value * total_f / 1e12,
            "tflops_equivalent_note": "standard operation count of KF + FIS (Cholesky + two N-RHS solves "
                                      "for the gain), as if the path executed it",
            "roofline": roof,
            "roofline_smoother": roof_smoother,
            "roofline_solve": roof_solve,
            "gpu_launches": launches,
            "clocks": clocks,
            "e2e": {"value": world * T / e2e_time, "unit": "timesteps/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "phase_ms": {names[c]: prof[c][1] / args.steps for c in prof}}

    if rank == 0 and world == 1 and args.batch_epochs > 0:
        line["batched"] = batched_sample(args, B, synth)
    if rank == 0 and world == 1 and args.serve_requests > 0:
        line["serve"] = serving_sample(args, B, synth)
    if rank == 0 and world == 1 and not args.no_fp64_plain and args.prec != "fp64":
        line["fp64_plain"] = fp64_plain_prefix(prob, B, solver, synth, torch)
    if rank == 0 and world == 1 and not args.no_solve_variants and args.prec == "mixed":
        line["solve_variants"] = solve_variants(args, B, solver, prob, torch)
    if rank == 0 and world == 1 and args.config1_prefix > 0:
        line["config1"] = config1_sample(args, B, solver, synth, torch)
    if rank == 0 and world == 1 and not args.no_config2_mesh:
        line["config2_mesh_recompute"] = config2_mesh_sample(args, B, solver, synth, torch)
    if rank == 0 and world == 1:
        line["mne_init"] = mne_init_sample(prob, B, solver, torch)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["config0"] = config0_sample(B, solver, synth, torch)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        per, sample = cpu_oracle_timestep(synth.config2(T=2))
        line["cpu_baseline"] = {"value": 1.0 / per, "unit": "timesteps/s", "cores": host_threads(), "kind": "oracle",
                                "sample": sample}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def serving_sample(args, B, synth):
    """The first requests of the seeded Poisson stream (20 req/s; N in {1024, 2048, 5124, 8196},
    m = 306, T ~ U{50..400}), served with admission by footprint against 160 GB."""
    from paper_1107_4192_gb300 import serve
    arrivals = synth.serving_arrivals(2000, 20.0, seed=4)[:args.serve_requests]
    reqs = []
    for i, (t, N, m, T) in enumerate(arrivals):
        prob = synth.mesh_problem(N, m, T, seed=4000 + i, identity_F=(i % 2 == 0))
        reqs.append(serve.Request(i, t, prob))
    res = serve.Server(160 * 10 ** 9, max_slots=4).run(reqs)
    out = serve.summarize(res)
    out["sample"] = (f"first {len(reqs)} requests of the 2000-request stream (arrivals over "
                     f"{arrivals[-1][0]:.2f} s), mixed path, 4 slots")
    return out


def batched_sample(args, B, synth):
    """Uneven epochs (N ~ U{256..2048 step 128}, m in {64,128,306}, T ~ U{20..200}, F = I or mesh)
    all submitted at once and run concurrently, 8 at a time."""
    from paper_1107_4192_gb300 import serve
    probs = synth.batched_epochs(args.batch_epochs, seed=3)
    _, summ = serve.run_batch(probs, max_slots=8)
    summ["epochs_per_s"] = summ["completed"] / summ["wall_s"] if summ["wall_s"] > 0 else 0.0
    summ["sample"] = f"{len(probs)} epochs, 8 concurrent plans on separate streams"
    return summ


def solve_variants(args, B, solver, prob, torch):
    """The same workload (whole epochs, inputs resident) with the other tensor-core solve modes, so
    the price of each precision contract of the smoother-gain solve is visible beside the headline."""
    out = {}
    modes = {"fp64tc": B.KF_SOLVE_FP64_TC, "fp64mean": B.KF_SOLVE_FP64_MEAN, "fp32": B.KF_SOLVE_FP32}
    for name, sv in modes.items():
        if name == args.solve:
            continue
        r, dt, _ = _epoch_rate(prob, B, solver, torch, reps=2, prec=B.KF_PREC_MIXED_BF16X3, solve_prec=sv,
                               joseph_every=16)
        out[name] = {"value": r, "unit": "timesteps/s", "s_per_epoch": dt}
    out["note"] = ("fp64tc: every J_t float64-accurate; fp64mean: the smoothed mean's solve float64-accurate, "
                   "J_t inside the split-bf16 covariance product float32-class; fp32: float32-class solve")
    return out


def _epoch_rate(prob, B, solver, torch, reps=1, **kw):
    """timesteps/s of filter + smoother over the whole problem (inputs resident), after one warm-up."""
    d = solver.upload(prob)
    plan = solver.Plan.for_inputs(d, prob.N, prob.m, prob.T, stream=torch.cuda.current_stream().cuda_stream, **kw)
    x = torch.empty(prob.T, prob.N, dtype=torch.float64, device="cuda")

    def run():
        B.kf_filter(plan.handle, d.F, d.F_rowptr, d.F_col, d.Q, d.H, d.R, d.Y, d.x0, d.P0, x)
        B.fis_smooth(plan.handle, x)

    run()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        run()
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / reps
    ck = B.kf_plan_footprint(plan.desc)[3]
    plan.close()
    return prob.T / dt, dt, ck


def config1_sample(args, B, solver, synth, torch):
    """Config 1 (N = 5124 sources on two icospheres, mesh F, m = 306, T = 200): float64 and float32
    on the GPU on a T-prefix (the float64 smoother takes ~0.6 s per step at this N), and the mixed
    path with the float64-accurate tensor-core solve over the whole epoch."""
    T_pre = args.config1_prefix
    out = {"workload": "N5124_m306_T200_mesh (config 1)", "unit": "timesteps/s"}
    pre = synth.config1(T=T_pre)
    for name, kw in (("fp64", dict(prec=B.KF_PREC_FP64)),
                     ("fp32", dict(prec=B.KF_PREC_FP32, solve_prec=B.KF_SOLVE_FP64))):
        r, dt, _ = _epoch_rate(pre, B, solver, torch, **kw)
        out[f"{name}_prefix"] = {"value": r, "sample": f"T={T_pre} prefix, filter + smoother", "s": dt}
    full = synth.config1()
    r, dt, _ = _epoch_rate(full, B, solver, torch, prec=B.KF_PREC_MIXED_BF16X3, solve_prec=B.KF_SOLVE_FP64_TC,
                           joseph_every=16)
    out["mixed_fp64tc"] = {"value": r, "sample": "whole T=200 epoch, split-bf16 bulk, float64-accurate solve", "s": dt}
    return out


def config2_mesh_sample(args, B, solver, synth, torch):
    """Config 2 (ii): N = 8196 with the mesh coupling F = 0.9 I + 0.016 A, m = 306, T = 300, mixed path.
    The footprint rule of the workload, 2 N^2 T float32 words (predicted and filtered covariances),
    is 161 GB > 160 GB, so the epoch runs in recompute mode: checkpoints of P_{t|t} every
    round(sqrt(T)) steps, the other steps recomputed forward during the smoother.  (This plan
    stores only P_{t|t} and rebuilds P_{t+1|t} = F P F^T + Q from it, so its full store would
    take half that.)  One whole epoch."""
    prob = synth.config2(identity_F=False)
    budget = 160 * 10 ** 9
    rule = 2 * prob.N * prob.N * prob.T * 4
    ck = int(round(np.sqrt(prob.T))) if rule > budget else 0
    solve = {"fp32": B.KF_SOLVE_FP32, "fp64": B.KF_SOLVE_FP64, "fp64tc": B.KF_SOLVE_FP64_TC,
             "fp64mean": B.KF_SOLVE_FP64_MEAN}[args.solve]
    r, dt, ck_used = _epoch_rate(prob, B, solver, torch, prec=B.KF_PREC_MIXED_BF16X3, solve_prec=solve,
                                 joseph_every=16, mem_budget_bytes=budget, checkpoint_every=ck)
    return {"workload": prob.name, "value": r, "unit": "timesteps/s", "s": dt, "checkpoint_every": ck_used,
            "footprint_rule_bytes": rule, "budget_bytes": budget, "solve": args.solve}


def mne_init_sample(prob, B, solver, torch):
    """The paper's initialisation (x0 = minimum-norm estimate, Q = sample covariance of the
    differenced estimates) on the whole workload: one call after one warm-up call."""
    h = solver.host_inputs(prob)
    t = lambda a: torch.from_numpy(a).cuda()
    H, R, Y, C = t(h["H"]), t(h["R"]), t(h["Y"]), t(np.array([1.0]))
    x0 = torch.empty(prob.N, dtype=torch.float64, device="cuda")
    Q = torch.empty(prob.N, prob.N, dtype=torch.float64, device="cuda")
    args = (H, C, 0, R, h["r_kind"], Y, prob.N, prob.m, prob.T, 1.0, None, x0, Q)
    B.mne_init(*args)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    B.mne_init(*args)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3
    del Q
    return {"ms": ms, "sample": f"x0 and dense Q from the {prob.T} float64 minimum-norm estimates (C = I, "
                                f"lambda = 1), N = {prob.N}, m = {prob.m}; includes its own allocations"}


def fp64_plain_prefix(prob, B, solver, synth, torch, T_pre=3):
    """Plain float64 path on the first T_pre steps of the same workload (a full
    float64 epoch takes minutes); rate = 1 / (filter step + smoother step)."""
    p = synth.config2(T=T_pre)
    d = solver.upload(p)
    plan = solver.Plan.for_inputs(d, p.N, p.m, T_pre, prec=B.KF_PREC_FP64,
                                  stream=torch.cuda.current_stream().cuda_stream)
    x = torch.empty(T_pre, p.N, dtype=torch.float64, device="cuda")
    B.kf_filter(plan.handle, d.F, d.F_rowptr, d.F_col, d.Q, d.H, d.R, d.Y, d.x0, d.P0, x)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    B.kf_filter(plan.handle, d.F, d.F_rowptr, d.F_col, d.Q, d.H, d.R, d.Y, d.x0, d.P0, x)
    t1 = time.perf_counter()
    B.fis_smooth(plan.handle, x)
    t2 = time.perf_counter()
    plan.close()
    per = (t1 - t0) / T_pre + (t2 - t1) / (T_pre - 1)
    return {"value": 1.0 / per, "unit": "timesteps/s", "sample": f"T={T_pre} prefix, float64 throughout",
            "filter_ms_per_step": (t1 - t0) / T_pre * 1e3, "smoother_ms_per_step": (t2 - t1) / (T_pre - 1) * 1e3}


if __name__ == "__main__":
    main()
