"""Python front end: device inputs for a problem and a plan wrapper.

Marshalling only; the filter and smoother run inside libkfmeg.so.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional

import numpy as np

from . import binding as B


@dataclass
class DeviceInputs:
    """Inputs of kf_filter as float64/int64 CUDA tensors (None where unused)."""
    f_kind: int
    F: Optional[object]
    F_rowptr: Optional[object]
    F_col: Optional[object]
    f_nnz: int
    q_kind: int
    Q: object
    H: object
    r_kind: int
    R: object
    Y: object
    x0: object
    P0: object


def host_inputs(prob, dense_F=False):
    """numpy arrays in the layout of the C interface (row-major, float64/int64).
    dense_F: pass F as a dense N x N matrix (KF_F_DENSE) instead of compressed rows."""
    f64 = lambda a: np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if prob.F is None and not dense_F:
        f_kind, F, rp, col, nnz = B.KF_F_IDENTITY, None, None, None, 0
    elif dense_F:
        f_kind, F, rp, col, nnz = B.KF_F_DENSE, f64(prob.F_dense()), None, None, 0
    else:
        f_kind, nnz = B.KF_F_CSR, prob.F.nnz
        F, rp, col = f64(prob.F.val), np.ascontiguousarray(prob.F.rowptr, np.int64), \
            np.ascontiguousarray(prob.F.col, np.int64)
    Q = f64(np.reshape(prob.Q, (1,)) if prob.q_kind == 0 else prob.Q)
    R = f64(np.reshape(prob.R, (1,)) if prob.r_kind == 0 else prob.R)
    P0 = f64(prob.P0) if prob.P0 is not None else f64(prob.p0_scale * np.eye(prob.N))
    return dict(f_kind=f_kind, F=F, F_rowptr=rp, F_col=col, f_nnz=nnz, q_kind=prob.q_kind, Q=Q, H=f64(prob.H),
                r_kind=prob.r_kind, R=R, Y=f64(prob.Y), x0=f64(prob.x0), P0=P0)


def upload(prob, device="cuda", dense_F=False) -> DeviceInputs:
    import torch
    h = host_inputs(prob, dense_F)
    t = lambda a: None if a is None else torch.from_numpy(a).to(device)
    if prob.P0 is None:  # build the scaled identity on the device
        P0 = torch.eye(prob.N, dtype=torch.float64, device=device) * float(prob.p0_scale)
    else:
        P0 = t(h["P0"])
    return DeviceInputs(h["f_kind"], t(h["F"]), t(h["F_rowptr"]), t(h["F_col"]), h["f_nnz"], h["q_kind"],
                        t(h["Q"]), t(h["H"]), h["r_kind"], t(h["R"]), t(h["Y"]), t(h["x0"]), P0)


class Plan:
    """One kf_plan for the shape of a problem; filter() then smooth()."""

    def __init__(self, N, m, T, f_kind=B.KF_F_IDENTITY, f_nnz=0, prec=B.KF_PREC_FP64,
                 solve_prec=B.KF_SOLVE_FP64, q_kind=B.KF_COV_SCALAR, r_kind=B.KF_COV_SCALAR, joseph_every=0,
                 mem_budget_bytes=0, checkpoint_every=0, split_terms=0, stream=None):
        self.N, self.m, self.T = N, m, T
        self.desc = B.make_desc(N, m, T, f_kind, prec, solve_prec, q_kind, r_kind, joseph_every, f_nnz,
                                mem_budget_bytes, checkpoint_every, split_terms, stream)
        self.handle = B.kf_plan(self.desc)

    @classmethod
    def for_inputs(cls, d: DeviceInputs, N, m, T, **kw):
        return cls(N, m, T, f_kind=d.f_kind, f_nnz=d.f_nnz, q_kind=d.q_kind, r_kind=d.r_kind, **kw)

    def filter(self, d: DeviceInputs, want_diag=True):
        import torch
        dev = d.H.device
        x = torch.empty(self.T, self.N, dtype=torch.float64, device=dev)
        dp = torch.empty(self.T, self.N, dtype=torch.float64, device=dev) if want_diag else None
        B.kf_filter(self.handle, d.F, d.F_rowptr, d.F_col, d.Q, d.H, d.R, d.Y, d.x0, d.P0, x, dp)
        return x, dp

    def smooth(self, want_diag=True, t_full=-1):
        import torch
        dev = torch.device("cuda")
        x = torch.empty(self.T, self.N, dtype=torch.float64, device=dev)
        dp = torch.empty(self.T, self.N, dtype=torch.float64, device=dev) if want_diag else None
        Pf = torch.empty(self.N, self.N, dtype=torch.float64, device=dev) if t_full > 0 else None
        B.fis_smooth(self.handle, x, dp, Pf, t_full)
        return x, dp, Pf

    def close(self):
        if self.handle:
            B.kf_plan_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def run(prob, prec=B.KF_PREC_FP64, solve_prec=B.KF_SOLVE_FP64, joseph_every=0, checkpoint_every=0,
        t_full=-1, split_terms=0, device="cuda", dense_F=False):
    """Filter + smoother for a synthetic problem; returns numpy outputs."""
    d = upload(prob, device, dense_F)
    with Plan.for_inputs(d, prob.N, prob.m, prob.T, prec=prec, solve_prec=solve_prec, joseph_every=joseph_every,
                         checkpoint_every=checkpoint_every, split_terms=split_terms) as plan:
        xf, df = plan.filter(d)
        xs, ds, Pf = plan.smooth(t_full=t_full)
        out = dict(x_filt=xf.cpu().numpy(), diagP_filt=df.cpu().numpy(), x_smooth=xs.cpu().numpy(),
                   diagP_smooth=ds.cpu().numpy())
        if Pf is not None:
            out["P_smooth_at"] = Pf.cpu().numpy()
    return out
