"""Seeded synthetic inputs for the state-space MEG model (eqns 1-3).

This module only draws random inputs.  It holds none of the filter or
smoother arithmetic, so both the CUDA path and the CPU oracle can consume
its output without sharing any of the method's code.

The paper's own inputs (an MRI-derived BEM lead field over a decimated
cortical mesh, Sec. 4.1, and real MEG recordings, Sec. 4.2) are not
available, so every workload here is a synthetic stand-in with the same
shapes:

* lead field H (m x N): i.i.d. N(0,1) entries, column j multiplied by
  exp(-d_j) with depth d_j ~ U(0,3) (deep sources have weak fields);
* cortical mesh: recursively subdivided icosahedra (Sec. 4.1 uses "the
  topology of a recursively subdivided icosahedron"), one sphere per
  hemisphere; octahedra when the vertex count must be 4*4^k+2;
* neighbourhood dynamics (eqn 2 generalised to eqn 3):
  F = 0.9 I + 0.016 A with A the mesh adjacency (six direct neighbours);
* active sources: Gaussian-smoothed patches over graph distance carrying a
  10-20 Hz sinusoid times a 0.4 Hz envelope sampled at 600 Hz (Sec. 4.1).
"""
from __future__ import annotations

from collections import deque
from dataclasses import dataclass, field
from functools import lru_cache
from typing import Optional

import numpy as np

SAMPLE_HZ = 600.0

# ---------------------------------------------------------------- meshes


def _subdivide(verts: np.ndarray, faces: np.ndarray, levels: int):
    verts = [tuple(v) for v in verts]
    faces = [tuple(f) for f in faces]
    for _ in range(levels):
        cache = {}
        new_faces = []

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                p = np.add(verts[a], verts[b]) * 0.5
                p = p / np.linalg.norm(p)
                cache[key] = len(verts)
                verts.append(tuple(p))
            return cache[key]

        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            new_faces += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = new_faces
    return np.asarray(verts), np.asarray(faces, dtype=np.int64)


def icosphere(levels: int):
    """Icosahedron subdivided `levels` times: 10*4^levels + 2 vertices."""
    t = (1.0 + 5 ** 0.5) / 2.0
    v = np.array([[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
                  [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
                  [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], dtype=float)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
                  [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
                  [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
                  [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]])
    return _subdivide(v, f, levels)


def octasphere(levels: int):
    """Octahedron subdivided `levels` times: 4*4^levels + 2 vertices."""
    v = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], float)
    f = np.array([[0, 2, 4], [2, 1, 4], [1, 3, 4], [3, 0, 4],
                  [2, 0, 5], [1, 2, 5], [3, 1, 5], [0, 3, 5]])
    return _subdivide(v, f, levels)


def fibonacci_sphere(n: int):
    """n points on the unit sphere triangulated by their convex hull."""
    from scipy.spatial import ConvexHull
    i = np.arange(n) + 0.5
    phi = np.arccos(1 - 2 * i / n)
    theta = np.pi * (1 + 5 ** 0.5) * i
    v = np.stack([np.cos(theta) * np.sin(phi), np.sin(theta) * np.sin(phi), np.cos(phi)], 1)
    return v, ConvexHull(v).simplices.astype(np.int64)


def faces_to_neighbours(n: int, faces: np.ndarray):
    nb = [set() for _ in range(n)]
    for a, b, c in faces:
        nb[a] |= {b, c}
        nb[b] |= {a, c}
        nb[c] |= {a, b}
    return [sorted(s) for s in nb]


def sphere_for(n_vertices: int):
    """A triangulated sphere with exactly n_vertices vertices."""
    for k in range(0, 8):
        if 10 * 4 ** k + 2 == n_vertices:
            return icosphere(k)
        if 4 * 4 ** k + 2 == n_vertices:
            return octasphere(k)
    return fibonacci_sphere(n_vertices)


@lru_cache(maxsize=16)
def _hemisphere_mesh_cached(N: int):
    return tuple(tuple(s) for s in _hemisphere_mesh(N))


def hemisphere_mesh(N: int):
    """Neighbour lists for N sources split over two hemispheres (blocks)."""
    return [list(s) for s in _hemisphere_mesh_cached(N)]


def _hemisphere_mesh(N: int):
    halves = [N // 2, N - N // 2] if N >= 8 else [N]
    neigh, off = [], 0
    for h in halves:
        if h < 4:
            nb = [[j for j in range(h) if j != i] for i in range(h)]
        else:
            _, faces = sphere_for(h)
            nb = faces_to_neighbours(h, faces)
        neigh += [[off + j for j in s] for s in nb]
        off += h
    return neigh


@dataclass
class CSR:
    """Sparse matrix in compressed-row form (int64 indices, fp64 values)."""
    n: int
    rowptr: np.ndarray
    col: np.ndarray
    val: np.ndarray

    @property
    def nnz(self):
        return int(self.rowptr[-1])


def mesh_coupling(neigh, diag: float = 0.9, off: float = 0.016) -> CSR:
    """F = diag*I + off*A over the neighbour lists, rows sorted by column."""
    n = len(neigh)
    rowptr = np.zeros(n + 1, np.int64)
    cols, vals = [], []
    for i, s in enumerate(neigh):
        row = sorted(set(s) | {i})
        cols += row
        vals += [diag if j == i else off for j in row]
        rowptr[i + 1] = len(cols)
    return CSR(n, rowptr, np.asarray(cols, np.int64), np.asarray(vals, float))


def graph_distance(neigh, src: int, limit: int):
    dist = {src: 0}
    q = deque([src])
    while q:
        u = q.popleft()
        if dist[u] >= limit:
            continue
        for v in neigh[u]:
            if v not in dist:
                dist[v] = dist[u] + 1
                q.append(v)
    return dist


# ---------------------------------------------------------------- problems


@dataclass
class Problem:
    """One epoch of the state-space model x_t = F x_{t-1} + v_t, y_t = H x_t + e_t.

    (x0, P0) describe the state at t = 0; Y[t-1] is the measurement of step t.
    q_kind / r_kind: 0 = scalar * I, 1 = diagonal (vector), 2 = dense matrix.
    """
    N: int
    m: int
    T: int
    H: np.ndarray                 # m x N
    Y: np.ndarray                 # T x m
    x0: np.ndarray                # N
    p0_scale: float               # P0 = p0_scale * I unless P0 is given
    q_kind: int
    Q: np.ndarray                 # scalar (shape ()), N, or N x N
    r_kind: int
    R: np.ndarray                 # scalar, m, or m x m
    F: Optional[CSR] = None       # None = identity
    P0: Optional[np.ndarray] = None
    x_true: Optional[np.ndarray] = None
    name: str = ""
    seed: int = 0
    meta: dict = field(default_factory=dict)

    def P0_dense(self) -> np.ndarray:
        if self.P0 is not None:
            return self.P0
        return self.p0_scale * np.eye(self.N)

    def Q_dense(self) -> np.ndarray:
        return _cov_dense(self.q_kind, self.Q, self.N)

    def R_dense(self) -> np.ndarray:
        return _cov_dense(self.r_kind, self.R, self.m)

    def F_dense(self) -> np.ndarray:
        if self.F is None:
            return np.eye(self.N)
        A = np.zeros((self.N, self.N))
        for i in range(self.N):
            s, e = self.F.rowptr[i], self.F.rowptr[i + 1]
            A[i, self.F.col[s:e]] = self.F.val[s:e]
        return A


def _cov_dense(kind, v, n):
    if kind == 0:
        return float(v) * np.eye(n)
    if kind == 1:
        return np.diag(np.asarray(v, float))
    return np.asarray(v, float)


def lead_field(rng, m: int, N: int) -> np.ndarray:
    depth = rng.uniform(0.0, 3.0, size=N)
    return rng.standard_normal((m, N)) * np.exp(-depth)[None, :]


def simulate_state_space(rng, N, m, T, F_dense, Qd, Rd, x0_mean, P0d, H):
    """Draws x_0..x_T and y_1..y_T from eqns 1 and 3 (model simulation only)."""
    Lp = np.linalg.cholesky(P0d)
    Lq = np.linalg.cholesky(Qd)
    Lr = np.linalg.cholesky(Rd)
    x = x0_mean + Lp @ rng.standard_normal(N)
    xs, ys = [], []
    for _ in range(T):
        x = F_dense @ x + Lq @ rng.standard_normal(N)
        xs.append(x)
        ys.append(H @ x + Lr @ rng.standard_normal(m))
    return np.asarray(xs), np.asarray(ys)


def patch_sources(rng, neigh, T: int, n_patches: int = 3, width: float = 3.0):
    """Gaussian-smoothed patches carrying 10-20 Hz sinusoids x 0.4 Hz envelope."""
    N = len(neigh)
    x = np.zeros((T, N))
    t = np.arange(1, T + 1)
    env = np.sin(2 * np.pi * 0.4 * t / SAMPLE_HZ)
    for _ in range(n_patches):
        c = int(rng.integers(N))
        f = rng.uniform(10.0, 20.0)
        sig = np.sin(2 * np.pi * f * t / SAMPLE_HZ) * env
        for v, g in graph_distance(neigh, c, int(3 * width)).items():
            x[:, v] += np.exp(-g * g / (2 * width * width)) * sig
    return x


def random_walk_problem(N: int, m: int, T: int, seed: int, q: float = 0.01,
                        r: float = 1.0, p0: float = 1.0, name: str = "") -> Problem:
    """F = I, Q = q I, R = r I, P0 = p0 I, x0 = 0; y simulated from the model."""
    rng = np.random.default_rng(seed)
    H = lead_field(rng, m, N)
    _, Y = simulate_state_space(rng, N, m, T, np.eye(N), q * np.eye(N), r * np.eye(m),
                                np.zeros(N), p0 * np.eye(N), H)
    return Problem(N, m, T, H, Y, np.zeros(N), p0, 0, np.array(q), 0, np.array(r),
                   name=name or f"randwalk_N{N}_m{m}_T{T}", seed=seed)


def mesh_problem(N: int, m: int, T: int, seed: int, identity_F: bool = False,
                 q: float = 1e-2, p0: float = 1.0, name: str = "") -> Problem:
    """Mesh-coupled dynamics (or F = I), diagonal R ~ U(0.5, 2), patch sources."""
    rng = np.random.default_rng(seed)
    neigh = hemisphere_mesh(N)
    Fm = None if identity_F else mesh_coupling(neigh)
    H = lead_field(rng, m, N)
    Rv = rng.uniform(0.5, 2.0, size=m)
    x_true = patch_sources(rng, neigh, T)
    Y = x_true @ H.T + rng.standard_normal((T, m)) * np.sqrt(Rv)[None, :]
    return Problem(N, m, T, H, Y, np.zeros(N), p0, 0, np.array(q), 1, Rv, F=Fm,
                   x_true=x_true, name=name or f"mesh_N{N}_m{m}_T{T}", seed=seed)


def random_dense_problem(N: int, m: int, T: int, seed: int, name: str = "") -> Problem:
    """General problem for parity tests: non-symmetric sparse F, dense Q, R, P0."""
    rng = np.random.default_rng(seed)
    neigh = hemisphere_mesh(N) if N >= 4 else [[j for j in range(N) if j != i] for i in range(N)]
    base = mesh_coupling(neigh)
    val = base.val * rng.uniform(0.6, 1.0, size=base.val.shape)   # breaks symmetry of F
    Fm = CSR(N, base.rowptr, base.col, val)
    Aq = rng.standard_normal((N, N)) / np.sqrt(N)
    Qd = 0.02 * np.eye(N) + 0.01 * Aq @ Aq.T
    Ar = rng.standard_normal((m, m)) / np.sqrt(m)
    Rd = 0.5 * np.eye(m) + 0.2 * Ar @ Ar.T
    Ap = rng.standard_normal((N, N)) / np.sqrt(N)
    P0 = 0.5 * np.eye(N) + 0.3 * Ap @ Ap.T
    H = lead_field(rng, m, N)
    x0 = rng.standard_normal(N)
    prob = Problem(N, m, T, H, np.zeros((T, m)), x0, 1.0, 2, Qd, 2, Rd, F=Fm, P0=P0,
                   name=name or f"dense_N{N}_m{m}_T{T}", seed=seed)
    _, Y = simulate_state_space(rng, N, m, T, prob.F_dense(), Qd, Rd, x0, P0, H)
    prob.Y = Y
    return prob


def dense_dynamics_problem(N: int, m: int, T: int, seed: int, name: str = "") -> Problem:
    """Fully dense, non-symmetric F = 0.85 I + 0.05 G / sqrt(N) (G Gaussian, spectral radius
    below 1), dense Q, R and P0, non-zero x0: the general linear model of eqn 3.  F is kept in
    compressed-row form with every entry present, so it can be passed either way."""
    rng = np.random.default_rng(seed)
    Fd = 0.85 * np.eye(N) + 0.05 * rng.standard_normal((N, N)) / np.sqrt(N)
    Fm = CSR(N, np.arange(0, N * N + 1, N, dtype=np.int64), np.tile(np.arange(N, dtype=np.int64), N),
             Fd.reshape(-1).copy())
    Aq = rng.standard_normal((N, N)) / np.sqrt(N)
    Qd = 0.02 * np.eye(N) + 0.01 * Aq @ Aq.T
    Ar = rng.standard_normal((m, m)) / np.sqrt(m)
    Rd = 0.5 * np.eye(m) + 0.2 * Ar @ Ar.T
    Ap = rng.standard_normal((N, N)) / np.sqrt(N)
    P0 = 0.5 * np.eye(N) + 0.3 * Ap @ Ap.T
    H = lead_field(rng, m, N)
    x0 = rng.standard_normal(N)
    _, Y = simulate_state_space(rng, N, m, T, Fd, Qd, Rd, x0, P0, H)
    return Problem(N, m, T, H, Y, x0, 1.0, 2, Qd, 2, Rd, F=Fm, P0=P0,
                   name=name or f"densedyn_N{N}_m{m}_T{T}", seed=seed)


# ------------------------------------------------------- named workloads

def config0() -> Problem:
    """Plain FP64 case: N=384, m=64, T=40, F=I, Q=0.01 I, R=I, P0=I, x0=0 (seed 0)."""
    return random_walk_problem(384, 64, 40, seed=0, name="N384_m64_T40_randwalk")


def config1(T: Optional[int] = None) -> Problem:
    """Paper-scale epoch: N=5124 (two 2562-vertex icospheres), m=306, T=200 (seed 1)."""
    return mesh_problem(5124, 306, T or 200, seed=1, name="N5124_m306_T200_mesh")


def config2(T: Optional[int] = None, identity_F: bool = True) -> Problem:
    """Mixed-precision epoch: N=8196 (two 4098-vertex octaspheres), m=306, T=300 (seed 2)."""
    return mesh_problem(8196, 306, T or 300, seed=2, identity_F=identity_F,
                        name="N8196_m306_T300_" + ("randwalk" if identity_F else "mesh"))


def batched_epochs(n_epochs: int = 64, seed: int = 3):
    """Uneven epochs: N ~ U{256..2048 step 128}, m in {64,128,306}, T ~ U{20..200}."""
    rng = np.random.default_rng(seed)
    out = []
    for e in range(n_epochs):
        N = int(rng.choice(np.arange(256, 2049, 128)))
        m = int(rng.choice([64, 128, 306]))
        T = int(rng.integers(20, 201))
        ident = bool(rng.integers(2))
        out.append(mesh_problem(N, m, T, seed=seed * 1000 + e, identity_F=ident,
                                name=f"batch{e}_N{N}_m{m}_T{T}"))
    return out


def serving_arrivals(n_requests: int = 2000, rate_hz: float = 20.0, seed: int = 4):
    """Poisson arrivals: (arrival_s, N, m, T) with N in {1024,2048,5124,8196}, T ~ U{50..400}."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, size=n_requests)
    t = np.cumsum(gaps)
    Ns = rng.choice([1024, 2048, 5124, 8196], size=n_requests)
    Ts = rng.integers(50, 401, size=n_requests)
    return [(float(t[i]), int(Ns[i]), 306, int(Ts[i])) for i in range(n_requests)]
