"""Seeded synthetic linear-quadratic OCP instances (inputs only).

This module defines the in-memory layout of an OCP instance and draws seeded
random instances shaped like the five benchmark workloads.  It holds none of
the solver's arithmetic: both the CPU oracle and the CUDA library consume what
it produces, and nothing here depends on either of them.

Problem (paper Sec. 2, eq. ``ocp-eq`` with E_j = I):

    minimise  sum_k 1/2 [u;x]^T [R_k S_k; S_k^T Q_k] [u;x] + [r_k; q_k]^T [u;x]
              + 1/2 x_N^T Q_N x_N + q_N^T x_N
    s.t.      x_0 = x_init,  x_{k+1} = A_k x_k + B_k u_k + c_k   (0 <= k < N)

with S_k in R^{nu x nx} (the paper's orientation, cost term u^T S x), and an
optional diagonal regularisation Sigma_k added to diag(R_k, Q_k) (and Sigma_N to
Q_N), read as the augmented-Lagrangian term of Sec. 5.1 with box constraints
on every input and state.

Flat layout of one instance (all float64, every matrix block column-major):

    Q      (N+1) blocks nx*nx     k = 0..N   (Q_0 is never read: x_0 is fixed)
    R      N blocks     nu*nu     k = 0..N-1
    S      N blocks     nu*nx     k = 0..N-1 (S_0 is never read)
    A      N blocks     nx*nx     k = 0..N-1 (A_0 is never read by the KKT matrix)
    B      N blocks     nx*nu     k = 0..N-1
    Sigma  (N+1) records of nu+nx  [Sigma_u_k | Sigma_x_k]; record 0's x part and
           record N's u part are never read
    q      (N+1)*nx,  r  N*nu,  c  N*nx,  x0  nx

A batch concatenates the per-instance arrays of each kind in instance order.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence

import numpy as np

__all__ = [
    "OCPInstance", "Batch", "CONFIGS", "make_instance", "make_batch",
    "config_dims", "instance_dims", "blocks_to_flat", "flat_to_blocks",
    "ALMData", "make_alm", "concat_alm", "config_alm",
]


def blocks_to_flat(blocks: np.ndarray) -> np.ndarray:
    """Stack of matrices (K, rows, cols) -> flat column-major blocks."""
    return np.ascontiguousarray(np.asarray(blocks, dtype=np.float64).transpose(0, 2, 1)).ravel()


def flat_to_blocks(flat: np.ndarray, count: int, rows: int, cols: int) -> np.ndarray:
    """Inverse of :func:`blocks_to_flat` (returns a (count, rows, cols) copy)."""
    a = np.asarray(flat, dtype=np.float64)[: count * rows * cols]
    return np.ascontiguousarray(a.reshape(count, cols, rows).transpose(0, 2, 1))


@dataclasses.dataclass
class OCPInstance:
    N: int
    nx: int
    nu: int
    Q: np.ndarray
    R: np.ndarray
    S: np.ndarray
    A: np.ndarray
    B: np.ndarray
    Sigma: Optional[np.ndarray]
    # one (q, r, c, x0) tuple per right-hand side
    rhs: List[tuple]

    # ---- block accessors (layout only) ----
    def Qk(self, k: int) -> np.ndarray:
        n = self.nx
        return self.Q[k * n * n:(k + 1) * n * n].reshape(n, n).T.copy()

    def Rk(self, k: int) -> np.ndarray:
        m = self.nu
        return self.R[k * m * m:(k + 1) * m * m].reshape(m, m).T.copy()

    def Sk(self, k: int) -> np.ndarray:
        m, n = self.nu, self.nx
        return self.S[k * m * n:(k + 1) * m * n].reshape(n, m).T.copy()

    def Ak(self, k: int) -> np.ndarray:
        n = self.nx
        return self.A[k * n * n:(k + 1) * n * n].reshape(n, n).T.copy()

    def Bk(self, k: int) -> np.ndarray:
        m, n = self.nu, self.nx
        return self.B[k * n * m:(k + 1) * n * m].reshape(m, n).T.copy()

    def Sigma_u(self, k: int) -> np.ndarray:
        if self.Sigma is None:
            return np.zeros(self.nu)
        w = self.nu + self.nx
        return self.Sigma[k * w:k * w + self.nu].copy()

    def Sigma_x(self, k: int) -> np.ndarray:
        if self.Sigma is None:
            return np.zeros(self.nx)
        w = self.nu + self.nx
        return self.Sigma[k * w + self.nu:(k + 1) * w].copy()

    @property
    def kkt_size(self) -> int:
        """Unknowns u_0..u_{N-1}, x_1..x_N, lambda_0..lambda_{N-1}."""
        return self.N * (self.nu + 2 * self.nx)


@dataclasses.dataclass
class Batch:
    """Concatenation of instances; arrays are flat float64 (host)."""
    N: np.ndarray
    nx: np.ndarray
    nu: np.ndarray
    Q: np.ndarray
    R: np.ndarray
    S: np.ndarray
    A: np.ndarray
    B: np.ndarray
    Sigma: Optional[np.ndarray]
    rhs: List[tuple]   # per right-hand side: (q, r, c, x0) concatenated over instances
    instances: List[OCPInstance]

    @property
    def size(self) -> int:
        return int(len(self.N))

    @property
    def stages(self) -> int:
        return int(self.N.sum())

    @property
    def kkt_size(self) -> int:
        return int((self.N * (self.nu + 2 * self.nx)).sum())


# ---------------------------------------------------------------------------
# Workload recipes.  Each config names the five benchmark workloads by their
# shape; the drawing rules are stated in the design notes.
# ---------------------------------------------------------------------------
CONFIGS = {
    # single OCP, N=32, nx=8, nu=4, S=0, Q_N=Q_0, one factor + one solve
    "single_n32_nx8_nu4": dict(batch=1, N=32, nx=8, nu=4, S=False, sigma=None,
                               nrhs=1, QN_equals_Q0=True, seed=0),
    # 1024 OCPs, N=64, nx=12, nu=4, S~0.1N(0,1) (stage block kept SPD), Sigma in LU[1e-6,1e6], 4 RHS
    "batch1024_n64_nx12_nu4": dict(batch=1024, N=64, nx=12, nu=4, S=True, sigma=(1e-6, 1e6),
                                   nrhs=4, QN_equals_Q0=False, seed=1),
    # 8 OCPs, N=4096, nx=32, nu=16, dense random S, Sigma in LU[1e-4,1e4]
    "long_n4096_nx32_nu16": dict(batch=8, N=4096, nx=32, nu=16, S=True, sigma=(1e-4, 1e4),
                                 nrhs=1, QN_equals_Q0=False, seed=2),
    # 4096 OCPs, N~U[16,256], nx~U{4..64}, nu~U{2..32}, Sigma in LU[1e-6,1e6]
    "uneven4096": dict(batch=4096, N=(16, 256), nx=(4, 64), nu=(2, 32), S=True, sigma=(1e-6, 1e6),
                       nrhs=1, QN_equals_Q0=False, seed=3),
    # 512 OCPs, N=128, nx=24, nu=8, S=0, no Sigma (differentiation workload)
    "adjoint512_n128_nx24_nu8": dict(batch=512, N=128, nx=24, nu=8, S=False, sigma=None,
                                     nrhs=1, QN_equals_Q0=False, seed=4),
    # the paper's mass-spring MPC (Sec. 8.1): M = 18 masses (nx = 36, nu = 9), N = 96,
    # 150 initial states; Sigma (ALM penalties) on the boxed coordinates only
    "massspring150_M18_N96": dict(kind="mass_spring", batch=150, M=18, N=96, nx=36, nu=9, S=False,
                                  sigma=(1e-2, 1e4), nrhs=1, QN_equals_Q0=True, seed=5),
    # Newton step of the augmented Lagrangian inner problem (Sec. 5) on the batch1024
    # shapes: 16 general constraint rows per stage (C, D dense), boxes around [-1, 1]
    # (a mix of active and inactive rows), penalties log-uniform in [1e-2, 1e4]
    "newton1024_n64_nx12_nu4_ny16": dict(batch=1024, N=64, nx=12, nu=4, S=True, sigma=None, nrhs=1,
                                         QN_equals_Q0=False, seed=6,
                                         alm=dict(ny=16, bounds="mixed", sigma=(1e-2, 1e4))),
}


def mass_spring_dynamics(M: int, Ts: float):
    """Zero-order-hold discretization (A, B) of the mass-spring chain of Sec. 8.1:
    M unit masses joined by unit springs, the outer ones to walls at distance
    zero, no friction; actuators between pairs of masses in the 6 x 3 pattern W,
    repeated M/6 times.  The continuous model x' = A_c x + B_c u is integrated
    over one sampling interval with u held constant, through the exponential of
    the augmented matrix [[A_c, B_c], [0, 0]] Ts (scipy's scaling-and-squaring
    Pade routine)."""
    import scipy.linalg
    if M % 6:
        raise ValueError("M must be a multiple of 6")
    nx, nu = 2 * M, M // 2
    V = -2.0 * np.eye(M) + np.eye(M, k=1) + np.eye(M, k=-1)
    W = np.zeros((6, 3))
    W[0, 0], W[1, 0] = 1.0, -1.0
    W[2, 1], W[4, 1] = 1.0, -1.0
    W[3, 2], W[5, 2] = 1.0, -1.0
    Ac = np.block([[np.zeros((M, M)), np.eye(M)], [V, np.zeros((M, M))]])
    Bc = np.vstack([np.zeros((M, nu)), scipy.linalg.block_diag(*([W] * (M // 6)))])
    aug = np.zeros((nx + nu, nx + nu))
    aug[:nx, :nx] = Ac
    aug[:nx, nx:] = Bc
    E = scipy.linalg.expm(aug * Ts)
    return E[:nx, :nx].copy(), E[:nx, nx:].copy(), Ac, Bc


def _make_mass_spring(cfg, index: int, N: int, nrhs: int, g) -> "OCPInstance":
    """Instance `index` of a mass-spring config: the paper's dynamics and costs
    (Q = Q_N = R = I, S = 0, steady state at the origin, so q = r = c = 0),
    Sigma log-uniform in cfg["sigma"] on the positions and the inputs (the
    boxed coordinates; velocities have none), initial positions uniform in
    [-3, 3] and zero velocities."""
    M = int(cfg["M"])
    nx, nu = 2 * M, M // 2
    Ad, Bd, _, _ = mass_spring_dynamics(M, 15.0 / N)
    A = np.broadcast_to(Ad, (N, nx, nx)).copy()
    B = np.broadcast_to(Bd, (N, nx, nu)).copy()
    Q = np.broadcast_to(np.eye(nx), (N + 1, nx, nx)).copy()
    R = np.broadcast_to(np.eye(nu), (N, nu, nu)).copy()
    S = np.zeros((N, nu, nx))
    lo, hi = cfg["sigma"]
    sig = 10.0 ** g.uniform(np.log10(lo), np.log10(hi), size=(N + 1, nu + nx))
    sig[:, nu + M:] = 0.0   # velocities are not boxed
    rhs = []
    for _ in range(nrhs):
        x0 = np.concatenate([g.uniform(-3.0, 3.0, size=M), np.zeros(M)])
        rhs.append((np.zeros((N + 1) * nx), np.zeros(N * nu), np.zeros(N * nx), x0))
    return OCPInstance(N=N, nx=nx, nu=nu, Q=blocks_to_flat(Q), R=blocks_to_flat(R), S=blocks_to_flat(S),
                       A=blocks_to_flat(A), B=blocks_to_flat(B), Sigma=sig.reshape(-1), rhs=rhs)

_DIMS_STREAM = 0x5EED_D135


def instance_dims(cfg: dict, index: int):
    """(N, nx, nu) of instance ``index``: fixed, or drawn from the instance's own
    dimension stream (config seed, dims, index) for uneven workloads."""
    if isinstance(cfg["N"], tuple):
        g = np.random.Generator(np.random.PCG64([cfg["seed"], _DIMS_STREAM, index]))
        N = int(g.integers(cfg["N"][0], cfg["N"][1], endpoint=True))
        nx = int(g.integers(cfg["nx"][0], cfg["nx"][1], endpoint=True))
        nu = int(g.integers(cfg["nu"][0], cfg["nu"][1], endpoint=True))
        return N, nx, nu
    return int(cfg["N"]), int(cfg["nx"]), int(cfg["nu"])


def config_dims(cfg: dict, batch: Optional[int] = None, indices: Optional[Sequence[int]] = None):
    """Per-instance (N, nx, nu) arrays of a config (instances 0..batch-1 or ``indices``)."""
    if indices is None:
        indices = range(cfg["batch"] if batch is None else batch)
    d = np.array([instance_dims(cfg, int(i)) for i in indices], dtype=np.int32).reshape(-1, 3)
    return d[:, 0].copy(), d[:, 1].copy(), d[:, 2].copy()


def _spd(g, count, n):
    M = g.standard_normal((count, n, n))
    return M @ M.transpose(0, 2, 1) / n + 0.1 * np.eye(n)


def make_instance(cfg, index: int, *, N: Optional[int] = None, nx: Optional[int] = None,
                  nu: Optional[int] = None, nrhs: Optional[int] = None) -> OCPInstance:
    """Draw instance ``index`` of ``cfg`` (a CONFIGS key or dict).

    Every instance has its own PCG64 stream seeded by (config seed, 1, index),
    so any subset of a batch can be regenerated alone.  Draw order: A, B, M
    (for Q), P (for R), S, Sigma, then (q, r, c, x0) for each right-hand side.
    ``N``/``nx``/``nu`` override the config's dimensions (small test cases).
    """
    if isinstance(cfg, str):
        cfg = CONFIGS[cfg]
    dN, dnx, dnu = instance_dims(cfg, index)
    N = dN if N is None else int(N)
    nx = dnx if nx is None else int(nx)
    nu = dnu if nu is None else int(nu)
    nrhs = cfg["nrhs"] if nrhs is None else nrhs
    g = np.random.Generator(np.random.PCG64([cfg["seed"], 1, index]))
    if cfg.get("kind") == "mass_spring":
        return _make_mass_spring(cfg, index, N, nrhs, g)

    # A_k: Gaussian scaled to spectral radius 0.95
    G = g.standard_normal((N, nx, nx))
    rho = np.abs(np.linalg.eigvals(G)).max(axis=1)
    A = 0.95 * G / rho[:, None, None]
    # B_k ~ N(0, 1/nx)  (variance 1/nx)
    B = g.standard_normal((N, nx, nu)) / np.sqrt(nx)
    # Q_k = M M^T / nx + 0.1 I (k = 0..N), R_k = P P^T / nu + 0.1 I
    Q = _spd(g, N + 1, nx)
    if cfg.get("QN_equals_Q0"):
        Q[N] = Q[0]
    R = _spd(g, N, nu)
    if cfg["S"]:
        S = 0.1 * g.standard_normal((N, nu, nx))
        # keep the stage block [R S; S^T Q] SPD: shift both diagonal blocks so
        # that its smallest eigenvalue is at least 0.05
        H = np.zeros((N, nu + nx, nu + nx))
        H[:, :nu, :nu] = R
        H[:, :nu, nu:] = S
        H[:, nu:, :nu] = S.transpose(0, 2, 1)
        H[:, nu:, nu:] = Q[:N]
        lmin = np.linalg.eigvalsh(H)[:, 0]
        delta = np.maximum(0.0, 0.05 - lmin)
        R = R + delta[:, None, None] * np.eye(nu)
        Q[:N] = Q[:N] + delta[:, None, None] * np.eye(nx)
    else:
        S = np.zeros((N, nu, nx))
    Sigma = None
    if cfg["sigma"] is not None:
        lo, hi = cfg["sigma"]
        Sigma = 10.0 ** g.uniform(np.log10(lo), np.log10(hi), size=(N + 1) * (nu + nx))
    rhs = []
    for _ in range(nrhs):
        q = g.standard_normal((N + 1) * nx)
        r = g.standard_normal(N * nu)
        c = g.standard_normal(N * nx)
        x0 = g.standard_normal(nx)
        rhs.append((q, r, c, x0))
    return OCPInstance(N=N, nx=nx, nu=nu, Q=blocks_to_flat(Q), R=blocks_to_flat(R),
                       S=blocks_to_flat(S), A=blocks_to_flat(A), B=blocks_to_flat(B),
                       Sigma=Sigma, rhs=rhs)


def _make_chunk(args):
    cfg, idx, overrides = args
    return [make_instance(cfg, int(i), **overrides) for i in idx]


def make_batch(cfg, indices: Optional[Sequence[int]] = None, *, instances=None, workers: int = 0,
               **overrides) -> Batch:
    """Concatenate instances (``indices`` of ``cfg``, default all) into a Batch.

    ``workers > 1`` draws the instances in a pool of that many processes
    (spawn context; every instance has its own seed stream, so the result is
    identical to the serial draw).  ``workers = 0`` picks one per host core
    for batches of more than 64 instances."""
    if instances is None:
        if isinstance(cfg, str):
            cfg = CONFIGS[cfg]
        if indices is None:
            indices = range(cfg["batch"])
        indices = [int(i) for i in indices]
        import os
        if workers == 0:
            workers = min(32, os.cpu_count() or 1) if len(indices) > 64 else 1
        if workers > 1:
            import concurrent.futures
            import multiprocessing
            chunks = [indices[i::workers * 4] for i in range(workers * 4)]
            chunks = [c for c in chunks if c]
            ctx = multiprocessing.get_context("spawn")
            # one BLAS thread per worker process (spawned children inherit the environment)
            keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
            saved = {k: os.environ.get(k) for k in keys}
            for k in keys:
                os.environ[k] = "1"
            try:
                with concurrent.futures.ProcessPoolExecutor(max_workers=workers, mp_context=ctx) as ex:
                    parts = list(ex.map(_make_chunk, [(cfg, c, overrides) for c in chunks]))
            finally:
                for k, v in saved.items():
                    if v is None:
                        os.environ.pop(k, None)
                    else:
                        os.environ[k] = v
            by_index = {}
            for c, part in zip(chunks, parts):
                for i, inst in zip(c, part):
                    by_index[i] = inst
            instances = [by_index[i] for i in indices]
        else:
            instances = [make_instance(cfg, i, **overrides) for i in indices]
    insts = list(instances)
    cat = lambda name: np.concatenate([getattr(x, name) for x in insts]) if insts else np.zeros(0)
    has_sigma = any(x.Sigma is not None for x in insts)
    if has_sigma:
        sig = np.concatenate([x.Sigma if x.Sigma is not None else np.zeros((x.N + 1) * (x.nu + x.nx))
                              for x in insts])
    else:
        sig = None
    nrhs = min(len(x.rhs) for x in insts) if insts else 0
    rhs = []
    for j in range(nrhs):
        rhs.append(tuple(np.concatenate([x.rhs[j][t] for x in insts]) for t in range(4)))
    return Batch(N=np.array([x.N for x in insts], np.int32), nx=np.array([x.nx for x in insts], np.int32),
                 nu=np.array([x.nu for x in insts], np.int32), Q=cat("Q"), R=cat("R"), S=cat("S"),
                 A=cat("A"), B=cat("B"), Sigma=sig, rhs=rhs, instances=insts)


# ---------------------------------------------------------------------------
# Augmented Lagrangian inner problem (paper Sec. 5): inequality constraints
# b_l <= C_k x^k + D_k u^k <= b_u (k < N) and b_l <= C_N x^N <= b_u, multiplier
# estimates y, diagonal penalties Sigma, proximal weights Gamma and centres, and
# the current iterate (u, x).  Draws only.
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class ALMData:
    """Flat layout per instance (float64, blocks column-major):
        C     (N+1) blocks ny*nx    D  N blocks ny*nu
        bl, bu, y, sig   (N+1)*ny   (box, multiplier estimate, Sigma_k diagonal)
        gx  nx, gu  nu              (diagonals of Gamma_x^{-1}, Gamma_u^{-1})
        xbar (N+1)*nx, ubar N*nu    (proximal centres)
        u  N*nu, x  (N+1)*nx        (current iterate; x^0 is the fixed x_init)
    A batch concatenates the arrays of each kind in instance order (ny may
    differ between instances)."""
    ny: object
    C: np.ndarray
    D: np.ndarray
    bl: np.ndarray
    bu: np.ndarray
    y: np.ndarray
    sig: np.ndarray
    gx: np.ndarray
    gu: np.ndarray
    xbar: np.ndarray
    ubar: np.ndarray
    u: np.ndarray
    x: np.ndarray


def make_alm(inst: OCPInstance, ny: int, seed: int, index: int = 0, bounds: str = "mixed",
             sigma=(1e-2, 1e4)) -> ALMData:
    """Constraint data and an iterate for one instance.  C ~ N(0, 1/nx) and
    D ~ N(0, 1/nu) entries, iterate u, x ~ N(0, 1), y ~ 0.1 N(0, 1), Sigma
    log-uniform in `sigma`, Gamma^{-1} diagonals log-uniform in [1e-3, 1e-1],
    centres = iterate + 0.1 N(0, 1).  Bounds: "mixed" draws a box around
    [-1, 1] (each row's interval jittered), so that some rows are active and
    some not; "inactive" uses [-1e6, 1e6]; "fixed" alternates rows that stay
    inactive ([-1e6, 1e6]) and rows that are active on either side of a box
    far from the origin ([1e3, 2e3] or [-2e3, -1e3]); with penalties small
    against the cost's curvature a Newton step keeps that active set."""
    N, nx, nu = inst.N, inst.nx, inst.nu
    g = np.random.Generator(np.random.PCG64([seed, 7, index]))
    C = g.standard_normal((N + 1, ny, nx)) / np.sqrt(nx)
    D = g.standard_normal((N, ny, nu)) / np.sqrt(nu)
    u = g.standard_normal(N * nu)
    x = g.standard_normal((N + 1) * nx)
    y = 0.1 * g.standard_normal((N + 1) * ny)
    lo, hi = sigma
    sig = 10.0 ** g.uniform(np.log10(lo), np.log10(hi), size=(N + 1) * ny)
    gx = 10.0 ** g.uniform(-3.0, -1.0, size=nx)
    gu = 10.0 ** g.uniform(-3.0, -1.0, size=nu)
    xbar = x + 0.1 * g.standard_normal(x.shape)
    ubar = u + 0.1 * g.standard_normal(u.shape)
    m = (N + 1) * ny
    if bounds == "mixed":
        bl = -1.0 + 0.5 * g.standard_normal(m)
        bu = bl + 2.0 * g.uniform(0.5, 1.5, size=m)
    elif bounds == "inactive":
        bl, bu = np.full(m, -1e6), np.full(m, 1e6)
    elif bounds == "fixed":
        row = np.arange(m) % ny
        side = g.choice([-1.0, 1.0], size=m)
        bl = np.where(row % 2 == 0, -1e6, np.where(side > 0, 1e3, -2e3))
        bu = np.where(row % 2 == 0, 1e6, np.where(side > 0, 2e3, -1e3))
    else:
        raise ValueError(bounds)
    return ALMData(ny=ny, C=blocks_to_flat(C), D=blocks_to_flat(D), bl=bl, bu=bu, y=y, sig=sig, gx=gx, gu=gu,
                   xbar=xbar, ubar=ubar, u=u, x=x)


def config_alm(cfg, instances: Sequence[OCPInstance], indices: Sequence[int]) -> List[ALMData]:
    """The constraint data and iterate of a config with an ``alm`` entry, per instance."""
    if isinstance(cfg, str):
        cfg = CONFIGS[cfg]
    a = cfg["alm"]
    return [make_alm(inst, a["ny"], seed=cfg["seed"], index=int(i), bounds=a["bounds"], sigma=a["sigma"])
            for inst, i in zip(instances, indices)]


def concat_alm(items: Sequence[ALMData]) -> ALMData:
    """Batch layout: each kind concatenated in instance order; ny becomes an int32 array."""
    cat = lambda k: np.concatenate([getattr(a, k) for a in items])
    return ALMData(ny=np.array([a.ny for a in items], np.int32), **{k: cat(k) for k in (
        "C", "D", "bl", "bu", "y", "sig", "gx", "gu", "xbar", "ubar", "u", "x")})
