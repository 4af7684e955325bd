"""Newton system of the augmented Lagrangian inner problem (paper Sec. 5,
eqs. ocp-al, ocp-al-funcs, qpalm-ocp-hessians, newton-sys-with-x0, elim-x0),
written out from its definitions in plain numpy, stage by stage.

TEST INFRASTRUCTURE ONLY: only the test-suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this module.  It shares no code
with the CUDA library.

Arguments are duck-typed:
  inst  OCP data ``N, nx, nu, Q, R, S, A, B`` in the flat layout of ``oracle.c``
        (blocks column-major; Q has N+1 blocks, Q_0 unused; S_0, A_0 unused
        except through x_init)
  alm   ``ny`` and the flat arrays ``C`` ((N+1) blocks ny x nx), ``D`` (N blocks
        ny x nu), ``bl, bu, y, sig`` ((N+1) ny each: bounds, multiplier estimate,
        diagonal penalty Sigma_j), ``gx`` (nx: diagonal of Gamma_x^{-1}), ``gu``
        (nu: diagonal of Gamma_u^{-1}), ``xbar`` ((N+1) nx), ``ubar`` (N nu)
  q, r, f, x_init   linear cost terms ((N+1) nx, N nu), dynamics offsets (N nx)
        and initial state, as in the right-hand side of the OCP
  u, x  the current iterate: u (N nu), x ((N+1) nx; x^0 is replaced by x_init,
        the eliminated initial state of eq. elim-x0)

The point of every function is the definition: stage k's constraint block is
w = C_k x^k + D_k u^k (no D term at k = N), the active set J_k is the set of
rows where w + Sigma_k^{-1} y^k lies outside [bl, bu], Sigma^J keeps Sigma on J
and zeroes it elsewhere, and
  y^_k = y^k + Sigma_k (w - Pi(w + Sigma_k^{-1} y^k; [bl, bu])),
  H_k  = [R S; S^T Q]_k + [D^T; C^T] Sigma^J [D C] + diag(Gamma_u^{-1}, Gamma_x^{-1}),
  (r^k, q^k) = [R S; S^T Q]_k (u^k, x^k) + (r_k, q_k) + [D^T; C^T] y^_k
               + (Gamma_u^{-1}(u^k - ubar^k), Gamma_x^{-1}(x^k - xbar^k)),
  q^N = Q_N x^N + q_N + C_N^T y^_N + Gamma_x^{-1}(x^N - xbar^N),
  c^k = B_k u^k + A_k x^k + f^k - x^{k+1}.
"""
from __future__ import annotations

import numpy as np


def _blk(flat, k, rows, cols):
    n = rows * cols
    return np.asarray(flat[k * n:(k + 1) * n]).reshape(cols, rows).T


def _vec(flat, k, n):
    return np.asarray(flat[k * n:(k + 1) * n])


def _state(x, x_init, k, nx):
    return np.asarray(x_init, dtype=np.float64) if k == 0 else _vec(x, k, nx)


def stage_constraints(inst, alm, u, x, x_init, k):
    """(w, active, y^) of stage k (0 <= k <= N)."""
    N, nx, nu, ny = inst.N, inst.nx, inst.nu, alm.ny
    xk = _state(x, x_init, k, nx)
    w = _blk(alm.C, k, ny, nx) @ xk
    if k < N:
        w = w + _blk(alm.D, k, ny, nu) @ _vec(u, k, nu)
    y, sig = _vec(alm.y, k, ny), _vec(alm.sig, k, ny)
    bl, bu = _vec(alm.bl, k, ny), _vec(alm.bu, k, ny)
    zz = w + y / sig
    active = (zz < bl) | (zz > bu)
    proj = np.minimum(np.maximum(zz, bl), bu)
    yhat = y + sig * (w - proj)
    return w, active, yhat


def newton_assembly(inst, alm, q, r, f, x_init, u, x):
    """The blocks and vectors of the Newton system, in the layout of the OCP data:
    Q~ ((N+1) blocks), R~, S~ (N blocks), q~ ((N+1) nx), r~ (N nu), c~ (N nx),
    active ((N+1) ny booleans), y^ ((N+1) ny).  The Newton step (du, dx, lambda)
    solves the KKT system of these blocks with right-hand side built from
    (q~, r~, c~) and a zero initial state (dx^0 = 0)."""
    N, nx, nu, ny = inst.N, inst.nx, inst.nu, alm.ny
    gx, gu = np.asarray(alm.gx), np.asarray(alm.gu)
    Qt = np.zeros((N + 1, nx, nx))
    Rt = np.zeros((N, nu, nu))
    St = np.zeros((N, nu, nx))
    qt = np.zeros((N + 1, nx))
    rt = np.zeros((N, nu))
    ct = np.zeros((N, nx))
    act = np.zeros((N + 1, ny), dtype=bool)
    yh = np.zeros((N + 1, ny))
    for k in range(N + 1):
        w, active, yhat = stage_constraints(inst, alm, u, x, x_init, k)
        act[k], yh[k] = active, yhat
        sJ = np.where(active, _vec(alm.sig, k, ny), 0.0)
        Ck = _blk(alm.C, k, ny, nx)
        xk = _state(x, x_init, k, nx)
        Qk = _blk(inst.Q, k, nx, nx)
        Qt[k] = Qk + Ck.T @ (sJ[:, None] * Ck) + np.diag(gx)
        qk = Qk @ xk + _vec(q, k, nx) + Ck.T @ yhat + gx * (xk - _vec(alm.xbar, k, nx))
        if k < N:
            Dk = _blk(alm.D, k, ny, nu)
            Rk, Sk = _blk(inst.R, k, nu, nu), _blk(inst.S, k, nu, nx)
            uk = _vec(u, k, nu)
            Rt[k] = Rk + Dk.T @ (sJ[:, None] * Dk) + np.diag(gu)
            St[k] = Sk + Dk.T @ (sJ[:, None] * Ck)
            rt[k] = Rk @ uk + Sk @ xk + _vec(r, k, nu) + Dk.T @ yhat + gu * (uk - _vec(alm.ubar, k, nu))
            qk = qk + Sk.T @ uk
            xn = _vec(x, k + 1, nx)
            ct[k] = _blk(inst.B, k, nx, nu) @ uk + _blk(inst.A, k, nx, nx) @ xk + _vec(f, k, nx) - xn
        qt[k] = qk
    flat = lambda a: np.ascontiguousarray(a.transpose(0, 2, 1)).reshape(-1)
    return dict(Q=flat(Qt), R=flat(Rt), S=flat(St), q=qt.reshape(-1), r=rt.reshape(-1), c=ct.reshape(-1),
                active=act.reshape(-1), yhat=yh.reshape(-1))


def al_value(inst, alm, q, r, x_init, u, x):
    """Sum over stages of the augmented Lagrangians of eq. ocp-al-funcs at (u, x)
    (x^0 = x_init): the LQ stage costs, (1/2) dist^2 in the Sigma-norm of
    C x + D u + Sigma^{-1} y to the box, and the proximal terms."""
    N, nx, nu, ny = inst.N, inst.nx, inst.nu, alm.ny
    gx, gu = np.asarray(alm.gx), np.asarray(alm.gu)
    total = 0.0
    for k in range(N + 1):
        xk = _state(x, x_init, k, nx)
        Qk = _blk(inst.Q, k, nx, nx)
        total += 0.5 * xk @ Qk @ xk + _vec(q, k, nx) @ xk
        dx = xk - _vec(alm.xbar, k, nx)
        total += 0.5 * dx @ (gx * dx)
        w = _blk(alm.C, k, ny, nx) @ xk
        if k < N:
            uk = _vec(u, k, nu)
            Rk, Sk = _blk(inst.R, k, nu, nu), _blk(inst.S, k, nu, nx)
            total += 0.5 * uk @ Rk @ uk + uk @ Sk @ xk + _vec(r, k, nu) @ uk
            du = uk - _vec(alm.ubar, k, nu)
            total += 0.5 * du @ (gu * du)
            w = w + _blk(alm.D, k, ny, nu) @ uk
        pt = w + _vec(alm.y, k, ny) / _vec(alm.sig, k, ny)
        dist = pt - np.minimum(np.maximum(pt, _vec(alm.bl, k, ny)), _vec(alm.bu, k, ny))
        total += 0.5 * float(np.sum(_vec(alm.sig, k, ny) * dist * dist))
    return float(total)


def stationarity(inst, alm, q, r, f, x_init, u, x, lam):
    """Residual of the optimality conditions of the inner problem at (u, x, lambda)
    (the Newton system's rows with the step replaced by the point itself):
    r^k + B_k^T lambda^k, q^k + A_k^T lambda^k - lambda^{k-1} (0 < k < N),
    q^N - lambda^{N-1}, c^k; as one vector."""
    N, nx, nu = inst.N, inst.nx, inst.nu
    g = newton_assembly(inst, alm, q, r, f, x_init, u, x)
    lam = np.asarray(lam).reshape(N, nx)
    out = []
    for k in range(N):
        out.append(g["r"][k * nu:(k + 1) * nu] + _blk(inst.B, k, nx, nu).T @ lam[k])
    for k in range(1, N + 1):
        v = g["q"][k * nx:(k + 1) * nx] - lam[k - 1]
        if k < N:
            v = v + _blk(inst.A, k, nx, nx).T @ lam[k]
        out.append(v)
    out.append(g["c"])
    return np.concatenate(out)
