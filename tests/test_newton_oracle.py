"""Pins of the Newton-system oracle (paper Sec. 5: eqs. ocp-al-funcs,
qpalm-ocp-hessians, newton-sys-with-x0, elim-x0) against facts that do not go
through its formulas: the gradient is the derivative of the augmented
Lagrangian's value (written from the squared distance to the box), the
generalized Hessian is the derivative of the gradient where the active set does
not change, a problem without constraints reduces to an LQ problem solved
directly, and one Newton step reaches a stationary point when the active set
stays fixed."""
import numpy as np
import pytest

import oracle
from oracle import newton
from paper_2512_09058_gb300 import inputs


def _case(N, nx, nu, ny, bounds, seed=0, S=True, sigma=(1e-2, 1e4)):
    cfg = dict(batch=1, N=N, nx=nx, nu=nu, S=S, sigma=None, nrhs=1, QN_equals_Q0=False, seed=seed)
    inst = inputs.make_instance(cfg, 0)
    alm = inputs.make_alm(inst, ny, seed=seed + 100, bounds=bounds, sigma=sigma)
    q, r, f, x0 = inst.rhs[0]
    return inst, alm, q, r, f, x0


def _directional(inst, g, du, dx):
    """Sum_k r~_k . du_k + sum_{k>=1} q~_k . dx_k (x^0 is fixed)."""
    nx = inst.nx
    return float(g["r"] @ du + g["q"][nx:] @ dx[nx:])


@pytest.mark.parametrize("dims", [(6, 3, 2, 4), (9, 5, 3, 8), (4, 2, 1, 3)])
def test_gradient_is_the_derivative_of_the_al_value(dims):
    inst, alm, q, r, f, x0 = _case(*dims, bounds="mixed", seed=dims[0])
    g = newton.newton_assembly(inst, alm, q, r, f, x0, alm.u, alm.x)
    assert 0 < g["active"].sum() < g["active"].size       # a mix of active and inactive rows
    rng = np.random.default_rng(1)
    for _ in range(5):
        du, dx = rng.standard_normal(alm.u.shape), rng.standard_normal(alm.x.shape)
        dx[:inst.nx] = 0.0
        h = 1e-6
        vp = newton.al_value(inst, alm, q, r, x0, alm.u + h * du, alm.x + h * dx)
        vm = newton.al_value(inst, alm, q, r, x0, alm.u - h * du, alm.x - h * dx)
        fd = (vp - vm) / (2 * h)
        an = _directional(inst, g, du, dx)
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (fd, an)


def _hessian_times(inst, g, du, dx):
    """The Newton system's Hessian part applied to (du, dx): rows of u^k and x^k."""
    N, nx, nu = inst.N, inst.nx, inst.nu
    blk = lambda a, k, r, c: a[k * r * c:(k + 1) * r * c].reshape(c, r).T
    hu = np.zeros(N * nu)
    hx = np.zeros((N + 1) * nx)
    for k in range(N + 1):
        dxk = dx[k * nx:(k + 1) * nx]
        hx[k * nx:(k + 1) * nx] = blk(g["Q"], k, nx, nx) @ dxk
        if k < N:
            duk = du[k * nu:(k + 1) * nu]
            Rk, Sk = blk(g["R"], k, nu, nu), blk(g["S"], k, nu, nx)
            hu[k * nu:(k + 1) * nu] = Rk @ duk + Sk @ dxk
            hx[k * nx:(k + 1) * nx] += Sk.T @ duk
    return hu, hx


@pytest.mark.parametrize("dims", [(6, 3, 2, 4), (8, 4, 3, 7)])
def test_hessian_is_the_derivative_of_the_gradient(dims):
    inst, alm, q, r, f, x0 = _case(*dims, bounds="mixed", seed=10 + dims[0])
    g0 = newton.newton_assembly(inst, alm, q, r, f, x0, alm.u, alm.x)
    rng = np.random.default_rng(2)
    du, dx = 1e-7 * rng.standard_normal(alm.u.shape), 1e-7 * rng.standard_normal(alm.x.shape)
    dx[:inst.nx] = 0.0
    g1 = newton.newton_assembly(inst, alm, q, r, f, x0, alm.u + du, alm.x + dx)
    assert np.array_equal(g0["active"], g1["active"])       # the step stays in one piece
    hu, hx = _hessian_times(inst, g0, du, dx)
    nx = inst.nx
    dgu, dgx = g1["r"] - g0["r"], (g1["q"] - g0["q"])[nx:]
    scale = np.abs(np.concatenate([hu, hx[nx:]])).max()
    assert np.abs(dgu - hu).max() <= 1e-6 * scale
    assert np.abs(dgx - hx[nx:]).max() <= 1e-6 * scale


def test_without_constraints_the_newton_step_solves_the_proximal_lq_problem():
    """C = D = 0 and an unbounded box: the inner problem is the LQ problem with
    Q + Gamma_x^{-1}, R + Gamma_u^{-1} and linear terms shifted by the proximal
    centres; one Newton step from any point lands on its solution, computed here
    without the assembly."""
    inst, alm, q, r, f, x0 = _case(7, 4, 2, 3, bounds="inactive", seed=3)
    alm.C[:] = 0.0
    alm.D[:] = 0.0
    g = newton.newton_assembly(inst, alm, q, r, f, x0, alm.u, alm.x)
    assert not g["active"].any()
    N, nx, nu = inst.N, inst.nx, inst.nu
    # Newton step: the KKT system of the assembled blocks, right-hand side from (q~, r~, c~), dx^0 = 0
    step_inst = inputs.OCPInstance(N=N, nx=nx, nu=nu, Q=g["Q"], R=g["R"], S=g["S"], A=inst.A, B=inst.B,
                                   Sigma=None, rhs=[])
    b = oracle.build_rhs(step_inst, g["q"], g["r"], g["c"], np.zeros(nx))
    d = oracle.riccati_solve(step_inst, b).reshape(N, nu + 2 * nx)
    u1 = alm.u + d[:, :nu].reshape(-1)
    x1 = alm.x[nx:] + d[:, nu:nu + nx].reshape(-1)
    # the proximal LQ problem solved directly
    gxI = np.tile(np.diag(alm.gx).T.reshape(-1), N + 1)
    guI = np.tile(np.diag(alm.gu).T.reshape(-1), N)
    lq = inputs.OCPInstance(N=N, nx=nx, nu=nu, Q=inst.Q + gxI, R=inst.R + guI, S=inst.S, A=inst.A, B=inst.B,
                            Sigma=None, rhs=[])
    qp = q - np.tile(alm.gx, N + 1) * alm.xbar
    rp = r - np.tile(alm.gu, N) * alm.ubar
    z = oracle.riccati_solve(lq, oracle.build_rhs(lq, qp, rp, f, x0)).reshape(N, nu + 2 * nx)
    assert np.abs(u1 - z[:, :nu].reshape(-1)).max() <= 1e-10 * max(1.0, np.abs(u1).max())
    assert np.abs(x1 - z[:, nu:nu + nx].reshape(-1)).max() <= 1e-10 * max(1.0, np.abs(x1).max())


@pytest.mark.parametrize("dims", [(6, 3, 2, 4), (10, 4, 2, 6), (5, 6, 3, 9)])
def test_newton_step_is_stationary_when_the_active_set_is_fixed(dims):
    """Rows whose box is far from every reachable point keep their side of it
    (penalties small against the cost's curvature, so the step moves each row a
    small part of the way to its box), so the inner problem is one quadratic and
    one Newton step solves it: the optimality conditions (gradient + multiplier
    terms, dynamics) vanish at the new point with the step's multipliers."""
    inst, alm, q, r, f, x0 = _case(*dims, bounds="fixed", seed=20 + dims[0], sigma=(1e-3, 1e-1))
    g = newton.newton_assembly(inst, alm, q, r, f, x0, alm.u, alm.x)
    assert 0 < g["active"].sum() < g["active"].size
    N, nx, nu = inst.N, inst.nx, inst.nu
    step_inst = inputs.OCPInstance(N=N, nx=nx, nu=nu, Q=g["Q"], R=g["R"], S=g["S"], A=inst.A, B=inst.B,
                                   Sigma=None, rhs=[])
    b = oracle.build_rhs(step_inst, g["q"], g["r"], g["c"], np.zeros(nx))
    d = oracle.riccati_solve(step_inst, b).reshape(N, nu + 2 * nx)
    u1 = alm.u + d[:, :nu].reshape(-1)
    x1 = alm.x.copy()
    x1[nx:] += d[:, nu:nu + nx].reshape(-1)
    lam = d[:, nu + nx:].reshape(-1)
    g1 = newton.newton_assembly(inst, alm, q, r, f, x0, u1, x1)
    assert np.array_equal(g["active"], g1["active"])
    res = newton.stationarity(inst, alm, q, r, f, x0, u1, x1, lam)
    r0 = newton.stationarity(inst, alm, q, r, f, x0, alm.u, alm.x, np.zeros(N * nx))
    assert np.abs(res).max() <= 1e-12 * np.abs(r0).max(), (np.abs(res).max(), np.abs(r0).max())


def test_active_set_and_multiplier_estimate_by_hand():
    """One stage, one constraint row: the active flag and y^ from the definition
    with hand-picked numbers (w = C x + D u = 1.5; Sigma = 2, y = 1 -> w + y/Sigma
    = 2 is above bu = 1.75: active, y^ = 1 + 2 (1.5 - 1.75) = 0.5; with bu = 3 the
    row is inactive and y^ = 0)."""
    inst = inputs.OCPInstance(N=1, nx=1, nu=1, Q=np.array([1.0, 1.0]), R=np.array([1.0]), S=np.array([0.0]),
                              A=np.array([0.0]), B=np.array([1.0]), Sigma=None, rhs=[])
    for bu, act, yh in [(1.75, True, 0.5), (3.0, False, 0.0)]:
        alm = inputs.ALMData(ny=1, C=np.array([1.0, 0.0]), D=np.array([0.5]), bl=np.array([-5.0, -5.0]),
                             bu=np.array([bu, 5.0]), y=np.array([1.0, 0.0]), sig=np.array([2.0, 1.0]),
                             gx=np.array([0.0]), gu=np.array([0.0]), xbar=np.zeros(2), ubar=np.zeros(1),
                             u=np.array([1.0]), x=np.array([0.0, 0.0]))
        g = newton.newton_assembly(inst, alm, np.zeros(2), np.zeros(1), np.zeros(1), np.array([1.0]),
                                   alm.u, alm.x)
        assert bool(g["active"][0]) == act
        assert abs(g["yhat"][0] - yh) <= 1e-15
        # H_0: R + D^T Sigma^J D = 1 + (2 * 0.25 if active)
        assert abs(g["R"][0] - (1.0 + (0.5 if act else 0.0))) <= 1e-15
