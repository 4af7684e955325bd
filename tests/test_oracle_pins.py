"""Pins of the CPU oracle against facts that do not come from the oracle itself.

* brute force: dense KKT assembly solved by numpy's LAPACK solver (and by the
  oracle's own elimination, itself checked against numpy);
* closed forms: the N = 1 scalar KKT solution by hand elimination, and the
  scalar discrete algebraic Riccati equation (positive root of a quadratic);
* optimality: the primal trajectory minimises the cost computed by a direct
  rollout of the dynamics from x_init (no KKT code involved);
* invariants: K symmetric with inertia (N*(nu+nx) positive, N*nx negative
  eigenvalues, Sylvester), cost-to-go matrices P_k symmetric positive
  definite, linearity of the solve;
* adjoint: central finite differences of the oracle solve.
"""
import numpy as np
import pytest

import oracle
from paper_2512_09058_gb300 import inputs


def _small(seed, N, nx, nu, S=True, sigma=None, nrhs=1):
    cfg = dict(batch=1, N=N, nx=nx, nu=nu, S=S, sigma=sigma, nrhs=nrhs, QN_equals_Q0=False, seed=seed)
    return inputs.make_instance(cfg, 0)


CASES = [(1, 1, 1), (1, 3, 2), (2, 2, 1), (3, 4, 2), (5, 3, 3), (8, 4, 2), (6, 5, 1), (4, 2, 4)]


def _rollout_cost(inst, u, q, r, c, x0, Sigma=True):
    """Cost and trajectory of controls u (N, nu) rolled out from x_init."""
    N, nx, nu = inst.N, inst.nx, inst.nu
    x = np.zeros((N + 1, nx))
    x[0] = x0
    for k in range(N):
        x[k + 1] = inst.Ak(k) @ x[k] + inst.Bk(k) @ u[k] + c[k * nx:(k + 1) * nx]
    J = 0.0
    for k in range(N):
        Rk = inst.Rk(k) + np.diag(inst.Sigma_u(k))
        Qk = inst.Qk(k) + np.diag(inst.Sigma_x(k)) if k > 0 else inst.Qk(k)
        Sk = inst.Sk(k)
        J += 0.5 * u[k] @ Rk @ u[k] + u[k] @ Sk @ x[k] + 0.5 * x[k] @ Qk @ x[k]
        J += r[k * nu:(k + 1) * nu] @ u[k] + q[k * nx:(k + 1) * nx] @ x[k]
    QN = inst.Qk(N) + np.diag(inst.Sigma_x(N))
    J += 0.5 * x[N] @ QN @ x[N] + q[N * nx:] @ x[N]
    return J, x


def _split(inst, z):
    N, nx, nu = inst.N, inst.nx, inst.nu
    w = nu + 2 * nx
    Z = z.reshape(N, w)
    return Z[:, :nu], Z[:, nu:nu + nx], Z[:, nu + nx:]


@pytest.mark.parametrize("N,nx,nu", CASES)
@pytest.mark.parametrize("with_sigma", [False, True])
def test_riccati_matches_dense_bruteforce(N, nx, nu, with_sigma):
    inst = _small(7 * N + nx, N, nx, nu, sigma=(1e-2, 1e2) if with_sigma else None)
    q, r, c, x0 = inst.rhs[0]
    b = oracle.build_rhs(inst, q, r, c, x0)
    K = oracle.kkt_dense(inst)
    z_np = np.linalg.solve(K, b)            # library LU (LAPACK gesv)
    z = oracle.riccati_solve(inst, b)
    assert np.linalg.norm(z - z_np) <= 1e-12 * np.linalg.norm(z_np)
    z_ge = oracle.dense_solve(K, b)
    assert np.linalg.norm(z_ge - z_np) <= 1e-12 * np.linalg.norm(z_np)


@pytest.mark.parametrize("N,nx,nu", CASES)
def test_dense_matrix_equals_structured_matvec_and_is_symmetric(N, nx, nu):
    inst = _small(100 + N, N, nx, nu, sigma=(1e-1, 1e1))
    K = oracle.kkt_dense(inst)
    assert np.array_equal(K, K.T)
    rng = np.random.default_rng(N)
    for _ in range(3):
        v = rng.standard_normal(K.shape[0])
        assert np.allclose(K @ v, oracle.kkt_matvec(inst, v), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("N,nx,nu", CASES)
def test_abs_matvec_equals_dense_abs_product(N, nx, nu):
    inst = _small(150 + N, N, nx, nu, sigma=(1e-3, 1e3))
    K = oracle.kkt_dense(inst)
    rng = np.random.default_rng(7 + N)
    v = rng.standard_normal(K.shape[0])
    assert np.allclose(np.abs(K) @ np.abs(v), oracle.kkt_abs_matvec(inst, v), rtol=1e-13, atol=0.0)


def _exact_residual(inst, z, b):
    """||b - K z|| / ||b|| in exact rational arithmetic from the optimality
    conditions of the OCP (gradient of the Lagrangian in u^k and x^{k+1}, the
    dynamics), with Sigma on the diagonals of R and Q; only the final norm is
    rounded (to float64, after an exact sum of squares)."""
    from fractions import Fraction as F
    N, nx, nu = inst.N, inst.nx, inst.nu
    w = nu + 2 * nx
    Z = [F(float(v)) for v in z]
    res = []
    for k in range(N):
        u = Z[k * w:k * w + nu]
        xn = Z[k * w + nu:k * w + nu + nx]
        lam = Z[k * w + nu + nx:(k + 1) * w]
        xk = Z[(k - 1) * w + nu:(k - 1) * w + nu + nx] if k > 0 else None
        Rk, Bk = inst.Rk(k), inst.Bk(k)
        su = inst.Sigma_u(k) if inst.Sigma is not None else np.zeros(nu)
        for i in range(nu):
            g = sum(F(float(Rk[i, j])) * u[j] for j in range(nu)) + F(float(su[i])) * u[i]
            g += sum(F(float(Bk[j, i])) * lam[j] for j in range(nx))
            if xk is not None and inst.S is not None:
                g += sum(F(float(inst.Sk(k)[i, j])) * xk[j] for j in range(nx))
            res.append(F(float(b[k * w + i])) - g)
        j1 = k + 1
        Qj = inst.Qk(j1)
        sx = inst.Sigma_x(j1) if inst.Sigma is not None else np.zeros(nx)
        for i in range(nx):
            g = sum(F(float(Qj[i, m])) * xn[m] for m in range(nx)) + F(float(sx[i])) * xn[i] - lam[i]
            if j1 < N:
                un = Z[j1 * w:j1 * w + nu]
                ln = Z[j1 * w + nu + nx:(j1 + 1) * w]
                g += sum(F(float(inst.Ak(j1)[m, i])) * ln[m] for m in range(nx))
                if inst.S is not None:
                    g += sum(F(float(inst.Sk(j1)[m, i])) * un[m] for m in range(nu))
            res.append(F(float(b[k * w + nu + i])) - g)
        for i in range(nx):
            g = sum(F(float(Bk[i, m])) * u[m] for m in range(nu)) - xn[i]
            if xk is not None:
                g += sum(F(float(inst.Ak(k)[i, m])) * xk[m] for m in range(nx))
            res.append(F(float(b[k * w + nu + nx + i])) - g)
    rr = sum(r * r for r in res)
    bb = sum(F(float(v)) ** 2 for v in b)
    return float(np.sqrt(float(rr / bb)))


def _near_solutions(seed, N, nx, nu, sigma):
    inst = _small(300 + seed, N, nx, nu, sigma=sigma)
    q, r, c, x0 = inst.rhs[0]
    b = oracle.build_rhs(inst, q, r, c, x0)
    z0 = oracle.riccati_solve(inst, b)
    rng = np.random.default_rng(seed)
    # the solution itself (residual near the float64 floor) and a perturbed one
    return inst, b, (z0, z0 * (1.0 + 1e-9 * rng.standard_normal(z0.size)))


def test_accurate_residual_equals_exact_rational_arithmetic():
    """kkt_residual (compensated rows) against the residual computed exactly with
    fractions, on badly scaled instances (Sigma in [1e-6, 1e6]) where the terms
    of a row cancel by many orders of magnitude."""
    for seed, (N, nx, nu) in enumerate([(4, 3, 2), (5, 4, 1), (3, 5, 3)]):
        inst, b, zs = _near_solutions(seed, N, nx, nu, (1e-6, 1e6))
        for z in zs:
            exact = _exact_residual(inst, z, b)
            assert abs(oracle.kkt_residual(inst, z, b) - exact) <= 1e-14 * exact + 1e-24


def test_residual_evaluation_bound_holds():
    """A plain float64 evaluation of the residual of a near-solution differs from
    the exact residual (fractions) by at most the stated bound."""
    for seed, (N, nx, nu) in enumerate([(4, 3, 2), (5, 4, 1), (3, 5, 3)]):
        inst, b, zs = _near_solutions(seed, N, nx, nu, (1e-6, 1e6))
        for z in zs:
            exact = _exact_residual(inst, z, b)
            bound = oracle.residual_eval_bound(inst, z, b)
            assert abs(oracle.kkt_residual_fp64(inst, z, b) - exact) <= bound
            assert bound < 1e-10   # informative at the 1e-10 refinement target


@pytest.mark.parametrize("N,nx,nu", CASES)
def test_inertia_of_kkt_matrix(N, nx, nu):
    inst = _small(200 + N, N, nx, nu)
    ev = np.linalg.eigvalsh(oracle.kkt_dense(inst))
    assert (ev > 0).sum() == N * (nu + nx)
    assert (ev < 0).sum() == N * nx


def test_scalar_single_stage_closed_form():
    # N = 1, nx = nu = 1: R u + B l = bu ; Q x - l = bx ; B u - x = bl.
    inst = _small(3, 1, 1, 1, S=False)
    R, Q, B = inst.Rk(0)[0, 0], inst.Qk(1)[0, 0], inst.Bk(0)[0, 0]
    b = np.array([0.7, -1.3, 0.4])
    u = (b[0] + B * Q * b[2] + B * b[1]) / (R + B * B * Q)
    x = B * u - b[2]
    lam = Q * x - b[1]
    z = oracle.riccati_solve(inst, b)
    assert np.allclose(z, [u, x, lam], rtol=1e-14, atol=1e-14)


def test_scalar_riccati_converges_to_dare_root():
    # time-invariant scalar problem, long horizon: P_1 -> positive root of
    # B^2 P^2 + ((1-A^2) R - Q B^2 + 2 A B S) P + (S^2 - Q R) = 0
    N = 400
    A, Bv, Q, R, S = 0.9, 0.5, 2.0, 0.7, 0.3
    inst = _small(5, N, 1, 1)
    inst.A[:] = A
    inst.B[:] = Bv
    inst.Q[:] = Q
    inst.R[:] = R
    inst.S[:] = S
    inst.Sigma = None
    _, P = oracle.riccati_solve(inst, np.zeros(inst.kkt_size), return_P=True)
    a2 = Bv * Bv
    a1 = (1 - A * A) * R - Q * Bv * Bv + 2 * A * Bv * S
    a0 = S * S - Q * R
    root = (-a1 + np.sqrt(a1 * a1 - 4 * a2 * a0)) / (2 * a2)
    assert abs(P[0, 0, 0] - root) <= 1e-12 * root
    # the recursion P_N = Q, P_k = g(P_{k+1}) is monotone here: check a few steps by hand
    g = lambda p: Q + A * A * p - (S + A * Bv * p) ** 2 / (R + Bv * Bv * p)
    p = Q
    for k in range(N - 1, N - 6, -1):
        p = g(p)
        assert abs(P[k - 1, 0, 0] - p) <= 1e-13 * p


@pytest.mark.parametrize("N,nx,nu", [(4, 3, 2), (10, 4, 2), (7, 2, 3)])
def test_primal_solution_minimises_rollout_cost(N, nx, nu):
    inst = _small(300 + N, N, nx, nu, sigma=(1e-1, 1e1))
    q, r, c, x0 = inst.rhs[0]
    z = oracle.riccati_solve(inst, oracle.build_rhs(inst, q, r, c, x0))
    u, x, lam = _split(inst, z)
    J0, xr = _rollout_cost(inst, u, q, r, c, x0)
    assert np.allclose(xr[1:], x, rtol=1e-12, atol=1e-12)      # primal feasibility
    rng = np.random.default_rng(N)
    for _ in range(5):
        du = rng.standard_normal(u.shape)
        t = 1e-3
        Jp, _ = _rollout_cost(inst, u + t * du, q, r, c, x0)
        Jm, _ = _rollout_cost(inst, u - t * du, q, r, c, x0)
        assert Jp > J0 and Jm > J0
        # J is quadratic in u: (Jp - Jm) / 2t is the exact directional derivative (= 0)
        assert abs(Jp - Jm) / (2 * t) <= 1e-9 * (1 + abs(J0))
    # terminal multiplier (first KKT row): lambda^{N-1} = Q_N x^N + q^N
    QN = inst.Qk(N) + np.diag(inst.Sigma_x(N))
    assert np.allclose(lam[N - 1], QN @ x[N - 1] + q[N * nx:], rtol=1e-11, atol=1e-11)


def test_cost_to_go_spd_and_linearity():
    inst = _small(11, 12, 4, 2, sigma=(1e-2, 1e2), nrhs=2)
    b1 = oracle.build_rhs(inst, *inst.rhs[0])
    b2 = oracle.build_rhs(inst, *inst.rhs[1])
    z1, P = oracle.riccati_solve(inst, b1, return_P=True)
    for Pk in P:
        assert np.allclose(Pk, Pk.T, rtol=0, atol=1e-12 * np.abs(Pk).max())
        assert np.linalg.eigvalsh(Pk).min() > 0
    z2 = oracle.riccati_solve(inst, b2)
    z12 = oracle.riccati_solve(inst, 2.0 * b1 - 3.0 * b2)
    assert np.allclose(z12, 2.0 * z1 - 3.0 * z2, rtol=1e-12, atol=1e-12)
    assert np.array_equal(oracle.riccati_solve(inst, np.zeros_like(b1)), np.zeros_like(b1))
    # multi-rhs call equals single calls
    Z = oracle.riccati_solve(inst, np.stack([b1, b2]))
    assert np.allclose(Z[0], z1, rtol=1e-14, atol=1e-14) and np.allclose(Z[1], z2, rtol=1e-14, atol=1e-14)


def test_residual_small_on_well_conditioned_workloads():
    for name in ["single_n32_nx8_nu4", "adjoint512_n128_nx24_nu8"]:
        inst = inputs.make_instance(name, 0)
        b = oracle.build_rhs(inst, *inst.rhs[0])
        z = oracle.riccati_solve(inst, b)
        assert oracle.kkt_residual(inst, z, b) <= 1e-12


def _loss_and_grad(z, inst):
    u, x, lam = _split(inst, z)
    L = float((x ** 2).sum() + (u ** 2).sum())
    g = np.zeros_like(z).reshape(inst.N, -1)
    g[:, :inst.nu] = 2 * u
    g[:, inst.nu:inst.nu + inst.nx] = 2 * x
    return L, g.ravel()


def test_adjoint_matches_central_finite_differences():
    inst = _small(21, 6, 3, 2, sigma=(1e-1, 1e1))
    q, r, c, x0 = [a.copy() for a in inst.rhs[0]]

    def loss():
        z = oracle.riccati_solve(inst, oracle.build_rhs(inst, q, r, c, x0))
        return _loss_and_grad(z, inst)[0]

    z = oracle.riccati_solve(inst, oracle.build_rhs(inst, q, r, c, x0))
    _, g = _loss_and_grad(z, inst)
    G = oracle.adjoint(inst, x0, z, g)
    h = 1e-6
    rng = np.random.default_rng(0)

    def fd(arr, idx, partner=None):
        old = arr[idx]
        oldp = arr[partner] if partner is not None else None
        arr[idx] = old + h
        if partner is not None and partner != idx:
            arr[partner] = oldp + h
        Lp = loss()
        arr[idx] = old - h
        if partner is not None and partner != idx:
            arr[partner] = oldp - h
        Lm = loss()
        arr[idx] = old
        if partner is not None and partner != idx:
            arr[partner] = oldp
        return (Lp - Lm) / (2 * h)

    N, nx, nu = inst.N, inst.nx, inst.nu
    checks = []
    for name, arr, grad in [("q", q, G["dq"]), ("r", r, G["dr"]), ("c", c, G["dc"]), ("x0", x0, G["dx0"]),
                            ("B", inst.B, G["dB"]), ("S", inst.S, G["dS"]), ("A", inst.A, G["dA"]),
                            ("Sigma", inst.Sigma, G["dSigma"])]:
        skip = set()
        if name == "q":
            skip = set(range(nx))                   # q_0 does not enter
        if name == "Sigma":
            w = nu + nx
            skip = set(range(nu, w)) | set(range(N * w, N * w + nu))
        idxs = [i for i in rng.choice(len(arr), size=min(10, len(arr)), replace=False) if i not in skip]
        for i in idxs:
            checks.append((name, fd(arr, i), grad[i]))
    # symmetric blocks: perturb (i,j) and (j,i) together; the symmetrised gradient gives G_ij + G_ji
    for name, arr, grad, m, count in [("Q", inst.Q, G["dQ"], nx, N + 1), ("R", inst.R, G["dR"], nu, N)]:
        for _ in range(8):
            k = int(rng.integers(1 if name == "Q" else 0, count))
            i, j = int(rng.integers(m)), int(rng.integers(m))
            a, bb = k * m * m + i + j * m, k * m * m + j + i * m
            expect = grad[a] + (grad[bb] if a != bb else 0.0)
            checks.append((name, fd(arr, a, bb), expect))
    for name, f, gr in checks:
        assert abs(f - gr) <= 1e-6 * max(1.0, abs(gr)), (name, f, gr)


def pad_instance(inst, extra):
    """The OCP with `extra` stages appended after the terminal stage: R = I,
    Q = I, S = A = B = 0, no Sigma, zero right-hand side (paper Sec. 4.6).  The
    dynamics after x^N are x^{k+1} = 0, so the original unknowns keep their
    values and every padded unknown is zero."""
    N, nx, nu = inst.N, inst.nx, inst.nu
    M = N + extra
    eye = lambda n: np.eye(n).T.reshape(-1)
    Q = np.concatenate([inst.Q] + [eye(nx)] * extra)
    R = np.concatenate([inst.R] + [eye(nu)] * extra)
    S = np.concatenate([inst.S] + [np.zeros(nu * nx)] * extra)
    A = np.concatenate([inst.A] + [np.zeros(nx * nx)] * extra)
    B = np.concatenate([inst.B] + [np.zeros(nx * nu)] * extra)
    Sigma = None
    if inst.Sigma is not None:
        Sigma = np.concatenate([inst.Sigma] + [np.zeros(nu + nx)] * extra)
    rhs = []
    for (q, r, c, x0) in inst.rhs:
        rhs.append((np.concatenate([q, np.zeros(extra * nx)]), np.concatenate([r, np.zeros(extra * nu)]),
                    np.concatenate([c, np.zeros(extra * nx)]), x0))
    return inputs.OCPInstance(N=M, nx=nx, nu=nu, Q=Q, R=R, S=S, A=A, B=B, Sigma=Sigma, rhs=rhs)


def test_padding_stages_leave_the_solution_unchanged():
    """Padding reading (Sec. 4.6): stages appended after the terminal stage with
    identity costs, zero dynamics and zero right-hand side do not change the
    solution, and their own unknowns are zero."""
    for seed, (N, nx, nu, extra) in enumerate([(5, 3, 2, 3), (7, 2, 1, 1), (4, 4, 3, 4)]):
        inst = _small(400 + seed, N, nx, nu, sigma=(1e-2, 1e2))
        pad = pad_instance(inst, extra)
        q, r, c, x0 = inst.rhs[0]
        z = oracle.riccati_solve(inst, oracle.build_rhs(inst, q, r, c, x0))
        qp, rp, cp, x0p = pad.rhs[0]
        zp = oracle.riccati_solve(pad, oracle.build_rhs(pad, qp, rp, cp, x0p))
        n = inst.kkt_size
        assert np.linalg.norm(zp[:n] - z) <= 1e-12 * np.linalg.norm(z)
        assert np.linalg.norm(zp[n:]) <= 1e-12 * np.linalg.norm(z)
