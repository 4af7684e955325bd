"""The mass-spring workload generator (Sec. 8.1): the zero-order-hold matrices
agree with an independent classical Runge-Kutta integration of the continuous
model over one sampling interval, and the instances have the paper's costs,
constraint structure and initial states."""
import numpy as np

from paper_2512_09058_gb300 import inputs


def _rk4_zoh(Ac, Bc, Ts, steps=400):
    """Integrate X' = Ac X, X(0) = I and Y' = Ac Y + Bc, Y(0) = 0 over [0, Ts]."""
    nx, nu = Bc.shape
    X, Y = np.eye(nx), np.zeros((nx, nu))
    h = Ts / steps
    fX = lambda X: Ac @ X
    fY = lambda Y: Ac @ Y + Bc
    for _ in range(steps):
        k1, l1 = fX(X), fY(Y)
        k2, l2 = fX(X + 0.5 * h * k1), fY(Y + 0.5 * h * l1)
        k3, l3 = fX(X + 0.5 * h * k2), fY(Y + 0.5 * h * l2)
        k4, l4 = fX(X + h * k3), fY(Y + h * l3)
        X = X + h / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
        Y = Y + h / 6.0 * (l1 + 2 * l2 + 2 * l3 + l4)
    return X, Y


def test_zero_order_hold_matches_runge_kutta():
    for M, N in [(6, 30), (12, 64)]:
        Ad, Bd, Ac, Bc = inputs.mass_spring_dynamics(M, 15.0 / N)
        X, Y = _rk4_zoh(Ac, Bc, 15.0 / N)
        assert np.abs(Ad - X).max() <= 1e-10 and np.abs(Bd - Y).max() <= 1e-10
        # the chain without friction is conservative: eigenvalues of A_d on the unit circle
        assert np.allclose(np.abs(np.linalg.eigvals(Ad)), 1.0, atol=1e-9)


def test_mass_spring_instances():
    cfg = inputs.CONFIGS["massspring150_M18_N96"]
    x = inputs.make_batch("massspring150_M18_N96", [7]).instances[0]
    M = cfg["M"]
    assert (x.N, x.nx, x.nu) == (96, 2 * M, M // 2)
    assert np.array_equal(x.Qk(0), np.eye(x.nx)) and np.array_equal(x.Qk(x.N), np.eye(x.nx))
    assert np.array_equal(x.Rk(3), np.eye(x.nu)) and not x.S.any()
    assert np.array_equal(x.Ak(5), x.Ak(60))
    for k in (0, 50, x.N):
        sx = x.Sigma_x(k)
        assert (sx[M:] == 0).all() and (sx[:M] > 0).all()      # positions boxed, velocities not
    q, r, c, x0 = x.rhs[0]
    assert not q.any() and not r.any() and not c.any()
    assert (np.abs(x0[:M]) <= 3).all() and not x0[M:].any()
