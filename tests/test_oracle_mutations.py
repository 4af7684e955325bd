"""The oracle's pins catch plausible mistakes: each mutant below is the oracle's
C source with one planted error (a dropped term, a wrong sign, a transposed
operand), compiled to its own library in a temporary folder; the pin battery
of tests/test_oracle_pins.py, run against that library, must fail for every
mutant, and pass for the unmodified source compiled the same way.  Every
mutation stays inside the arrays it touches (signs, dropped terms, transposes
of square blocks), so a mutant computes wrong numbers but never faults.
The Newton-system oracle (numpy) gets the same treatment against the pins of
tests/test_newton_oracle.py.
"""
import os
import subprocess
import types

import pytest

import oracle
import test_newton_oracle as npins
import test_oracle_pins as pins

SRC_DIR = os.path.dirname(os.path.abspath(oracle.__file__))

# (name, text in oracle.c, replacement); each text occurs exactly once
MUTANTS = [
    ("structured K z: sign of the -I coupling in the x rows",
     "for (int i = 0; i < nx; ++i) yx[i] -= lam[i];", "for (int i = 0; i < nx; ++i) yx[i] += lam[i];"),
    ("dense K: sign of the -I coupling in the x rows",
     "for (int a = 0; a < nx; ++a) KK(ix + a, il + a) = -1.0;", "for (int a = 0; a < nx; ++a) KK(ix + a, il + a) = 1.0;"),
    ("dense K: A^T block of the x rows not transposed",
     "KK(ix + a, ilj + c) = blkA(&p, j)[IX(c, a, nx)];", "KK(ix + a, ilj + c) = blkA(&p, j)[IX(a, c, nx)];"),
    ("Riccati: S dropped from H_ux",
     "Hux[i] += blkS(&p, k)[i];", "Hux[i] += 0.0 * blkS(&p, k)[i];"),
    ("Riccati: sign of q in the affine cost-to-go",
     "pk[i] += xn[i] - bx[i];", "pk[i] += xn[i] + bx[i];"),
    ("Riccati: A transposed in the forward rollout",
     "s += blkA(&p, k)[IX(i, j, nx)] * xs[j];", "s += blkA(&p, k)[IX(j, i, nx)] * xs[j];"),
    ("Sigma_x dropped from the effective Q (Riccati and K alike)",
     "out[IX(i, i, nx)] += p->Sigma[(size_t)k * (nu + nx) + nu + i];",
     "out[IX(i, i, nx)] += 0.0 * p->Sigma[(size_t)k * (nu + nx) + nu + i];"),
    ("accurate residual: Sigma_u term dropped",
     "acc2_sub_prod(&yu[i], Sigma[(size_t)k * (nu + nx) + i], u[i]);",
     "acc2_sub_prod(&yu[i], 0.0 * Sigma[(size_t)k * (nu + nx) + i], u[i]);"),
    ("accurate residual: sign of the -I coupling in the dynamics rows",
     "acc2_sub_prod(&yl[i], -1.0, xn[i]);", "acc2_sub_prod(&yl[i], 1.0, xn[i]);"),
    ("right-hand side: sign of S_0 x_init",
     "        b[i] -= s;\n", "        b[i] += s;\n"),
    ("adjoint: lambda w_x^T term of dA dropped",
     "-(wl[i] * xk[j] + (wxk ? lam[i] * wxk[j] : 0.0));", "-(wl[i] * xk[j]);"),
    ("adjoint: sign of lambda w_u^T in dB",
     "-(wl[i] * u[j] + lam[i] * wu[j]);", "-(wl[i] * u[j] - lam[i] * wu[j]);"),
    ("adjoint: S_0 term of dx_init dropped",
     "s += S[IX(i, j, nu)] * wu0[i];", "s += 0.0 * S[IX(i, j, nu)] * wu0[i];"),
    ("Cholesky: sign of the column update",
     "for (int t = 0; t < j; ++t) s -= M[IX(i, t, n)] * M[IX(j, t, n)];",
     "for (int t = 0; t < j; ++t) s += M[IX(i, t, n)] * M[IX(j, t, n)];"),
    ("|K| |z|: absolute value of z dropped",
     "for (int j = 0; j < n; ++j) s += fabs(A[IX(i, j, m)]) * fabs(x[j]);",
     "for (int j = 0; j < n; ++j) s += fabs(A[IX(i, j, m)]) * x[j];"),
]

BATTERY = [
    lambda: pins.test_riccati_matches_dense_bruteforce(3, 4, 2, True),
    lambda: pins.test_riccati_matches_dense_bruteforce(5, 3, 3, False),
    lambda: pins.test_dense_matrix_equals_structured_matvec_and_is_symmetric(3, 4, 2),
    lambda: pins.test_abs_matvec_equals_dense_abs_product(3, 4, 2),
    lambda: pins.test_accurate_residual_equals_exact_rational_arithmetic(),
    lambda: pins.test_residual_evaluation_bound_holds(),
    lambda: pins.test_inertia_of_kkt_matrix(3, 4, 2),
    lambda: pins.test_scalar_single_stage_closed_form(),
    lambda: pins.test_scalar_riccati_converges_to_dare_root(),
    lambda: pins.test_primal_solution_minimises_rollout_cost(4, 3, 2),
    lambda: pins.test_primal_solution_minimises_rollout_cost(7, 2, 3),
    lambda: pins.test_cost_to_go_spd_and_linearity(),
    lambda: pins.test_adjoint_matches_central_finite_differences(),
]


def _compile(source, folder):
    os.makedirs(folder, exist_ok=True)
    src = os.path.join(folder, "oracle.c")
    with open(src, "w") as f:
        f.write(source)
    lib = os.path.join(folder, "liboracle.so")
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-I", SRC_DIR, src,
                    "-o", lib, "-lm"], check=True)
    return lib


def _failures(monkeypatch, lib):
    """Pins of the battery that fail against the library at `lib`."""
    monkeypatch.setattr(oracle, "_lib", None)
    monkeypatch.setattr(oracle._build, "build", lambda force=False: lib)
    failed = []
    for k, pin in enumerate(BATTERY):
        try:
            pin()
        except Exception:   # an assertion, or an error the wrong numbers lead to
            failed.append(k)
    monkeypatch.setattr(oracle, "_lib", None)
    return failed


def test_unmodified_oracle_passes_the_battery(monkeypatch, tmp_path):
    source = open(os.path.join(SRC_DIR, "oracle.c")).read()
    lib = _compile(source, str(tmp_path / "original"))
    assert _failures(monkeypatch, lib) == []


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_every_planted_mistake_fails_a_pin(monkeypatch, tmp_path, name, old, new):
    source = open(os.path.join(SRC_DIR, "oracle.c")).read()
    assert source.count(old) == 1, name
    lib = _compile(source.replace(old, new), str(tmp_path / "mutant"))
    assert _failures(monkeypatch, lib), name


# The Newton-system oracle (numpy): each mutant is its source with one planted
# error, executed as a module of its own and put in place of oracle.newton for
# the pins of tests/test_newton_oracle.py.
NEWTON_MUTANTS = [
    ("multiplier estimate: sign of the penalty term",
     "yhat = y + sig * (w - proj)", "yhat = y - sig * (w - proj)"),
    ("active set: Sigma y instead of Sigma^-1 y",
     "zz = w + y / sig", "zz = w + y * sig"),
    ("gradient: sign of the proximal centre in q~",
     "gx * (xk - _vec(alm.xbar, k, nx))", "gx * (xk + _vec(alm.xbar, k, nx))"),
    ("gradient: S^T u dropped from q~",
     "qk = qk + Sk.T @ uk", "qk = qk + 0.0 * (Sk.T @ uk)"),
    ("Hessian: D^T Sigma^J C dropped from S~",
     "St[k] = Sk + Dk.T @ (sJ[:, None] * Ck)", "St[k] = Sk + 0.0 * (Dk.T @ (sJ[:, None] * Ck))"),
    ("Hessian: Gamma_x^-1 dropped from Q~",
     "Qt[k] = Qk + Ck.T @ (sJ[:, None] * Ck) + np.diag(gx)", "Qt[k] = Qk + Ck.T @ (sJ[:, None] * Ck)"),
    ("dynamics residual: sign of x^{k+1}",
     "+ _vec(f, k, nx) - xn", "+ _vec(f, k, nx) + xn"),
    ("stationarity: A^T lambda dropped",
     "v = v + _blk(inst.A, k, nx, nx).T @ lam[k]", "v = v + 0.0 * (_blk(inst.A, k, nx, nx).T @ lam[k])"),
]

NEWTON_BATTERY = [
    lambda: npins.test_gradient_is_the_derivative_of_the_al_value((6, 3, 2, 4)),
    lambda: npins.test_hessian_is_the_derivative_of_the_gradient((6, 3, 2, 4)),
    lambda: npins.test_without_constraints_the_newton_step_solves_the_proximal_lq_problem(),
    lambda: npins.test_newton_step_is_stationary_when_the_active_set_is_fixed((5, 3, 2, 4)),
    lambda: npins.test_active_set_and_multiplier_estimate_by_hand(),
]


def _newton_failures(monkeypatch, source):
    mod = types.ModuleType("newton_under_test")
    exec(compile(source, "newton_under_test.py", "exec"), mod.__dict__)
    monkeypatch.setattr(npins, "newton", mod)
    failed = []
    for k, pin in enumerate(NEWTON_BATTERY):
        try:
            pin()
        except Exception:
            failed.append(k)
    return failed


def _newton_source():
    return open(os.path.join(SRC_DIR, "newton.py")).read()


def test_unmodified_newton_oracle_passes_the_battery(monkeypatch):
    assert _newton_failures(monkeypatch, _newton_source()) == []


@pytest.mark.parametrize("name,old,new", NEWTON_MUTANTS, ids=[m[0] for m in NEWTON_MUTANTS])
def test_every_planted_newton_mistake_fails_a_pin(monkeypatch, name, old, new):
    source = _newton_source()
    assert source.count(old) == 1, name
    assert _newton_failures(monkeypatch, source.replace(old, new)), name
