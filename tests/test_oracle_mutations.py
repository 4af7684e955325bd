"""The oracle's pins catch plausible mistakes: each mutant below is the oracle's
C source with one planted error (a dropped term, a wrong sign, a transposed
operand), compiled to its own library in a temporary folder; the pin battery
of tests/test_oracle_pins.py, run against that library, must fail for every
mutant, and pass for the unmodified source compiled the same way.  Every
mutation stays inside the arrays it touches (signs, dropped terms, transposes
of square blocks), so a mutant computes wrong numbers but never faults.
"""
import os
import subprocess

import pytest

import oracle
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
