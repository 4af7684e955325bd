"""ctypes front-end of the plain FP64 CPU oracle (``oracle.c``).

TEST INFRASTRUCTURE ONLY: only the test-suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library (neither imports the other).

Every function takes an instance object with attributes ``N, nx, nu, Q, R, S,
A, B, Sigma`` in the flat layout documented in ``oracle.c`` (duck-typed, so this
package does not import the library or the input generator).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None
_D = ctypes.POINTER(ctypes.c_double)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        i, d, sz = ctypes.c_int, _D, ctypes.c_size_t
        L.oracle_build_rhs.argtypes = [i, i, i, d, d, d, d, d, d, d]
        L.oracle_build_rhs.restype = None
        L.oracle_kkt_matvec.argtypes = [i, i, i, d, d, d, d, d, d, d, d]
        L.oracle_kkt_matvec.restype = None
        L.oracle_kkt_abs_matvec.argtypes = [i, i, i, d, d, d, d, d, d, d, d]
        L.oracle_kkt_abs_matvec.restype = None
        L.oracle_kkt_residual.argtypes = [i, i, i, d, d, d, d, d, d, d, d, d]
        L.oracle_kkt_residual.restype = ctypes.c_double
        L.oracle_kkt_residual_fp64.argtypes = [i, i, i, d, d, d, d, d, d, d, d, d]
        L.oracle_kkt_residual_fp64.restype = ctypes.c_double
        L.oracle_kkt_dense.argtypes = [i, i, i, d, d, d, d, d, d, d]
        L.oracle_kkt_dense.restype = i
        L.oracle_dense_solve.argtypes = [i, d, d, d]
        L.oracle_dense_solve.restype = i
        L.oracle_riccati_solve.argtypes = [i, i, i, d, d, d, d, d, d, i, d, sz, d, sz, d]
        L.oracle_riccati_solve.restype = i
        L.oracle_adjoint.argtypes = [i, i, i, d, d, d, d, d, d, d, d, d, d] + [d] * 10
        L.oracle_adjoint.restype = i
        _lib = L
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _f(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _data(inst):
    return (int(inst.N), int(inst.nx), int(inst.nu), _f(inst.Q), _f(inst.R), _f(inst.S),
            _f(inst.A), _f(inst.B), _f(inst.Sigma))


def kkt_size(inst) -> int:
    return int(inst.N) * (int(inst.nu) + 2 * int(inst.nx))


def build_rhs(inst, q, r, c, x0) -> np.ndarray:
    """b = -(r~, q, f~) of eq. opt-cond-ocp-eq for one (q, r, c, x_init)."""
    N, nx, nu, Q, R, S, A, B, Sg = _data(inst)
    b = np.zeros(kkt_size(inst))
    q, r, c, x0 = _f(q), _f(r), _f(c), _f(x0)
    lib().oracle_build_rhs(N, nx, nu, _p(S), _p(A), _p(q), _p(r), _p(c), _p(x0), _p(b))
    return b


def kkt_matvec(inst, z) -> np.ndarray:
    N, nx, nu, Q, R, S, A, B, Sg = _data(inst)
    z = _f(z)
    y = np.zeros(kkt_size(inst))
    lib().oracle_kkt_matvec(N, nx, nu, _p(Q), _p(R), _p(S), _p(A), _p(B), _p(Sg), _p(z), _p(y))
    return y


def kkt_abs_matvec(inst, z) -> np.ndarray:
    """|K| |z| (absolute values of every coefficient and entry)."""
    N, nx, nu, Q, R, S, A, B, Sg = _data(inst)
    z = _f(z)
    y = np.zeros(kkt_size(inst))
    lib().oracle_kkt_abs_matvec(N, nx, nu, _p(Q), _p(R), _p(S), _p(A), _p(B), _p(Sg), _p(z), _p(y))
    return y


def residual_eval_bound(inst, z, b) -> float:
    """Bound on the error of any float64 evaluation of ||b - K z|| / ||b||:
    gamma_m || |b| + |K| |z| ||_2 / ||b||_2, the componentwise bound of a float64
    sum of products (Higham Sec. 3.1) with m the most roundings on one term's
    path.  A row has at most 2 nx + nu + 1 products and b: 2 nx + nu + 2 summands,
    and the diagonal term carries one rounding more, either forming Q_ii + Sigma_i
    (R_ii + Sigma_i) first or adding Sigma_i z_i as a summand of its own, so
    m = 2 nx + nu + 3."""
    u = 2.0 ** -53
    m = 2 * inst.nx + inst.nu + 3
    gamma = m * u / (1.0 - m * u)
    b = _f(b)
    return float(gamma * np.linalg.norm(np.abs(b) + kkt_abs_matvec(inst, z)) / np.linalg.norm(b))


def kkt_residual(inst, z, b) -> float:
    """Relative KKT residual ||b - K z||_2 / ||b||_2 of the data as given, every
    row accumulated by a compensated dot product (Ogita-Rump-Oishi Dot2) and
    rounded once: accurate to about 1e-16 relative plus u^2-size terms, so it
    measures the residual itself, not the rounding of a float64 evaluation."""
    N, nx, nu, Q, R, S, A, B, Sg = _data(inst)
    z, b = _f(z), _f(b)
    return float(lib().oracle_kkt_residual(N, nx, nu, _p(Q), _p(R), _p(S), _p(A), _p(B), _p(Sg),
                                           _p(z), _p(b), None))


def kkt_residual_fp64(inst, z, b) -> float:
    """The same residual evaluated in plain float64 (rounded products and sums,
    Sigma added to the diagonals first): one float64 evaluation, within
    residual_eval_bound of the exact value."""
    N, nx, nu, Q, R, S, A, B, Sg = _data(inst)
    z, b = _f(z), _f(b)
    return float(lib().oracle_kkt_residual_fp64(N, nx, nu, _p(Q), _p(R), _p(S), _p(A), _p(B), _p(Sg),
                                                _p(z), _p(b), None))


def kkt_dense(inst) -> np.ndarray:
    N, nx, nu, Q, R, S, A, B, Sg = _data(inst)
    n = kkt_size(inst)
    K = np.zeros((n, n))
    lib().oracle_kkt_dense(N, nx, nu, _p(Q), _p(R), _p(S), _p(A), _p(B), _p(Sg), _p(K))
    return K


def dense_solve(K, b) -> np.ndarray:
    K, b = _f(K), _f(b)
    x = np.zeros(len(b))
    st = lib().oracle_dense_solve(len(b), _p(K), _p(b), _p(x))
    if st:
        raise np.linalg.LinAlgError("singular KKT matrix")
    return x


def riccati_solve(inst, b, return_P: bool = False):
    """z = K^{-1} b by the textbook Riccati recursion; b may be (n,) or (nrhs, n)."""
    N, nx, nu, Q, R, S, A, B, Sg = _data(inst)
    b = _f(b)
    single = b.ndim == 1
    bb = b.reshape(1, -1) if single else b
    n = kkt_size(inst)
    assert bb.shape[1] == n
    z = np.zeros_like(bb)
    P = np.zeros(N * nx * nx) if return_P else None
    st = lib().oracle_riccati_solve(N, nx, nu, _p(Q), _p(R), _p(S), _p(A), _p(B), _p(Sg),
                                    bb.shape[0], _p(bb), n, _p(z), n, _p(P))
    if st:
        raise np.linalg.LinAlgError("stage %d: R + B^T P B not positive definite" % (st - 1))
    z = z[0] if single else z
    if return_P:
        return z, P.reshape(N, nx, nx).transpose(0, 2, 1).copy()
    return z


def adjoint(inst, x0, z, g):
    """Gradients of L(z(theta)) for dL/dz = g; returns a dict of arrays in the data layout."""
    N, nx, nu, Q, R, S, A, B, Sg = _data(inst)
    n = kkt_size(inst)
    out = dict(w=np.zeros(n), dQ=np.zeros((N + 1) * nx * nx), dq=np.zeros((N + 1) * nx),
               dR=np.zeros(N * nu * nu), dr=np.zeros(N * nu), dS=np.zeros(N * nu * nx),
               dA=np.zeros(N * nx * nx), dB=np.zeros(N * nx * nu), dc=np.zeros(N * nx),
               dx0=np.zeros(nx), dSigma=np.zeros((N + 1) * (nu + nx)))
    x0, z, g = _f(x0), _f(z), _f(g)
    st = lib().oracle_adjoint(N, nx, nu, _p(Q), _p(R), _p(S), _p(A), _p(B), _p(Sg), _p(x0),
                              _p(z), _p(g), _p(out["w"]), _p(out["dQ"]), _p(out["dq"]), _p(out["dR"]),
                              _p(out["dr"]), _p(out["dS"]), _p(out["dA"]), _p(out["dB"]),
                              _p(out["dc"]), _p(out["dx0"]), _p(out["dSigma"]))
    if st:
        raise np.linalg.LinAlgError("adjoint solve failed")
    return out
