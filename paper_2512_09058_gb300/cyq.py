"""Thin ctypes binding of the cyq C ABI (include/cyq.h).

Argument marshalling only: every step of factor, solve, refinement and adjoint
runs in the CUDA library ``libcyq.so``.  PyTorch provides device memory and the
current CUDA stream.  There is no CPU fallback: if the compiled library is
missing, loading fails with an error.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcyq.so")

CYQ_FP64 = 0
CYQ_FP32_REFINE = 1
CYQ_FP64_IR32 = 2
STATUS = {0: "ok", 1: "invalid argument", 2: "not positive definite", 3: "not converged", 4: "CUDA error",
          5: "timeout", 6: "no factor", 7: "unimplemented", 8: "no device", 9: "update rank above the workspace"}

# every entry point declared in include/cyq.h
EXPORTS = ["cyq_create", "cyq_destroy", "cyq_factor", "cyq_solve", "cyq_build_rhs", "cyq_residual",
           "cyq_solve_adjoint", "cyq_get_instance_status", "cyq_get_stats", "cyq_kkt_size", "cyq_workspace_bytes",
           "cyq_get_segments", "cyq_last_launch_count", "cyq_status_string", "cyq_last_error",
           "cyq_factor_solve_noalloc", "cyq_autotune", "cyq_get_launch_shapes", "cyq_tune_segments",
           "cyq_set_launch_shapes", "cyq_get_stage_factor", "cyq_assemble_newton", "cyq_set_pcr_tail",
           "cyq_get_pcr_tail", "cyq_pivot_eval", "cyq_set_factor_path", "cyq_get_factor_path", "cyq_apply_factor", "cyq_update_factor",
           "cyq_get_escalation_segments", "cyq_get_sweep_path", "cyq_set_sweep_path", "cyq_residual_compensated",
           "cyq_segment_stages"]


class CyqError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__("cyq error %d (%s)%s" % (code, STATUS.get(code, "?"), (": " + what) if what else ""))


class cyq_desc(ctypes.Structure):
    _fields_ = [("batch", ctypes.c_int32), ("N", ctypes.POINTER(ctypes.c_int32)),
                ("nx", ctypes.POINTER(ctypes.c_int32)), ("nu", ctypes.POINTER(ctypes.c_int32)),
                ("precision", ctypes.c_int32), ("P", ctypes.c_int32),
                ("P_per_instance", ctypes.POINTER(ctypes.c_int32)), ("max_nrhs", ctypes.c_int32),
                ("it_max", ctypes.c_int32), ("tol", ctypes.c_double), ("device", ctypes.c_int32),
                ("esc_max", ctypes.c_int32), ("recompute_factors", ctypes.c_int32),
                ("recompute_chunks", ctypes.c_int32), ("early_escalation", ctypes.c_int32),
                ("certify", ctypes.c_int32)]


class cyq_stats(ctypes.Structure):
    _fields_ = [("refine_steps", ctypes.c_int32), ("max_rel_residual", ctypes.c_double),
                ("max_certified", ctypes.c_double), ("P_min", ctypes.c_int32), ("P_max", ctypes.c_int32),
                ("work_items", ctypes.c_int64)]


class cyq_newton_in(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("Q", "R", "S", "A", "B", "q", "r", "c", "x_init", "u", "x")] + \
               [("ny", ctypes.POINTER(ctypes.c_int32))] + \
               [(n, ctypes.c_void_p) for n in ("C", "D", "bl", "bu", "y", "sigma", "gx", "gu", "xbar", "ubar")]


class cyq_newton_out(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("Q", "R", "S", "q", "r", "c", "active", "yhat")]


_lib = None


def load(path: str = LIB_PATH):
    """Load libcyq.so (built by ``paper_2512_09058_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libcyq.so not found at %s: build it with paper_2512_09058_gb300/build.py "
                           "(there is no CPU fallback)" % path)
    L = ctypes.CDLL(path)
    vp, i32, i64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    L.cyq_create.argtypes = [ctypes.POINTER(cyq_desc), ctypes.POINTER(vp)]
    L.cyq_destroy.argtypes = [vp]
    L.cyq_destroy.restype = None
    L.cyq_factor.argtypes = [vp] + [vp] * 6 + [vp]
    L.cyq_solve.argtypes = [vp, vp, vp, i32, vp]
    L.cyq_build_rhs.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    L.cyq_residual.argtypes = [vp, vp, vp, vp, vp, vp]
    L.cyq_solve_adjoint.argtypes = [vp] + [vp] * 14 + [vp]
    L.cyq_get_instance_status.argtypes = [vp, ctypes.POINTER(i32), vp]
    L.cyq_get_stats.argtypes = [vp, ctypes.POINTER(cyq_stats), vp]
    L.cyq_kkt_size.argtypes = [vp]
    L.cyq_kkt_size.restype = i64
    L.cyq_workspace_bytes.argtypes = [vp]
    L.cyq_workspace_bytes.restype = i64
    L.cyq_get_segments.argtypes = [vp, ctypes.POINTER(i32)]
    L.cyq_last_launch_count.argtypes = [vp]
    L.cyq_last_launch_count.restype = i64
    L.cyq_status_string.argtypes = [ctypes.c_int]
    L.cyq_status_string.restype = ctypes.c_char_p
    L.cyq_last_error.argtypes = []
    L.cyq_last_error.restype = ctypes.c_char_p
    pi32 = ctypes.POINTER(i32)
    L.cyq_autotune.argtypes = [vp] + [vp] * 6 + [vp, vp, i32, i32, vp]
    L.cyq_get_launch_shapes.argtypes = [vp, pi32, pi32, pi32, i32]
    L.cyq_tune_segments.argtypes = [ctypes.POINTER(cyq_desc)] + [vp] * 6 + [vp, vp, i32, i32, vp, pi32]
    L.cyq_set_launch_shapes.argtypes = [vp, pi32, pi32, i32]
    L.cyq_get_stage_factor.argtypes = [vp, i32, i32, ctypes.POINTER(d)]
    L.cyq_assemble_newton.argtypes = [vp, ctypes.POINTER(cyq_newton_in), ctypes.POINTER(cyq_newton_out), vp]
    L.cyq_set_pcr_tail.argtypes = [vp, i32]
    L.cyq_get_pcr_tail.argtypes = [vp, pi32]
    L.cyq_pivot_eval.argtypes = [vp] * 6 + [i64, vp]
    L.cyq_set_factor_path.argtypes = [vp, i32]
    L.cyq_apply_factor.argtypes = [vp, vp, vp, i32, vp]
    L.cyq_update_factor.argtypes = [vp, vp, vp, vp, vp, vp, i32, vp]
    L.cyq_get_factor_path.argtypes = [vp, pi32, ctypes.POINTER(i64)]
    L.cyq_get_escalation_segments.argtypes = [vp, pi32]
    L.cyq_get_sweep_path.argtypes = [vp, pi32, ctypes.POINTER(i64)]
    L.cyq_set_sweep_path.argtypes = [vp, i32]
    L.cyq_residual_compensated.argtypes = [vp] * 6
    L.cyq_segment_stages.argtypes = [i32, i32, i32, pi32, pi32]
    for name in ["cyq_create", "cyq_factor", "cyq_solve", "cyq_build_rhs", "cyq_residual", "cyq_solve_adjoint",
                 "cyq_get_instance_status", "cyq_get_stats", "cyq_get_segments", "cyq_autotune",
                 "cyq_get_escalation_segments", "cyq_get_sweep_path", "cyq_set_sweep_path",
                 "cyq_residual_compensated", "cyq_segment_stages",
                 "cyq_get_launch_shapes", "cyq_tune_segments", "cyq_set_launch_shapes",
                 "cyq_get_stage_factor", "cyq_pivot_eval", "cyq_set_factor_path", "cyq_get_factor_path",
                 "cyq_apply_factor", "cyq_update_factor"]:
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(code: int):
    if code != 0:
        what = _lib.cyq_last_error().decode() if code == 4 else ""
        raise CyqError(code, what)


def _ptr(t) -> Optional[int]:
    """Device pointer of a torch CUDA tensor (float64, contiguous) or None."""
    if t is None:
        return None
    import torch
    assert t.is_cuda and t.is_contiguous(), "expected a contiguous CUDA tensor"
    return t.data_ptr()


def _stream(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


class _Desc:
    """A cyq_desc with the host arrays it points to kept alive."""

    def __init__(self, N, nx, nu, precision="fp64", P=0, P_per_instance=None, max_nrhs=1, it_max=-1,
                 tol=1e-10, device=-1, esc_max=-1, recompute_chunks=0, early_escalation=False, certify=False):
        i32p = ctypes.POINTER(ctypes.c_int32)
        self.N = np.ascontiguousarray(N, dtype=np.int32)
        self.nx = np.ascontiguousarray(nx, dtype=np.int32)
        self.nu = np.ascontiguousarray(nu, dtype=np.int32)
        self.precision = {"fp64": CYQ_FP64, "fp32_refine": CYQ_FP32_REFINE, "fp64_ir32": CYQ_FP64_IR32}[precision]
        pp = None
        if P_per_instance is not None:
            self.P = np.ascontiguousarray(P_per_instance, dtype=np.int32)
            pp = self.P.ctypes.data_as(i32p)
        self.desc = cyq_desc(len(self.N), self.N.ctypes.data_as(i32p), self.nx.ctypes.data_as(i32p),
                             self.nu.ctypes.data_as(i32p), self.precision, P, pp, max_nrhs, it_max, tol, device,
                             esc_max, 1 if recompute_chunks > 0 else 0, int(recompute_chunks),
                             1 if early_escalation else 0, 1 if certify else 0)


def tune_segments(N, nx, nu, data, b, nrhs: int = 1, reps: int = 2, stream=None, **desc_kw) -> np.ndarray:
    """Segment counts per instance chosen by timing (cyq_tune_segments); pass the
    result as ``P_per_instance`` to :class:`Solver`.  ``data`` holds the device
    arrays Q, R, S, A, B, Sigma; ``b`` the nrhs right-hand sides."""
    import torch
    L = load()
    d = _Desc(N, nx, nu, max_nrhs=nrhs, **desc_kw)
    z = torch.empty_like(b)
    out = np.zeros(len(d.N), np.int32)
    _check(L.cyq_tune_segments(ctypes.byref(d.desc), _ptr(data["Q"]), _ptr(data["R"]), _ptr(data.get("S")),
                               _ptr(data["A"]), _ptr(data["B"]), _ptr(data.get("Sigma")), _ptr(b), _ptr(z), nrhs,
                               reps, _stream(stream), out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
    return out


def segment_stages(N: int, P: int, c: int) -> np.ndarray:
    """Stages of segment c (of P) of a horizon of N stages, in the order the
    factorization processes them (cyq_segment_stages; host only)."""
    L = load()
    n = ctypes.c_int32(0)
    _check(L.cyq_segment_stages(int(N), int(P), int(c), None, ctypes.byref(n)))
    out = np.zeros(n.value, np.int32)
    _check(L.cyq_segment_stages(int(N), int(P), int(c), out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                ctypes.byref(n)))
    return out


class Solver:
    """A planned batch of OCP KKT systems (one cyq handle)."""

    def __init__(self, N: Sequence[int], nx: Sequence[int], nu: Sequence[int], precision: str = "fp64",
                 P: int = 0, P_per_instance: Optional[Sequence[int]] = None, max_nrhs: int = 1,
                 it_max: int = -1, tol: float = 1e-10, device: int = -1, esc_max: int = -1,
                 recompute_chunks: int = 0, early_escalation: bool = False, certify: bool = False):
        """recompute_chunks > 0: keep the stage factors of one chunk of instances at a
        time (the batch in that many chunks) and factor each chunk again in every solve
        and adjoint (cyq_desc.recompute_factors).  early_escalation: float32 mode factors
        the slowly converging instances in float64 after two corrections, on a second
        stream (cyq_desc.early_escalation).
        certify: stop only where the worst-case float64 evaluation bound allows (cyq_desc.certify)."""
        L = load()
        d = _Desc(N, nx, nu, precision, P, P_per_instance, max_nrhs, it_max, tol, device, esc_max,
                  recompute_chunks, early_escalation, certify)
        self._desc = d
        self.N, self.nx, self.nu = d.N, d.nx, d.nu
        self.batch = len(self.N)
        self.precision = d.precision
        self.max_nrhs = max_nrhs
        desc = d.desc
        h = ctypes.c_void_p()
        _check(L.cyq_create(ctypes.byref(desc), ctypes.byref(h)))
        self._h = h
        self.kkt_size = int(L.cyq_kkt_size(h))
        self.workspace_bytes = int(L.cyq_workspace_bytes(h))
        self._data = None
        self.factor_version = 0

    def close(self):
        if getattr(self, "_h", None):
            _lib.cyq_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def segments(self) -> np.ndarray:
        out = np.zeros(self.batch, np.int32)
        _check(_lib.cyq_get_segments(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
        return out

    def launch_count(self) -> int:
        return int(_lib.cyq_last_launch_count(self._h))

    def autotune(self, Q, R, S, A, B, Sigma, b, nrhs: int = 1, reps: int = 3, stream=None):
        """Pick launch shapes by timing (cyq_autotune); leaves the solver factored."""
        import torch
        z = torch.empty_like(b)
        self._data = (Q, R, S, A, B, Sigma)
        _check(_lib.cyq_autotune(self._h, _ptr(Q), _ptr(R), _ptr(S), _ptr(A), _ptr(B), _ptr(Sigma), _ptr(b),
                                 _ptr(z), nrhs, reps, _stream(stream)))
        self.factor_version += 1

    def stage_factor(self, instance: int, stage: int) -> np.ndarray:
        """Stored (nu+nx)^2 factor of one stage as a float64 matrix (lower: the Cholesky
        factor of H^_s; strict upper: the stored triangular inverses, transposed)."""
        n = int(self.nx[instance] + self.nu[instance])
        out = np.zeros(n * n)
        _check(_lib.cyq_get_stage_factor(self._h, instance, stage,
                                         out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out.reshape(n, n).T.copy()

    def launch_shapes(self, nrhs: int = 1) -> dict:
        i32p = ctypes.POINTER(ctypes.c_int32)
        n = ctypes.c_int32(0)
        _check(_lib.cyq_get_launch_shapes(self._h, ctypes.byref(n), None, None, nrhs))
        f = np.zeros(n.value, np.int32)
        w = np.zeros(n.value, np.int32)
        _check(_lib.cyq_get_launch_shapes(self._h, ctypes.byref(n), f.ctypes.data_as(i32p), w.ctypes.data_as(i32p),
                                          nrhs))
        return dict(factor=f.tolist(), sweep=w.tolist())

    def set_launch_shapes(self, factor=None, sweep=None, nrhs: int = 1):
        """Threads per work item per size class (0 = default); None leaves a kind unchanged."""
        i32p = ctypes.POINTER(ctypes.c_int32)
        f = None if factor is None else np.ascontiguousarray(factor, dtype=np.int32)
        w = None if sweep is None else np.ascontiguousarray(sweep, dtype=np.int32)
        _check(_lib.cyq_set_launch_shapes(self._h, None if f is None else f.ctypes.data_as(i32p),
                                          None if w is None else w.ctypes.data_as(i32p), nrhs))

    def factor(self, Q, R, S, A, B, Sigma=None, stream=None):
        self._data = (Q, R, S, A, B, Sigma)   # borrowed until the last solve
        _check(_lib.cyq_factor(self._h, _ptr(Q), _ptr(R), _ptr(S), _ptr(A), _ptr(B), _ptr(Sigma),
                               _stream(stream)))
        self.factor_version += 1

    def solve(self, b, z=None, nrhs: int = 1, stream=None):
        import torch
        if z is None:
            z = torch.empty_like(b)
        _check(_lib.cyq_solve(self._h, _ptr(b), _ptr(z), nrhs, _stream(stream)))
        return z

    def update_factor(self, Q, R, S, w, delta, m_max: int, stream=None):
        """Update the stored factor to that of the stage matrices H_s + sum delta w w^T
        (see cyq_update_factor); Q, R, S are the updated data for later residuals."""
        _check(_lib.cyq_update_factor(self._h, _ptr(Q), _ptr(R), _ptr(S), _ptr(w), _ptr(delta), int(m_max),
                                      _stream(stream)))

    def apply_factor(self, r, dz=None, nrhs: int = 1, stream=None):
        """dz = K~^{-1} r with the stored factor (one substitution, no refinement)."""
        import torch
        if dz is None:
            dz = torch.empty_like(r)
        _check(_lib.cyq_apply_factor(self._h, _ptr(r), _ptr(dz), int(nrhs), _stream(stream)))
        return dz

    def build_rhs(self, q, r, c, x0, b=None, stream=None):
        import torch
        if b is None:
            b = torch.empty(self.kkt_size, dtype=torch.float64, device=q.device)
        _check(_lib.cyq_build_rhs(self._h, _ptr(q), _ptr(r), _ptr(c), _ptr(x0), _ptr(b), _stream(stream)))
        return b

    def set_pcr_tail(self, levels: int):
        """Solve the last `levels` levels of the coupling system by parallel cyclic
        reduction (0: plain cyclic reduction); factor again afterwards."""
        _check(_lib.cyq_set_pcr_tail(self._h, int(levels)))

    def set_factor_path(self, one_warp_per_item: bool):
        """Float32 factor: one persistent launch, a team of 32, 64 or 128 threads
        per item (True, the default), or the per-size-class kernels (False);
        factor again afterwards."""
        _check(_lib.cyq_set_factor_path(self._h, 1 if one_warp_per_item else 0))

    def factor_path(self) -> dict:
        on, n = ctypes.c_int32(0), ctypes.c_int64(0)
        _check(_lib.cyq_get_factor_path(self._h, ctypes.byref(on), ctypes.byref(n)))
        p, m = ctypes.c_int32(0), ctypes.c_int64(0)
        _check(_lib.cyq_get_sweep_path(self._h, ctypes.byref(p), ctypes.byref(m)))
        return {"one_warp_per_item": bool(on.value), "warp_items": int(n.value), "sweep_persistent": bool(p.value),
                "sweep_items": int(m.value)}

    def set_sweep_path(self, persistent: bool):
        """Float32 sweeps as one persistent launch (True) or per size class (False)."""
        _check(_lib.cyq_set_sweep_path(self._h, 1 if persistent else 0))

    def escalation_segments(self) -> np.ndarray:
        """Segments per instance of the float64 escalation plan (0: the handle's own plan)."""
        out = np.zeros(self.batch, np.int32)
        _check(_lib.cyq_get_escalation_segments(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
        return out

    def pcr_tail(self) -> int:
        v = ctypes.c_int32(0)
        _check(_lib.cyq_get_pcr_tail(self._h, ctypes.byref(v)))
        return v.value

    def assemble_newton(self, data, q, r, c, x_init, u, x, alm, out=None, stream=None):
        """Newton system of the augmented Lagrangian inner problem at (u, x):
        returns dict(Q, R, S, q, r, c, active, yhat) of device tensors in the data
        layout (see cyq_assemble_newton).  `data`: dict of device Q, R, S, A, B;
        `alm`: dict of device C, D, bl, bu, y, sigma and optional gx, gu, xbar,
        ubar, plus `ny` (host int32 array [batch])."""
        import torch
        dev = q.device
        ny = np.ascontiguousarray(alm["ny"], dtype=np.int32)
        N, nx, nu = self.N.astype(np.int64), self.nx.astype(np.int64), self.nu.astype(np.int64)
        if out is None:
            f64 = lambda n: torch.empty(int(n), dtype=torch.float64, device=dev)
            out = dict(Q=f64(((N + 1) * nx * nx).sum()), R=f64((N * nu * nu).sum()), S=f64((N * nu * nx).sum()),
                       q=f64(((N + 1) * nx).sum()), r=f64((N * nu).sum()), c=f64((N * nx).sum()),
                       active=torch.empty(int(((N + 1) * ny).sum()), dtype=torch.int32, device=dev),
                       yhat=f64(((N + 1) * ny).sum()))
        g = lambda k: _ptr(alm.get(k))
        a = cyq_newton_in(Q=_ptr(data["Q"]), R=_ptr(data["R"]), S=_ptr(data.get("S")), A=_ptr(data["A"]),
                          B=_ptr(data["B"]), q=_ptr(q), r=_ptr(r), c=_ptr(c), x_init=_ptr(x_init), u=_ptr(u),
                          x=_ptr(x), ny=ny.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), C=g("C"), D=g("D"),
                          bl=g("bl"), bu=g("bu"), y=g("y"), sigma=g("sigma"), gx=g("gx"), gu=g("gu"),
                          xbar=g("xbar"), ubar=g("ubar"))
        o = cyq_newton_out(**{k: _ptr(out.get(k)) for k in ("Q", "R", "S", "q", "r", "c", "active", "yhat")})
        _check(_lib.cyq_assemble_newton(self._h, ctypes.byref(a), ctypes.byref(o), _stream(stream)))
        return out

    def residual(self, b, z, res=None, stream=None, compensated=False):
        """Per-instance ||b - K z|| / ||b|| (res: optional output of b - K z); compensated
        rows evaluate it as if in twice the float64 precision (cyq_residual_compensated)."""
        import torch
        rel = torch.empty(self.batch, dtype=torch.float64, device=b.device)
        fn = _lib.cyq_residual_compensated if compensated else _lib.cyq_residual
        _check(fn(self._h, _ptr(b), _ptr(z), _ptr(res), _ptr(rel), _stream(stream)))
        return rel

    def solve_adjoint(self, x0, z, dL_dz, stream=None, want=("w", "dQ", "dq", "dR", "dr", "dS", "dA", "dB", "dc",
                                                              "dx0", "dSigma")):
        import torch
        dev = z.device
        N, nx, nu = self.N.astype(np.int64), self.nx.astype(np.int64), self.nu.astype(np.int64)
        sizes = dict(w=self.kkt_size, dQ=int(((N + 1) * nx * nx).sum()), dq=int(((N + 1) * nx).sum()),
                     dR=int((N * nu * nu).sum()), dr=int((N * nu).sum()), dS=int((N * nu * nx).sum()),
                     dA=int((N * nx * nx).sum()), dB=int((N * nx * nu).sum()), dc=int((N * nx).sum()),
                     dx0=int(nx.sum()), dSigma=int(((N + 1) * (nu + nx)).sum()))
        out = {k: torch.empty(sizes[k], dtype=torch.float64, device=dev) for k in want}
        g = lambda k: _ptr(out.get(k))
        _check(_lib.cyq_solve_adjoint(self._h, _ptr(x0), _ptr(z), _ptr(dL_dz), g("w"), g("dQ"), g("dq"), g("dR"),
                                      g("dr"), g("dS"), g("dA"), g("dB"), g("dc"), g("dx0"), g("dSigma"),
                                      _stream(stream)))
        return out

    def instance_status(self, stream=None) -> np.ndarray:
        out = np.zeros(self.batch, np.int32)
        _lib.cyq_get_instance_status(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _stream(stream))
        return out

    def stats(self, stream=None) -> dict:
        s = cyq_stats()
        _check(_lib.cyq_get_stats(self._h, ctypes.byref(s), _stream(stream)))
        return dict(refine_steps=s.refine_steps, max_rel_residual=s.max_rel_residual,
                    max_certified=s.max_certified, P_min=s.P_min,
                    P_max=s.P_max, work_items=s.work_items)


def to_device(batch, device="cuda"):
    """Copy a host Batch (float64 numpy arrays) to torch CUDA tensors (data + rhs list)."""
    import torch
    t = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(device)
    data = dict(Q=t(batch.Q), R=t(batch.R), S=t(batch.S), A=t(batch.A), B=t(batch.B), Sigma=t(batch.Sigma))
    rhs = [tuple(t(x) for x in r) for r in batch.rhs]
    return data, rhs
