"""The allocation-free entry point cyq_factor_solve_noalloc, called through the
C ABI, must give the same solution as the regular entry points
(cyq_create / cyq_factor / cyq_solve with one segment, float64), on two calls
in a row with different problems (its fixed workspace keeps the previous
call's contents, which must not leak into the next result).

Callers that cannot allocate device memory while they run (real-time loops
that allocate only at start-up, hosts whose device memory belongs to another
allocator) use that entry point.  The cases cover every team size of its
kernels (nu + nx up to 24, 48 and beyond) and problems without S and Sigma.
This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2512_09058_gb300 import inputs

pytestmark = pytest.mark.gpu


def _instance(seed, N, nx, nu, S=True, sigma=(1e-2, 1e2)):
    cfg = dict(batch=1, N=N, nx=nx, nu=nu, S=S, sigma=sigma, nrhs=1, QN_equals_Q0=False, seed=seed)
    return inputs.make_instance(cfg, 0)


def _regular(cyq, torch, inst, b):
    s = cyq.Solver([inst.N], [inst.nx], [inst.nu], precision="fp64", P=1, it_max=0)
    t = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()
    s.factor(t(inst.Q), t(inst.R), t(inst.S), t(inst.A), t(inst.B), t(inst.Sigma))
    z = s.solve(t(b))
    torch.cuda.synchronize()
    out = z.cpu().numpy()
    s.close()
    return out


def _noalloc(lib, torch, inst, b):
    t = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()
    Q, R, S, A, B, Sg, bt = t(inst.Q), t(inst.R), t(inst.S), t(inst.A), t(inst.B), t(inst.Sigma), t(b)
    z = torch.empty_like(bt)
    st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    p = lambda x: None if x is None else ctypes.c_void_p(x.data_ptr())
    code = lib.cyq_factor_solve_noalloc(inst.N, inst.nx, inst.nu, p(Q), p(R), p(S), p(A), p(B), p(Sg), p(bt),
                                        p(z), p(st), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == 0, lib.cyq_last_error()
    torch.cuda.synchronize()
    return z.cpu().numpy(), int(st.item())


def test_noalloc_matches_regular_entry_points_twice():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    from paper_2512_09058_gb300 import build, cyq
    build.build()
    lib = cyq.load()
    lib.cyq_factor_solve_noalloc.argtypes = [ctypes.c_int32] * 3 + [ctypes.c_void_p] * 10
    lib.cyq_factor_solve_noalloc.restype = ctypes.c_int
    cases = [(41, (40, 10, 4), True, (1e-2, 1e2)), (42, (17, 6, 3), True, (1e-2, 1e2)),
             (43, (16, 32, 12), True, (1e-2, 1e2)), (44, (9, 40, 16), False, None),
             (45, (12, 7, 5), False, None)]
    for seed, (N, nx, nu), S, sigma in cases:
        inst = _instance(seed, N, nx, nu, S=S, sigma=sigma)
        assert (inst.Sigma is None) == (sigma is None)
        if not S:   # S = 0: both paths get a NULL S pointer
            assert not np.any(inst.S)
            inst.S = None
        b = oracle.build_rhs(inst, *inst.rhs[0])
        z_reg = _regular(cyq, torch, inst, b)
        z_na, status = _noalloc(lib, torch, inst, b)
        assert status == 0
        assert np.linalg.norm(z_na - z_reg) <= 1e-10 * np.linalg.norm(z_reg)
        # and both agree with the oracle at the parity tolerance
        zo = oracle.riccati_solve(inst, b)
        assert np.linalg.norm(z_na - zo) <= 1e-10 * np.linalg.norm(zo)


def test_noalloc_rejects_problems_above_its_workspace():
    torch = pytest.importorskip("torch")
    from paper_2512_09058_gb300 import build, cyq
    build.build()
    lib = cyq.load()
    lib.cyq_factor_solve_noalloc.argtypes = [ctypes.c_int32] * 3 + [ctypes.c_void_p] * 10
    lib.cyq_factor_solve_noalloc.restype = ctypes.c_int
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    code = lib.cyq_factor_solve_noalloc(100000, 32, 16, p, p, None, p, p, None, p, p, None, None)
    assert code == 1
    assert b"workspace" in lib.cyq_last_error()
