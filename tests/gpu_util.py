"""Shared helpers of the GPU tests: build/load the CUDA library, run it on a
host Batch, and compare with the CPU oracle instance by instance."""
import numpy as np
import pytest

import oracle
from paper_2512_09058_gb300 import inputs


# Refinement target of the tests: the gate 1e-10 with a factor-2 margin for the
# difference between two float64 evaluations of the same residual (the
# device's and the oracle's differ by up to a few percent near the gate), so
# that the oracle's own evaluation of a refined z is itself <= 1e-10.
REFINE_TARGET = 5e-11
GATE = 1e-10


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    from paper_2512_09058_gb300 import build, cyq
    build.build()
    cyq.load()
    return torch, cyq


def split_instances(batch, flat):
    """Split a concatenated KKT vector into per-instance pieces."""
    out, off = [], 0
    for x in batch.instances:
        n = x.kkt_size
        out.append(flat[off:off + n])
        off += n
    return out


def oracle_rhs(batch, rhs_index=0):
    return np.concatenate([oracle.build_rhs(x, *x.rhs[rhs_index]) for x in batch.instances])


def gpu_solve(batch, precision="fp64", P=0, P_per_instance=None, nrhs=1, it_max=0, tol=REFINE_TARGET, b_host=None):
    """Factor + solve on the GPU through the C ABI; returns (z (nrhs, kkt), solver, device data)."""
    torch, cyq = require_gpu()
    s = cyq.Solver(batch.N, batch.nx, batch.nu, precision=precision, P=P, P_per_instance=P_per_instance,
                   max_nrhs=nrhs, it_max=it_max, tol=tol)
    data, rhs = cyq.to_device(batch)
    s.factor(data["Q"], data["R"], data["S"], data["A"], data["B"], data["Sigma"])
    if b_host is None:
        b_host = np.stack([oracle_rhs(batch, j) for j in range(nrhs)])
    b = torch.from_numpy(np.ascontiguousarray(b_host.reshape(-1))).cuda()
    z = s.solve(b, nrhs=nrhs)
    torch.cuda.synchronize()
    return z.cpu().numpy().reshape(nrhs, -1), s, data, b_host.reshape(nrhs, -1)


def rel_err(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def block_rel_err(inst, z, zo):
    """Worst blockwise relative error: the maximum over the stage blocks u^k,
    x^{k+1}, lambda^k of ||z_blk - zo_blk|| / ||zo_blk|| (blocks whose reference
    norm is below 1e-6 ||zo|| are skipped: a ratio there measures nothing).  A
    wrong small block can hide under the normwise error of a long horizon; it
    cannot hide here."""
    nu, nx = inst.nu, inst.nx
    w = nu + 2 * nx
    Z, ZO = z.reshape(inst.N, w), zo.reshape(inst.N, w)
    floor = 1e-6 * np.linalg.norm(zo)
    worst = 0.0
    for lo, hi in ((0, nu), (nu, nu + nx), (nu + nx, w)):
        e = np.linalg.norm(Z[:, lo:hi] - ZO[:, lo:hi], axis=1)
        n = np.linalg.norm(ZO[:, lo:hi], axis=1)
        keep = n > floor
        if keep.any():
            worst = max(worst, float((e[keep] / n[keep]).max()))
    return worst


def small_cfg(seed, S=True, sigma=(1e-2, 1e2)):
    return dict(batch=1, N=8, nx=3, nu=2, S=S, sigma=sigma, nrhs=1, QN_equals_Q0=False, seed=seed)


def ragged_batch(seed, dims, S=True, sigma=(1e-2, 1e2), nrhs=1):
    insts = []
    for i, (N, nx, nu) in enumerate(dims):
        cfg = dict(batch=1, N=N, nx=nx, nu=nu, S=S, sigma=sigma, nrhs=nrhs, QN_equals_Q0=False, seed=seed)
        insts.append(inputs.make_instance(cfg, i))
    return inputs.make_batch(None, instances=insts)
