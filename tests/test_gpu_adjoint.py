"""Adjoint kernel (cyq_solve_adjoint) against the oracle's dense adjoint and
against FP64 central finite differences of the GPU solve itself."""
import numpy as np
import pytest

import oracle
from paper_2512_09058_gb300 import inputs

from gpu_util import oracle_rhs, ragged_batch, rel_err, require_gpu, split_instances

pytestmark = pytest.mark.gpu


def _loss_grad(batch, z):
    g = np.zeros_like(z)
    off = 0
    for x in batch.instances:
        w = x.nu + 2 * x.nx
        Z = z[off:off + x.kkt_size].reshape(x.N, w)
        G = np.zeros_like(Z)
        G[:, :x.nu + x.nx] = 2 * Z[:, :x.nu + x.nx]
        g[off:off + x.kkt_size] = G.ravel()
        off += x.kkt_size
    return g


def _gpu_adjoint(batch, precision="fp64", P=1):
    torch, cyq = require_gpu()
    s = cyq.Solver(batch.N, batch.nx, batch.nu, precision=precision, P=P)
    data, rhs = cyq.to_device(batch)
    s.factor(data["Q"], data["R"], data["S"], data["A"], data["B"], data["Sigma"])
    q, r, c, x0 = rhs[0]
    b = s.build_rhs(q, r, c, x0)
    z = s.solve(b)
    g = torch.from_numpy(_loss_grad(batch, z.cpu().numpy())).cuda()
    out = s.solve_adjoint(x0, z, g)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}, z.cpu().numpy(), g.cpu().numpy()


@pytest.mark.parametrize("precision,P", [("fp64", 1), ("fp64", 4), ("fp32_refine", 2)])
def test_adjoint_matches_oracle(precision, P):
    batch = ragged_batch(31, [(10, 4, 2), (7, 3, 3), (16, 6, 2)], sigma=(1e-1, 1e1))
    G, z, g = _gpu_adjoint(batch, precision, P)
    offs = dict(dQ=0, dq=0, dR=0, dr=0, dS=0, dA=0, dB=0, dc=0, dx0=0, dSigma=0, w=0)
    for inst in batch.instances:
        N, nx, nu = inst.N, inst.nx, inst.nu
        sizes = dict(w=inst.kkt_size, dQ=(N + 1) * nx * nx, dq=(N + 1) * nx, dR=N * nu * nu, dr=N * nu,
                     dS=N * nu * nx, dA=N * nx * nx, dB=N * nx * nu, dc=N * nx, dx0=nx, dSigma=(N + 1) * (nu + nx))
        zi = z[offs["w"]:offs["w"] + inst.kkt_size]
        gi = g[offs["w"]:offs["w"] + inst.kkt_size]
        ref = oracle.adjoint(inst, inst.rhs[0][3], zi, gi)
        for k, n in sizes.items():
            got = G[k][offs[k]:offs[k] + n]
            assert rel_err(got, ref[k]) <= 1e-9, (k, rel_err(got, ref[k]))
            offs[k] += n


def test_adjoint_matches_finite_differences_of_gpu_solve():
    torch, cyq = require_gpu()
    batch = ragged_batch(32, [(6, 3, 2)], sigma=None)
    inst = batch.instances[0]
    G, z, g = _gpu_adjoint(batch)
    q, r, c, x0 = [a.copy() for a in inst.rhs[0]]

    def loss():
        s = cyq.Solver(batch.N, batch.nx, batch.nu, P=1, it_max=0)
        d, _ = cyq.to_device(batch)
        s.factor(d["Q"], d["R"], d["S"], d["A"], d["B"], d["Sigma"])
        t = lambda a: torch.from_numpy(a).cuda()
        zz = s.solve(s.build_rhs(t(q), t(r), t(c), t(x0))).cpu().numpy()
        Z = zz.reshape(inst.N, -1)
        return float((Z[:, :inst.nu + inst.nx] ** 2).sum())

    h = 1e-6
    rng = np.random.default_rng(0)
    for name, arr, key in [("A", batch.A, "dA"), ("B", batch.B, "dB"), ("q", q, "dq"), ("c", c, "dc"),
                           ("x0", x0, "dx0"), ("r", r, "dr")]:
        for i in rng.choice(len(arr), size=min(4, len(arr)), replace=False):
            if name == "q" and i < inst.nx:
                continue
            old = arr[i]
            arr[i] = old + h
            lp = loss()
            arr[i] = old - h
            lm = loss()
            arr[i] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - G[key][i]) <= 1e-6 * max(1.0, abs(fd)), (name, i, fd, G[key][i])


def test_adjoint_vector_is_the_solve_of_the_loss_gradient():
    """K is symmetric, so w = K^{-1} dL/dz is exactly a solve with dL/dz as the
    right-hand side (the same kernels on the same factor)."""
    torch, cyq = require_gpu()
    batch = ragged_batch(53, [(9, 3, 2), (14, 5, 2)], sigma=(1e-2, 1e2))
    s = cyq.Solver(batch.N, batch.nx, batch.nu, precision="fp64", P=2, it_max=0)
    data, rhs = cyq.to_device(batch)
    s.factor(data["Q"], data["R"], data["S"], data["A"], data["B"], data["Sigma"])
    g = torch.from_numpy(np.random.default_rng(5).standard_normal(s.kkt_size)).cuda()
    z = s.solve(g.clone())
    w = s.solve_adjoint(rhs[0][3], z, g, want=("w", "dA"))["w"]
    torch.cuda.synchronize()
    assert torch.equal(w, s.solve(g))
