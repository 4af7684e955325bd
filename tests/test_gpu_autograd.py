"""torch.autograd.Function over cyq (paper_2512_09058_gb300.autograd): the
gradients of a loss of the KKT solution match the oracle's adjoint, also when
the solver has factored another problem before the backward pass."""
import numpy as np
import pytest

import oracle

from gpu_util import ragged_batch, rel_err, require_gpu

pytestmark = pytest.mark.gpu


def _tensors(torch, batch, rg=True):
    t = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda().requires_grad_(rg)
    q, r, c, x0 = batch.rhs[0]
    return [t(batch.Q), t(batch.R), t(batch.S), t(batch.A), t(batch.B), t(batch.Sigma), t(q), t(r), t(c), t(x0)]


def _loss(torch, batch, z):
    tot = 0.0
    off = 0
    for x in batch.instances:
        Z = z[off:off + x.kkt_size].view(x.N, x.nu + 2 * x.nx)
        tot = tot + (Z[:, :x.nu + x.nx] ** 2).sum()
        off += x.kkt_size
    return tot


def _check_against_oracle(batch, args, z):
    names = ["Q", "R", "S", "A", "B", "Sigma", "q", "r", "c", "x0"]
    keys = {"Q": "dQ", "R": "dR", "S": "dS", "A": "dA", "B": "dB", "Sigma": "dSigma", "q": "dq", "r": "dr",
            "c": "dc", "x0": "dx0"}
    grads = {n: a.grad.cpu().numpy() for n, a in zip(names, args) if a is not None}
    zh = z.detach().cpu().numpy()
    offs = {n: 0 for n in names}
    zoff = 0
    for inst in batch.instances:
        N, nx, nu = inst.N, inst.nx, inst.nu
        sizes = dict(Q=(N + 1) * nx * nx, R=N * nu * nu, S=N * nu * nx, A=N * nx * nx, B=N * nx * nu,
                     Sigma=(N + 1) * (nu + nx), q=(N + 1) * nx, r=N * nu, c=N * nx, x0=nx)
        zi = zh[zoff:zoff + inst.kkt_size]
        g = np.zeros_like(zi).reshape(N, -1)
        g[:, :nu + nx] = 2 * zi.reshape(N, -1)[:, :nu + nx]
        ref = oracle.adjoint(inst, inst.rhs[0][3], zi, g.ravel())
        for n in names:
            if n in grads:
                got = grads[n][offs[n]:offs[n] + sizes[n]]
                assert rel_err(got, ref[keys[n]]) <= 1e-9, (n, rel_err(got, ref[keys[n]]))
            offs[n] += sizes[n]
        zoff += inst.kkt_size


@pytest.mark.parametrize("precision,P", [("fp64", 1), ("fp64", 3), ("fp32_refine", 2)])
def test_autograd_matches_oracle_adjoint(precision, P):
    torch, cyq = require_gpu()
    from paper_2512_09058_gb300.autograd import kkt_solve
    batch = ragged_batch(51, [(9, 4, 2), (12, 3, 3)], sigma=(1e-1, 1e1))
    s = cyq.Solver(batch.N, batch.nx, batch.nu, precision=precision, P=P)
    args = _tensors(torch, batch)
    z = kkt_solve(s, *args)
    _loss(torch, batch, z).backward()
    _check_against_oracle(batch, args, z)


def test_autograd_refactors_when_solver_was_reused():
    torch, cyq = require_gpu()
    from paper_2512_09058_gb300.autograd import kkt_solve
    dims = [(8, 3, 2), (10, 4, 1)]
    b1 = ragged_batch(52, dims, sigma=(1e-1, 1e1))
    b2 = ragged_batch(53, dims, sigma=(1e-1, 1e1))
    s = cyq.Solver(b1.N, b1.nx, b1.nu, precision="fp64", P=2)
    a1 = _tensors(torch, b1)
    z1 = kkt_solve(s, *a1)
    a2 = _tensors(torch, b2, rg=False)
    z2 = kkt_solve(s, *a2)          # the solver now holds the factor of the second problem
    _loss(torch, b1, z1).backward()
    _check_against_oracle(b1, a1, z1)
