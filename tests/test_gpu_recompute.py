"""Stage factors recomputed when memory requires it (cyq_desc.recompute_factors).

A recompute-mode handle keeps the stage factors of one chunk of instances at a
time and factors every chunk again inside each solve and adjoint.  Its
solutions and gradients are those of the handle that stores every factor (the
same kernels on the same data: equal to 1e-12), and its gradients match the
oracle's dense adjoint (1e-9).  Refined float32 solves reach the gate too.
"""
import numpy as np
import pytest

import oracle

from gpu_util import REFINE_TARGET, oracle_rhs, ragged_batch, rel_err, require_gpu, split_instances

pytestmark = pytest.mark.gpu

DIMS = [(10, 4, 2), (7, 3, 3), (16, 6, 2), (12, 24, 8), (9, 5, 5), (20, 8, 4), (6, 12, 3)]
SIZES = lambda x: dict(w=x.kkt_size, dQ=(x.N + 1) * x.nx * x.nx, dq=(x.N + 1) * x.nx, dR=x.N * x.nu * x.nu,
                       dr=x.N * x.nu, dS=x.N * x.nu * x.nx, dA=x.N * x.nx * x.nx, dB=x.N * x.nx * x.nu,
                       dc=x.N * x.nx, dx0=x.nx, dSigma=(x.N + 1) * (x.nu + x.nx))


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


def _run(batch, precision, chunks, it_max):
    torch, cyq = require_gpu()
    s = cyq.Solver(batch.N, batch.nx, batch.nu, precision=precision, P=1, it_max=it_max, recompute_chunks=chunks,
                   tol=REFINE_TARGET)
    data, rhs = cyq.to_device(batch)
    s.factor(data["Q"], data["R"], data["S"], data["A"], data["B"], data["Sigma"])
    q, r, c, x0 = rhs[0]
    b = s.build_rhs(q, r, c, x0)
    z = s.solve(b)
    g = torch.from_numpy(_loss_grad(batch, z.cpu().numpy())).cuda()
    out = s.solve_adjoint(x0, z, g)
    torch.cuda.synchronize()
    st = s.instance_status()
    return {k: v.cpu().numpy() for k, v in out.items()}, z.cpu().numpy(), g.cpu().numpy(), b.cpu().numpy(), st


@pytest.mark.parametrize("chunks", [2, 3, 7])
def test_recomputed_factors_give_the_stored_factor_results(chunks):
    batch = ragged_batch(91, DIMS, sigma=(1e-1, 1e1))
    G0, z0, g0, b0, st0 = _run(batch, "fp64", 0, 3)
    G1, z1, g1, b1, st1 = _run(batch, "fp64", chunks, 3)
    assert (st0 == 0).all() and (st1 == 0).all()
    assert np.array_equal(b0, b1)
    assert rel_err(z1, z0) <= 1e-12
    for k in G0:
        assert rel_err(G1[k], G0[k]) <= 1e-12, k
    # and the oracle's dense adjoint
    offs = {k: 0 for k in G1}
    for x in batch.instances:
        zi = z1[offs["w"]:offs["w"] + x.kkt_size]
        gi = g1[offs["w"]:offs["w"] + x.kkt_size]
        ref = oracle.adjoint(x, x.rhs[0][3], zi, gi)
        for k, n in SIZES(x).items():
            got = G1[k][offs[k]:offs[k] + n]
            assert rel_err(got, ref[k]) <= 1e-9, (k, x.N, x.nx, x.nu, rel_err(got, ref[k]))
            offs[k] += n


def test_recompute_mode_float32_refinement_reaches_the_gate():
    batch = ragged_batch(92, DIMS, sigma=(1e-2, 1e2))
    _, z, _, b, st = _run(batch, "fp32_refine", 3, 10)
    assert (st == 0).all()
    for x, zi, bi in zip(batch.instances, split_instances(batch, z), split_instances(batch, b)):
        assert oracle.kkt_residual(x, zi, bi) <= 1e-10
