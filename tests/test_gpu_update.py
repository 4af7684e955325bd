"""Factorization updates (cyq_update_factor, Sec. 6) against the plain
definition: the factor of the modified KKT matrix.

Stage matrices change by sum_r delta_r w_r w_r^T (rows with delta > 0 add
constraint penalties, delta < 0 remove them).  After the update the solve
must equal the oracle's solve of the modified problem, built here by adding
the rank terms to R, S and Q, and the GPU's own refactorization of that
problem; an update followed by the downdate of the same rows gives back the
original solution.  Float32 and three-precision handles reach the refinement
gate with the updated factor.
"""
import numpy as np
import pytest

import oracle
from paper_2512_09058_gb300 import inputs

from gpu_util import REFINE_TARGET, oracle_rhs, ragged_batch, rel_err, require_gpu, split_instances

pytestmark = pytest.mark.gpu

DIMS = [(12, 6, 3), (20, 12, 4), (9, 3, 2), (16, 8, 8), (7, 20, 10), (25, 5, 1)]


def _rows(batch, m_max, seed, prob=0.3, sign=1.0):
    """Random update rows per stage (stage 0: u-only or x-only rows)."""
    g = np.random.default_rng(seed)
    W, D = [], []
    for x in batch.instances:
        n = x.nu + x.nx
        w = g.standard_normal((x.N, m_max, n)) / np.sqrt(n)
        d = np.where(g.uniform(size=(x.N, m_max)) < prob, sign * 10.0 ** g.uniform(-2, 1, size=(x.N, m_max)), 0.0)
        # stage 0 couples u^0 with x^N: a row there is a row of D_0 (u part) or of C_N (x part)
        for r in range(m_max):
            if r % 2 == 0:
                w[0, r, x.nu:] = 0.0
            else:
                w[0, r, :x.nu] = 0.0
        W.append(w)
        D.append(d)
    return W, D


def _modified(x, w, d):
    """The instance with its stage matrices changed by the rank terms (data layout of inputs)."""
    N, nx, nu = x.N, x.nx, x.nu
    R, S, Q = x.R.copy(), x.S.copy(), x.Q.copy()
    for s in range(N):
        for r in range(w.shape[1]):
            if d[s, r] == 0.0:
                continue
            wu, wx = w[s, r, :nu], w[s, r, nu:]
            R[s * nu * nu:(s + 1) * nu * nu] += (d[s, r] * np.outer(wu, wu)).flatten(order="F")
            xq = s if s > 0 else N
            Q[xq * nx * nx:(xq + 1) * nx * nx] += (d[s, r] * np.outer(wx, wx)).flatten(order="F")
            if s > 0:
                S[s * nu * nx:(s + 1) * nu * nx] += (d[s, r] * np.outer(wu, wx)).flatten(order="F")
    return inputs.OCPInstance(N=N, nx=nx, nu=nu, Q=Q, R=R, S=S, A=x.A, B=x.B, Sigma=x.Sigma, rhs=x.rhs)


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _solver(batch, precision, it_max):
    torch, cyq = require_gpu()
    s = cyq.Solver(batch.N, batch.nx, batch.nu, precision=precision, P=1, it_max=it_max, tol=REFINE_TARGET)
    data, _ = cyq.to_device(batch)
    s.factor(data["Q"], data["R"], data["S"], data["A"], data["B"], data["Sigma"])
    return torch, s, data


def _update(torch, s, mod, W, D, m_max):
    wd = _dev(torch, np.concatenate([w.reshape(-1) for w in W]))
    dd = _dev(torch, np.concatenate([d.reshape(-1) for d in D]))
    md = {k: _dev(torch, getattr(mod, k)) for k in ("Q", "R", "S")}
    s.update_factor(md["Q"], md["R"], md["S"], wd, dd, m_max)
    return md, wd, dd


@pytest.mark.parametrize("m_max", [1, 3])
def test_update_equals_the_factor_of_the_modified_problem(m_max):
    batch = ragged_batch(81, DIMS, sigma=(1e-2, 1e2))
    W, D = _rows(batch, m_max, 82)
    mod = inputs.make_batch(None, instances=[_modified(x, w, d) for x, w, d in zip(batch.instances, W, D)])
    torch, s, data = _solver(batch, "fp64", 0)
    md, _, _ = _update(torch, s, mod, W, D, m_max)
    b = oracle_rhs(mod)   # the right-hand side does not depend on R, Q (S_0 is not read)
    z = s.solve(_dev(torch, b)).cpu().numpy()
    assert (s.instance_status() == 0).all()
    # the GPU's refactorization of the modified data
    _, cyq = require_gpu()
    s2 = cyq.Solver(mod.N, mod.nx, mod.nu, precision="fp64", P=1, it_max=0)
    d2, _ = cyq.to_device(mod)
    s2.factor(d2["Q"], d2["R"], d2["S"], d2["A"], d2["B"], d2["Sigma"])
    z2 = s2.solve(_dev(torch, b)).cpu().numpy()
    for x, zi, z2i, bi in zip(mod.instances, split_instances(mod, z), split_instances(mod, z2),
                              split_instances(mod, b)):
        zo = oracle.riccati_solve(x, bi)
        assert rel_err(zi, zo) <= 1e-10, (x.N, x.nx, x.nu, rel_err(zi, zo))
        assert rel_err(zi, z2i) <= 1e-11
    # the stored stage factor of the updated problem is the refactorization's (L^Q L^Q^T = cost-to-go)
    for i, x in enumerate(mod.instances):
        for st in (0, x.N - 1, 1):
            L1, L2 = s.stage_factor(i, st), s2.stage_factor(i, st)
            lo = np.tril(np.ones_like(L1, dtype=bool))
            assert np.linalg.norm((L1 - L2)[lo]) <= 1e-11 * np.linalg.norm(L2[lo]), (i, st)


def test_update_then_downdate_restores_the_solution():
    batch = ragged_batch(83, DIMS, sigma=(1e-2, 1e2))
    W, D = _rows(batch, 2, 84)
    mod = inputs.make_batch(None, instances=[_modified(x, w, d) for x, w, d in zip(batch.instances, W, D)])
    torch, s, data = _solver(batch, "fp64", 0)
    b = oracle_rhs(batch)
    z0 = s.solve(_dev(torch, b)).cpu().numpy()
    md1 = _update(torch, s, mod, W, D, 2)
    md2 = _update(torch, s, batch, W, [-d for d in D], 2)   # the same rows removed again
    z1 = s.solve(_dev(torch, b)).cpu().numpy()
    assert (s.instance_status() == 0).all()
    for x, a, c in zip(batch.instances, split_instances(batch, z0), split_instances(batch, z1)):
        assert rel_err(c, a) <= 1e-10, (x.N, x.nx, x.nu)


@pytest.mark.parametrize("precision", ["fp32_refine", "fp64_ir32"])
def test_updated_factor_with_refinement_reaches_the_gate(precision):
    batch = ragged_batch(85, DIMS, sigma=(1e-2, 1e2))
    W, D = _rows(batch, 2, 86)
    mod = inputs.make_batch(None, instances=[_modified(x, w, d) for x, w, d in zip(batch.instances, W, D)])
    torch, s, data = _solver(batch, precision, 10)
    md, _, _ = _update(torch, s, mod, W, D, 2)   # the handle borrows the updated data: keep it alive
    b = oracle_rhs(mod)
    z = s.solve(_dev(torch, b)).cpu().numpy()
    assert (s.instance_status() == 0).all()
    for x, zi, bi in zip(mod.instances, split_instances(mod, z), split_instances(mod, b)):
        assert oracle.kkt_residual(x, zi, bi) <= 1e-10


def test_rank_above_the_workspace_and_multi_segment_handles_are_reported():
    batch = ragged_batch(87, [(60, 4, 2), (8, 4, 2)], sigma=(1e-2, 1e2))
    W, D = _rows(batch, 2, 88, prob=1.0)   # two new rows at every stage: 2 N columns carried
    mod = inputs.make_batch(None, instances=[_modified(x, w, d) for x, w, d in zip(batch.instances, W, D)])
    torch, s, data = _solver(batch, "fp64", 0)
    _update(torch, s, mod, W, D, 2)
    st = s.instance_status()
    assert st[0] == 9 and st[1] == 0
    torch, cyq = require_gpu()
    s3 = cyq.Solver(batch.N, batch.nx, batch.nu, precision="fp64", P=2, it_max=0)
    s3.factor(data["Q"], data["R"], data["S"], data["A"], data["B"], data["Sigma"])
    with pytest.raises(cyq.CyqError) as e:
        _update(torch, s3, mod, W, D, 2)
    assert e.value.code == 7
