"""Newton-system assembly (cyq_assemble_newton) against the oracle written from
the paper's definitions (Sec. 5), and the Newton step it feeds (assembly +
cyq_factor + cyq_solve) against the oracle's step.

Tolerances: every assembled entry is one short float64 sum, so the blocks and
vectors agree with the oracle to 1e-12 of the largest entry of their kind in
the instance; the active flags agree exactly except for rows whose point lies
within 1e-9 (relative) of a bound, where both are correct; the Newton step is a
KKT solve on well-conditioned data (Sigma in [1e-2, 1e2]): 1e-10 relative, as
for the other parity tests."""
import numpy as np
import pytest

import oracle
from oracle import newton
from paper_2512_09058_gb300 import inputs

from gpu_util import ragged_batch, require_gpu, split_instances

pytestmark = pytest.mark.gpu


def _alm_batch(batch, nys, bounds="mixed", sigma=(1e-2, 1e4), seed=60):
    return [inputs.make_alm(inst, ny, seed=seed, index=i, bounds=bounds, sigma=sigma)
            for i, (inst, ny) in enumerate(zip(batch.instances, nys))]


def _to_dev(torch, alms):
    cat = inputs.concat_alm(alms)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    d = {k: t(getattr(cat, k)) for k in ("C", "D", "bl", "bu", "y", "gx", "gu", "xbar", "ubar")}
    d["sigma"] = t(cat.sig)
    d["ny"] = cat.ny
    return d, t(cat.u), t(cat.x)


def _split(batch, flat, sizes):
    out, o = [], 0
    for s in sizes:
        out.append(flat[o:o + s])
        o += s
    return out


def _gpu_assemble(torch, cyq, batch, alms):
    s = cyq.Solver(batch.N, batch.nx, batch.nu, precision="fp64", it_max=0)
    data, rhs = cyq.to_device(batch)
    q, r, c, x0 = rhs[0]
    alm_d, u, x = _to_dev(torch, alms)
    out = s.assemble_newton(data, q, r, c, x0, u, x, alm_d)
    torch.cuda.synchronize()
    return s, data, rhs, {k: v.cpu().numpy() for k, v in out.items()}


DIMS = [(6, 3, 2, 4), (1, 2, 1, 1), (9, 5, 3, 8), (17, 4, 4, 33), (12, 12, 4, 16), (3, 1, 2, 2)]


def test_assembly_matches_oracle():
    torch, cyq = require_gpu()
    batch = ragged_batch(61, [d[:3] for d in DIMS])
    alms = _alm_batch(batch, [d[3] for d in DIMS])
    s, _, _, g = _gpu_assemble(torch, cyq, batch, alms)
    insts = batch.instances
    sz = lambda f: [f(x, a) for x, a in zip(insts, alms)]
    parts = {
        "Q": _split(batch, g["Q"], sz(lambda x, a: (x.N + 1) * x.nx * x.nx)),
        "R": _split(batch, g["R"], sz(lambda x, a: x.N * x.nu * x.nu)),
        "S": _split(batch, g["S"], sz(lambda x, a: x.N * x.nu * x.nx)),
        "q": _split(batch, g["q"], sz(lambda x, a: (x.N + 1) * x.nx)),
        "r": _split(batch, g["r"], sz(lambda x, a: x.N * x.nu)),
        "c": _split(batch, g["c"], sz(lambda x, a: x.N * x.nx)),
        "yhat": _split(batch, g["yhat"], sz(lambda x, a: (x.N + 1) * a.ny)),
        "active": _split(batch, g["active"], sz(lambda x, a: (x.N + 1) * a.ny)),
    }
    n_act = 0
    for i, (inst, alm) in enumerate(zip(insts, alms)):
        q, r, f, x0 = inst.rhs[0]
        o = newton.newton_assembly(inst, alm, q, r, f, x0, alm.u, alm.x)
        for k in ("Q", "R", "S", "q", "r", "c", "yhat"):
            scale = max(1.0, np.abs(o[k]).max())
            assert np.abs(parts[k][i] - o[k]).max() <= 1e-12 * scale, (i, k)
        # active flags: exact away from ties
        zz = np.concatenate([newton.stage_constraints(inst, alm, alm.u, alm.x, x0, k)[0] for k in range(inst.N + 1)])
        zz = zz + alm.y / alm.sig
        tie = np.minimum(np.abs(zz - alm.bl), np.abs(zz - alm.bu)) <= 1e-9 * (1.0 + np.abs(zz))
        assert np.array_equal(parts["active"][i][~tie].astype(bool), o["active"][~tie]), i
        n_act += int(o["active"].sum())
    assert n_act > 0
    s.close()


@pytest.mark.parametrize("bounds", ["mixed", "fixed"])
def test_newton_step_matches_oracle(bounds):
    """Assembly, then cyq_factor of the assembled blocks and cyq_solve of the
    right-hand side built from (q~, r~, c~) with a zero initial state."""
    torch, cyq = require_gpu()
    batch = ragged_batch(62, [d[:3] for d in DIMS])
    sigma = (1e-2, 1e2) if bounds == "mixed" else (1e-3, 1e-1)
    alms = _alm_batch(batch, [d[3] for d in DIMS], bounds=bounds, sigma=sigma, seed=63)
    s, data, rhs, g = _gpu_assemble(torch, cyq, batch, alms)
    s.close()
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    step = cyq.Solver(batch.N, batch.nx, batch.nu, precision="fp64", it_max=0)
    step.factor(t(g["Q"]), t(g["R"]), t(g["S"]), data["A"], data["B"], None)
    zero = torch.zeros_like(rhs[0][3])
    b = step.build_rhs(t(g["q"]), t(g["r"]), t(g["c"]), zero)
    dz = step.solve(b.reshape(1, -1)).cpu().numpy()[0]
    assert (step.instance_status() == 0).all()
    step.close()
    for inst, alm, di in zip(batch.instances, alms, split_instances(batch, dz)):
        q, r, f, x0 = inst.rhs[0]
        o = newton.newton_assembly(inst, alm, q, r, f, x0, alm.u, alm.x)
        si = inputs.OCPInstance(N=inst.N, nx=inst.nx, nu=inst.nu, Q=o["Q"], R=o["R"], S=o["S"], A=inst.A,
                                B=inst.B, Sigma=None, rhs=[])
        do = oracle.riccati_solve(si, oracle.build_rhs(si, o["q"], o["r"], o["c"], np.zeros(inst.nx)))
        assert np.linalg.norm(di - do) <= 1e-10 * np.linalg.norm(do), (inst.N, inst.nx, inst.nu)
        if bounds == "fixed":
            # one step reaches the inner problem's stationary point (active set unchanged)
            N, nx, nu = inst.N, inst.nx, inst.nu
            d = di.reshape(N, nu + 2 * nx)
            u1 = alm.u + d[:, :nu].reshape(-1)
            x1 = alm.x.copy()
            x1[nx:] += d[:, nu:nu + nx].reshape(-1)
            res = newton.stationarity(inst, alm, q, r, f, x0, u1, x1, d[:, nu + nx:].reshape(-1))
            r0 = newton.stationarity(inst, alm, q, r, f, x0, alm.u, alm.x, np.zeros(N * nx))
            assert np.abs(res).max() <= 1e-10 * np.abs(r0).max()


def test_assembly_without_proximal_terms_and_without_S():
    """gx / gu / xbar / ubar and S absent (NULL): no proximal terms, S = 0."""
    torch, cyq = require_gpu()
    dims = [(5, 3, 2, 3), (8, 4, 1, 6)]
    batch = ragged_batch(64, [d[:3] for d in dims], S=False)
    alms = _alm_batch(batch, [d[3] for d in dims], seed=65)
    for a in alms:
        a.gx[:] = 0.0
        a.gu[:] = 0.0
    s = cyq.Solver(batch.N, batch.nx, batch.nu, precision="fp64", it_max=0)
    data, rhs = cyq.to_device(batch)
    data = dict(data, S=None)
    alm_d, u, x = _to_dev(torch, alms)
    for k in ("gx", "gu", "xbar", "ubar"):
        alm_d[k] = None
    q, r, c, x0 = rhs[0]
    out = s.assemble_newton(data, q, r, c, x0, u, x, alm_d)
    torch.cuda.synchronize()
    g = {k: v.cpu().numpy() for k, v in out.items()}
    s.close()
    oR, oq = 0, 0
    for inst, alm in zip(batch.instances, alms):
        qq, rr, f, xi = inst.rhs[0]
        inst.S[:] = 0.0
        o = newton.newton_assembly(inst, alm, qq, rr, f, xi, alm.u, alm.x)
        nR, nq = inst.N * inst.nu * inst.nu, (inst.N + 1) * inst.nx
        assert np.abs(g["R"][oR:oR + nR] - o["R"]).max() <= 1e-12 * max(1.0, np.abs(o["R"]).max())
        assert np.abs(g["q"][oq:oq + nq] - o["q"]).max() <= 1e-12 * max(1.0, np.abs(o["q"]).max())
        oR += nR
        oq += nq
