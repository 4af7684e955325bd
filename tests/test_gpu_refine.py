"""Iterative refinement on the GPU: float32 factor/solve + float64 residual
(and float64 factor + float64 residual), checked with the oracle's own FP64
residual routine on the returned z (gate: relative KKT residual <= 1e-10) and
against the oracle's solution."""
import numpy as np
import pytest

import oracle
from paper_2512_09058_gb300 import inputs

from gpu_util import GATE, REFINE_TARGET, gpu_solve, oracle_rhs, ragged_batch, rel_err, require_gpu, split_instances

pytestmark = pytest.mark.gpu

# The device refines to REFINE_TARGET (5e-11); the oracle's independent
# float64 evaluation of the same z must meet the gate (1e-10) itself.
TOL = GATE


def _residuals(batch, z, b):
    out = []
    for j in range(z.shape[0]):
        for inst, zi, bi in zip(batch.instances, split_instances(batch, z[j]), split_instances(batch, b[j])):
            res = oracle.kkt_residual(inst, zi, bi)
            out.append((res, rel_err(zi, oracle.riccati_solve(inst, bi))))
    return np.array(out)


@pytest.mark.parametrize("precision", ["fp32_refine", "fp64", "fp64_ir32"])
@pytest.mark.parametrize("P", [1, 4])
def test_refinement_reaches_tolerance_on_ragged_batch(precision, P):
    dims = [(8, 3, 2), (17, 6, 3), (32, 12, 4), (5, 2, 1), (40, 20, 8)]
    batch = ragged_batch(21, dims, sigma=(1e-3, 1e3), nrhs=2)
    z, s, _, b = gpu_solve(batch, precision=precision, nrhs=2, it_max=10,
                           P_per_instance=[min(P, d[0]) for d in dims])
    assert (s.instance_status() == 0).all()
    res = _residuals(batch, z, b)
    assert res[:, 0].max() <= TOL, res[:, 0].max()
    assert res[:, 1].max() <= 1e-8
    st = s.stats()
    assert st["max_rel_residual"] <= REFINE_TARGET
    assert 0 <= st["refine_steps"] <= 10


def test_fp32_refine_on_batch1024_workload_sampled():
    name = "batch1024_n64_nx12_nu4"
    batch = inputs.make_batch(name)
    z, s, _, b = gpu_solve(batch, precision="fp32_refine", nrhs=4, it_max=10)
    assert (s.instance_status() == 0).all()
    st = s.stats()
    print("fp32+refinement on batch1024:", st)
    assert st["max_rel_residual"] <= 1e-10
    rng = np.random.default_rng(3)
    sample = sorted(rng.choice(batch.size, size=16, replace=False))
    for j in range(4):
        zs, bs = split_instances(batch, z[j]), split_instances(batch, b[j])
        for i in sample:
            inst = batch.instances[i]
            assert (oracle.kkt_residual(inst, zs[i], bs[i]) <=
                    TOL)
            assert rel_err(zs[i], oracle.riccati_solve(inst, bs[i])) <= 1e-8


def test_fp64_float32_corrections_on_batch1024_workload_sampled():
    """float64 factor + solve, float32 correction sweeps (float32 copy of the
    float64 factor), float64 residual: one correction reaches 1e-10 here."""
    batch = inputs.make_batch("batch1024_n64_nx12_nu4", range(256))
    z, s, _, b = gpu_solve(batch, precision="fp64_ir32", nrhs=4, it_max=10)
    st = s.stats()
    print("fp64 + float32 corrections on batch1024[:256]:", st)
    assert (s.instance_status() == 0).all()
    assert st["max_rel_residual"] <= 1e-10 and st["refine_steps"] <= 2
    for j in (0, 3):
        zs, bs = split_instances(batch, z[j]), split_instances(batch, b[j])
        for i in (0, 17, 255):
            inst = batch.instances[i]
            assert (oracle.kkt_residual(inst, zs[i], bs[i]) <=
                    TOL)
            assert rel_err(zs[i], oracle.riccati_solve(inst, bs[i])) <= 1e-8


def test_fp64_one_refinement_step_on_batch1024_workload():
    batch = inputs.make_batch("batch1024_n64_nx12_nu4", range(128))
    z, s, _, b = gpu_solve(batch, precision="fp64", nrhs=4, it_max=10)
    st = s.stats()
    print("fp64+refinement on batch1024[:128]:", st)
    assert st["max_rel_residual"] <= 1e-10 and st["refine_steps"] <= 2


def test_no_refinement_budget_reports_not_converged():
    # it_max = 1 with float32 on a badly scaled problem cannot reach 1e-16
    batch = ragged_batch(22, [(12, 4, 2), (9, 3, 3)], sigma=(1e-6, 1e6))
    z, s, _, b = gpu_solve(batch, precision="fp32_refine", it_max=1, tol=1e-16)
    assert (s.instance_status() == 3).all()


def test_float64_escalation_rescues_hard_instances():
    # float32 with a 1-step budget cannot reach 1e-10 at Sigma in [1e-7, 1e7]; the
    # instances left above tol get a float64 factor and converge with it
    dims = [(30, 4, 24), (25, 5, 30), (16, 8, 8), (40, 3, 12)]
    batch = ragged_batch(23, dims, sigma=(1e-7, 1e7))
    z, s, _, b = gpu_solve(batch, precision="fp32_refine", it_max=1)
    assert (s.instance_status() == 0).all()
    res = _residuals(batch, z, b)
    assert res[:, 0].max() <= TOL, res[:, 0]


@pytest.mark.parametrize("early", [False, True])
@pytest.mark.parametrize("long", [False, True])
def test_float64_escalation_after_the_float32_budget_and_predicted_early(early, long):
    """Float32 corrections with float64 escalation: either after every float32
    correction, or predicted after two of them (the slow instances parked and
    factored in float64 on a second stream while the others continue).  Long
    horizons escalate on a float64 plan of their own with several segments
    per instance (halved runs of at least 12 stages)."""
    dims = [(30, 4, 24), (25, 5, 30), (16, 8, 8), (40, 3, 12), (20, 12, 4)]
    if long:
        dims = [(200, 4, 24), (97, 5, 30), (16, 8, 8), (64, 3, 12), (130, 12, 4), (48, 6, 20)]
    batch = ragged_batch(25, dims, sigma=(1e-7, 1e7))
    torch, cyq = require_gpu()
    s = cyq.Solver(batch.N, batch.nx, batch.nu, precision="fp32_refine", P=1, it_max=6, tol=REFINE_TARGET,
                   early_escalation=early)
    Pe = s.escalation_segments()
    # a float64 plan of its own: up to 16 segments of >= 12 stages per instance
    if long:
        assert list(Pe) == [16, 8, 1, 4, 8, 4], Pe
    else:
        assert list(Pe) == [2, 2, 1, 2, 1], Pe
    data, _ = cyq.to_device(batch)
    s.factor(data["Q"], data["R"], data["S"], data["A"], data["B"], data["Sigma"])
    b = oracle_rhs(batch)
    z = s.solve(torch.from_numpy(b).cuda()).cpu().numpy()
    assert (s.instance_status() == 0).all()
    for inst, zi, bi in zip(batch.instances, split_instances(batch, z), split_instances(batch, b)):
        assert oracle.kkt_residual(inst, zi, bi) <= TOL


def _certified(batch, precision, it_max, tol):
    torch, cyq = require_gpu()
    s = cyq.Solver(batch.N, batch.nx, batch.nu, precision=precision, it_max=it_max, tol=tol, certify=True)
    data, _ = cyq.to_device(batch)
    s.factor(data["Q"], data["R"], data["S"], data["A"], data["B"], data["Sigma"])
    b = oracle_rhs(batch)
    z = s.solve(torch.from_numpy(b).cuda()).cpu().numpy()
    return s, z, b


def test_certified_stop_value_bounds_the_oracle_evaluation():
    """certify: an instance stops once rel + 2 gamma_m || |b| + |K||z| || / ||b||
    <= tol (m = 2 nx + nu + 3).  Any other float64 evaluation (the oracle's) of
    the residual of the returned solution is then at most the certified value,
    and the certified value lies above the oracle's bound on its own evaluation."""
    dims = [(8, 3, 2), (17, 6, 3), (32, 12, 4), (40, 20, 8)]
    batch = ragged_batch(23, dims, sigma=(1e-3, 1e3))
    s, z, b = _certified(batch, "fp32_refine", 10, 1e-10)
    assert (s.instance_status() == 0).all()
    st = s.stats()
    assert st["max_rel_residual"] <= st["max_certified"] <= 1e-10
    for inst, zi, bi in zip(batch.instances, split_instances(batch, z), split_instances(batch, b)):
        res, bound = oracle.kkt_residual(inst, zi, bi), oracle.residual_eval_bound(inst, zi, bi)
        assert res <= st["max_certified"] and 2 * bound <= st["max_certified"]


def test_a_target_below_the_evaluation_bound_is_never_certified():
    """gamma_m || |b| + |K||z| || / ||b|| >= gamma_m (|b| alone), so a target
    below 2 gamma_m cannot be certified however small the residual gets."""
    dims = [(8, 3, 2), (12, 4, 2)]            # m = 11 and 13: 2 gamma_m >= 2.4e-15
    batch = ragged_batch(24, dims, sigma=(1e-1, 1e1))
    s, z, b = _certified(batch, "fp64", 3, 2e-15)
    print("residual reached", s.stats()["max_rel_residual"])
    assert (s.instance_status() == 3).all()
