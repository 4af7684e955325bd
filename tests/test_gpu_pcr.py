"""Parallel cyclic reduction for the last levels of the coupling solve
(cyq_set_pcr_tail; paper App. A, Alg. pcr): the solution agrees with the
oracle at the parity tolerance and with plain cyclic reduction to rounding,
for segment counts that are not powers of two, mixed in one batch with
instances of one segment, for every tail length up to all levels."""
import numpy as np
import pytest

import oracle
from paper_2512_09058_gb300 import inputs

from gpu_util import REFINE_TARGET, oracle_rhs, ragged_batch, rel_err, require_gpu, split_instances

pytestmark = pytest.mark.gpu

DIMS = [(40, 4, 2), (64, 6, 3), (33, 5, 2), (30, 3, 1), (9, 2, 2), (50, 8, 4)]
PS = [16, 12, 5, 3, 1, 9]


def _solve(cyq, torch, batch, data, b, tail, nrhs=1, precision="fp64", it_max=0):
    s = cyq.Solver(batch.N, batch.nx, batch.nu, precision=precision, P_per_instance=PS, max_nrhs=nrhs,
                   it_max=it_max, tol=REFINE_TARGET)
    if tail is not None:
        s.set_pcr_tail(tail)
    s.factor(data["Q"], data["R"], data["S"], data["A"], data["B"], data["Sigma"])
    z = s.solve(b, nrhs=nrhs).cpu().numpy()
    st = s.instance_status()
    used = s.pcr_tail()
    s.close()
    return z, st, used


@pytest.mark.parametrize("tail", [1, 2, 3, 10])
def test_pcr_tail_matches_oracle_and_plain_cyclic_reduction(tail):
    torch, cyq = require_gpu()
    batch = ragged_batch(71, DIMS, nrhs=2)
    data, _ = cyq.to_device(batch)
    bh = np.stack([oracle_rhs(batch, j) for j in range(2)])
    b = torch.from_numpy(bh.reshape(-1)).cuda()
    z0, st0, _ = _solve(cyq, torch, batch, data, b, None, nrhs=2)
    z1, st1, used = _solve(cyq, torch, batch, data, b, tail, nrhs=2)
    assert used == min(tail, 4)                  # ceil(log2 16) levels in all
    assert (st0 == 0).all() and (st1 == 0).all()
    n = batch.kkt_size
    assert rel_err(z1, z0) <= 1e-12
    for j in range(2):
        for inst, zi, bi in zip(batch.instances, split_instances(batch, z1[j * n:(j + 1) * n]),
                                split_instances(batch, bh[j])):
            assert rel_err(zi, oracle.riccati_solve(inst, bi)) <= 1e-10


def test_pcr_tail_under_refinement_and_reset():
    """Float32 factor + refinement with a tail of 2 levels certifies; tail 0 goes
    back to plain cyclic reduction; a solve after re-planning without a new
    factorization is refused."""
    torch, cyq = require_gpu()
    batch = ragged_batch(72, DIMS, sigma=(1e-3, 1e3))
    data, _ = cyq.to_device(batch)
    bh = oracle_rhs(batch)
    b = torch.from_numpy(bh).cuda()
    z, st, used = _solve(cyq, torch, batch, data, b, 2, precision="fp32_refine", it_max=8)
    assert used == 2 and (st == 0).all()
    for inst, zi, bi in zip(batch.instances, split_instances(batch, z), split_instances(batch, bh)):
        assert oracle.kkt_residual(inst, zi, bi) <= 1e-10
    s = cyq.Solver(batch.N, batch.nx, batch.nu, P_per_instance=PS, it_max=0)
    s.factor(data["Q"], data["R"], data["S"], data["A"], data["B"], data["Sigma"])
    s.set_pcr_tail(3)
    with pytest.raises(cyq.CyqError):
        s.solve(b)
    s.set_pcr_tail(0)
    assert s.pcr_tail() == 0
    s.factor(data["Q"], data["R"], data["S"], data["A"], data["B"], data["Sigma"])
    z0 = s.solve(b).cpu().numpy()
    s.close()
    for inst, zi, bi in zip(batch.instances, split_instances(batch, z0), split_instances(batch, bh)):
        assert rel_err(zi, oracle.riccati_solve(inst, bi)) <= 1e-10
