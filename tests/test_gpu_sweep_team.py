"""The float32 sweeps as one persistent launch over the whole batch against one
launch per size class.

Both run the same per-item sweep code (the backward and forward sweeps of the
segment solve, Sec. 4.2 and eq. chol-fac-K-cyqlone) with the same order of
operations in every dot product, so with one factor the two paths must give the
same solution bit for bit: a scheduling fault (an item skipped, run twice, or
given another item's slot) cannot hide under a tolerance.  The refined solves
of both reach the gate too.
"""
import numpy as np
import pytest

import oracle

from gpu_util import GATE, REFINE_TARGET, oracle_rhs, ragged_batch, require_gpu, split_instances

pytestmark = pytest.mark.gpu

DIMS = [(1, 3, 2), (2, 5, 1), (7, 4, 4), (12, 6, 3), (9, 13, 7), (16, 17, 5), (11, 29, 14), (8, 31, 30),
        (10, 33, 9), (6, 47, 18), (5, 60, 27), (4, 64, 32), (3, 62, 31), (13, 8, 2), (40, 20, 8), (25, 11, 3)]


def _solve(batch, P, it_max, persistent, s=None, data=None):
    torch, cyq = require_gpu()
    if s is None:
        s = cyq.Solver(batch.N, batch.nx, batch.nu, precision="fp32_refine", P=P, it_max=it_max, tol=REFINE_TARGET)
        data, _ = cyq.to_device(batch)
        s.factor(data["Q"], data["R"], data["S"], data["A"], data["B"], data["Sigma"])
    s.set_sweep_path(persistent)
    assert s.factor_path()["sweep_persistent"] == persistent
    b = oracle_rhs(batch)
    z = s.solve(torch.from_numpy(b).cuda())
    torch.cuda.synchronize()
    return s, data, z.cpu().numpy(), b


@pytest.mark.parametrize("P", [1, 3])
def test_persistent_sweeps_equal_the_per_class_sweeps_bit_for_bit(P):
    batch = ragged_batch(73, DIMS, sigma=(1e-2, 1e2))
    s, data, z1, b = _solve(batch, P, 0, True)
    _, _, z2, _ = _solve(batch, P, 0, False, s, data)
    assert np.array_equal(z1, z2)


def test_refined_solves_of_both_sweep_paths_reach_the_gate():
    batch = ragged_batch(74, DIMS, sigma=(1e-3, 1e3))
    for persistent in (True, False):
        s, data, z, b = _solve(batch, 1, 8, persistent)
        assert (s.instance_status() == 0).all()
        for x, zi, bi in zip(batch.instances, split_instances(batch, z), split_instances(batch, b)):
            assert oracle.kkt_residual(x, zi, bi) <= GATE
