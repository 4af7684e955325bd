"""Edge cases of the GPU path: the shortest horizons (N = 1, 2, 3, with segment
counts clamped to N), the largest stage blocks of the workloads (nx = 64,
nu = 32, no shared-memory staging of the raw stage), and the host-side
rejection of blocks too large for shared memory and of too many right-hand
sides."""
import numpy as np
import pytest

import oracle

from gpu_util import gpu_solve, oracle_rhs, ragged_batch, rel_err, require_gpu, split_instances

pytestmark = pytest.mark.gpu


def _check(batch, z, b, tol):
    for j in range(z.shape[0]):
        for inst, zi, bi in zip(batch.instances, split_instances(batch, z[j]), split_instances(batch, b[j])):
            assert rel_err(zi, oracle.riccati_solve(inst, bi)) <= tol, (inst.N, inst.nx, inst.nu)


@pytest.mark.parametrize("P", [1, 2, 3])
def test_shortest_horizons(P):
    batch = ragged_batch(61, [(1, 1, 1), (1, 3, 2), (2, 2, 1), (3, 1, 2), (2, 4, 3), (3, 3, 3)])
    z, s, _, b = gpu_solve(batch, P=P)
    assert list(s.segments) == [min(P, int(n)) for n in batch.N]
    assert (s.instance_status() == 0).all()
    _check(batch, z, b, 1e-10)


@pytest.mark.parametrize("precision,P", [("fp64", 1), ("fp32_refine", 1), ("fp32_refine", 2)])
def test_largest_workload_blocks(precision, P):
    batch = ragged_batch(62, [(5, 64, 32), (3, 64, 32), (4, 63, 31)], sigma=(1e-2, 1e2))
    z, s, _, b = gpu_solve(batch, precision=precision, P=P, it_max=0 if precision == "fp64" else 10)
    assert (s.instance_status() == 0).all()
    _check(batch, z, b, 1e-9)


def test_oversized_blocks_and_rhs_count_are_rejected():
    torch, cyq = require_gpu()
    with pytest.raises(cyq.CyqError) as e:
        cyq.Solver([4], [200], [120], precision="fp64")
    assert e.value.code == 1
    batch = ragged_batch(63, [(6, 3, 2)])
    s = cyq.Solver(batch.N, batch.nx, batch.nu, max_nrhs=1, it_max=0)
    data, _ = cyq.to_device(batch)
    s.factor(data["Q"], data["R"], data["S"], data["A"], data["B"], data["Sigma"])
    b = torch.zeros(2 * s.kkt_size, dtype=torch.float64, device="cuda")
    with pytest.raises(cyq.CyqError) as e:
        s.solve(b, nrhs=2)
    assert e.value.code == 1
