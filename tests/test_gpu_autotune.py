"""Launch-shape and segment-count autotuners (cyq_autotune, cyq_tune_segments).

Every output element of the stage factor and of the sweeps is computed by one
thread with the same arithmetic whatever the number of threads per work item,
so tuned and default launch shapes give the same solution (compared to 1e-12);
the tuned segment counts are valid and the solve with them matches the oracle.
"""
import numpy as np
import pytest

import oracle

from gpu_util import oracle_rhs, ragged_batch, rel_err, require_gpu, split_instances

pytestmark = pytest.mark.gpu

DIMS = [(24, 3, 2), (40, 12, 4), (33, 12, 4), (16, 30, 10), (50, 6, 1), (20, 52, 20)]


def _run(batch, precision, nrhs, tune, P=0, P_per_instance=None):
    torch, cyq = require_gpu()
    s = cyq.Solver(batch.N, batch.nx, batch.nu, precision=precision, P=P, P_per_instance=P_per_instance,
                   max_nrhs=nrhs, it_max=0 if precision == "fp64" else 10)
    data, _ = cyq.to_device(batch)
    b_host = np.stack([oracle_rhs(batch, j) for j in range(nrhs)])
    b = torch.from_numpy(np.ascontiguousarray(b_host.reshape(-1))).cuda()
    if tune:
        s.autotune(data["Q"], data["R"], data["S"], data["A"], data["B"], data["Sigma"], b, nrhs=nrhs, reps=2)
    else:
        s.factor(data["Q"], data["R"], data["S"], data["A"], data["B"], data["Sigma"])
    z = s.solve(b, nrhs=nrhs)
    torch.cuda.synchronize()
    return s, z.cpu().numpy().reshape(nrhs, -1), b_host


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
@pytest.mark.parametrize("P", [1, 4])
def test_autotuned_shapes_give_the_same_solution(precision, P):
    batch = ragged_batch(41, DIMS, nrhs=2)
    s0, z0, b = _run(batch, precision, 2, False, P=P)
    s1, z1, _ = _run(batch, precision, 2, True, P=P)
    shapes = s1.launch_shapes(nrhs=2)
    print(precision, "default", s0.launch_shapes(nrhs=2), "tuned", shapes)
    assert len(shapes["factor"]) >= 2
    assert all(t in (16, 32, 64, 128) for t in shapes["factor"])
    assert all(t in (32, 64, 128, 256) for t in shapes["sweep"])
    assert (s1.instance_status() == 0).all()
    assert rel_err(z1, z0) <= 1e-12
    for inst, zi, bi in zip(batch.instances, split_instances(batch, z1[0]), split_instances(batch, b[0])):
        assert rel_err(zi, oracle.riccati_solve(inst, bi)) <= 1e-8


def test_tuned_segment_counts_are_valid_and_solve_correctly():
    torch, cyq = require_gpu()
    batch = ragged_batch(42, [(512, 8, 4), (300, 6, 3), (128, 10, 2)])
    data, _ = cyq.to_device(batch)
    b_host = oracle_rhs(batch)
    b = torch.from_numpy(b_host).cuda()
    P = cyq.tune_segments(batch.N, batch.nx, batch.nu, data, b, nrhs=1, reps=2, it_max=0)
    print("tuned segments", P)
    assert P.shape == (batch.size,)
    assert ((P >= 1) & (P <= np.asarray(batch.N))).all()
    s, z, _ = _run(batch, "fp64", 1, False, P_per_instance=P)
    assert (s.segments == P).all()
    for inst, zi, bi in zip(batch.instances, split_instances(batch, z[0]), split_instances(batch, b_host)):
        assert rel_err(zi, oracle.riccati_solve(inst, bi)) <= 1e-9


@pytest.mark.parametrize("precision", ["fp32_refine", "fp64"])
def test_launch_shapes_agree_on_a_fixed_shape_batch(precision):
    """Stage shapes with compiled float32 kernels (nx = 12, nu = 4 and nx = 8,
    nu = 4): two items per warp (16 threads each), the one-warp path (registers
    and shuffles for interior stages in float32) and the multi-warp
    shared-memory path give the same solution."""
    torch, cyq = require_gpu()
    for dims, P in [((40, 12, 4), 1), ((33, 8, 4), 1), ((64, 12, 4), 4)]:
        batch = ragged_batch(43, [dims] * 6, sigma=None, nrhs=1)
        data, _ = cyq.to_device(batch)
        b_host = oracle_rhs(batch)
        b = torch.from_numpy(b_host).cuda()
        zs = []
        for team in (16, 32, 64, 128):
            s = cyq.Solver(batch.N, batch.nx, batch.nu, precision=precision, P=P, it_max=0)
            s.set_launch_shapes(factor=[team] * len(s.launch_shapes()["factor"]))
            assert s.launch_shapes()["factor"][0] == team
            s.factor(data["Q"], data["R"], data["S"], data["A"], data["B"], data["Sigma"])
            zs.append(s.solve(b).cpu().numpy())
            s.close()
        assert all(np.array_equal(zs[0], zk) for zk in zs[1:]), (dims, P, [rel_err(zs[0], zk) for zk in zs[1:]])
        tol = 1e-3 if precision == "fp32_refine" else 1e-9
        for inst, zi, bi in zip(batch.instances, split_instances(batch, zs[0]), split_instances(batch, b_host)):
            assert rel_err(zi, oracle.riccati_solve(inst, bi)) <= tol



@pytest.mark.parametrize("precision", ["fp64", "fp64_ir32"])
def test_two_items_per_warp_float64_factor_is_bitwise_the_one_warp_factor(precision):
    """The float64 stage factor with two items per warp (16 threads per item,
    stage shapes nx = 12, nu = 4 and nx = 8, nu = 4 compiled in, one segment per
    instance) against the one-warp and multi-warp factors: the same stored
    factor bit for bit, hence the same solutions, with S, Sigma over [1e-6, 1e6],
    horizons of different lengths (1 and 2 included) side by side in one warp,
    4 right-hand sides and float32 corrections from the factor's float32 copy;
    an instance of another shape in front puts the blocks of the others at odd
    offsets (8-byte copies instead of 16-byte ones)."""
    torch, cyq = require_gpu()
    for nx, nu, front in [(12, 4, []), (8, 4, []), (12, 4, [(3, 5, 3)])]:
        dims = front + [(64, nx, nu)] * 9 + [(17, nx, nu), (1, nx, nu), (2, nx, nu), (40, nx, nu)]
        batch = ragged_batch(44 + nx, dims, sigma=(1e-6, 1e6), nrhs=4)
        data, _ = cyq.to_device(batch)
        b = torch.from_numpy(np.stack([oracle_rhs(batch, j) for j in range(4)])).cuda()
        zs, facs, sts = [], [], []
        for team in (16, 32, 128):
            s = cyq.Solver(batch.N, batch.nx, batch.nu, precision=precision, P=1, max_nrhs=4, it_max=2)
            s.set_launch_shapes(factor=[team] * len(s.launch_shapes()["factor"]))
            s.factor(data["Q"], data["R"], data["S"], data["A"], data["B"], data["Sigma"])
            zs.append(s.solve(b, nrhs=4).cpu().numpy())
            o = len(front)
            facs.append([s.stage_factor(i, st) for i in (o, o + 9, o + 10, o + 11) for st in range(batch.instances[i].N)])
            sts.append(s.instance_status())
            s.close()
        assert (sts[0] != 2).all()   # every factorization succeeded
        for k in (1, 2):
            assert np.array_equal(sts[0], sts[k])
            assert np.array_equal(zs[0], zs[k]), (nx, nu, front, k, rel_err(zs[0], zs[k]))
            assert all(np.array_equal(x, y) for x, y in zip(facs[0], facs[k])), (nx, nu, front, k)
