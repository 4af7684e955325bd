"""The persistent float32 factor (one launch for the whole batch, a team of 32,
64 or 128 threads per work item) against the per-size-class kernels and the
oracle.

The two paths run the same recursion (Alg. fact-mod-riccati without the A^cl
terms on segment 0, then compute-schur) with different summation orders, so
their stored stage factors agree to float32 rounding, and the refined
solutions of both agree with the oracle at the refinement gate.  The shapes
cover every residue of nu and nx modulo 4 (the kernel pads both to multiples
of 4), the three register buckets (padded nx <= 16, 32, 64), the largest
padded blocks (nu + nx up to 96), horizons of one and two stages, and segment
counts 1 and 3 (segment 0 by the persistent kernel, the others by the
per-class kernels).
"""
import numpy as np
import pytest

import oracle

from gpu_util import oracle_rhs, ragged_batch, rel_err, require_gpu, split_instances

pytestmark = pytest.mark.gpu

DIMS = [(1, 3, 2), (2, 5, 1), (7, 4, 4), (12, 6, 3), (9, 13, 7), (16, 17, 5), (11, 29, 14), (8, 31, 30),
        (10, 33, 9), (6, 47, 18), (5, 60, 27), (4, 64, 32), (3, 62, 31), (13, 8, 2)]


def _solver(batch, P, warp):
    torch, cyq = require_gpu()
    s = cyq.Solver(batch.N, batch.nx, batch.nu, precision="fp32_refine", P=P, it_max=12)
    s.set_factor_path(warp)
    data, _ = cyq.to_device(batch)
    s.factor(data["Q"], data["R"], data["S"], data["A"], data["B"], data["Sigma"])
    b_host = oracle_rhs(batch)
    b = torch.from_numpy(b_host).cuda()
    z = s.solve(b)
    torch.cuda.synchronize()
    return s, z.cpu().numpy(), b_host


@pytest.mark.parametrize("P", [1, 3])
def test_one_warp_factor_matches_the_per_class_kernels_and_the_oracle(P):
    batch = ragged_batch(71, DIMS, sigma=(1e-2, 1e2))
    sw, zw, b = _solver(batch, P, True)
    sc, zc, _ = _solver(batch, P, False)
    path = sw.factor_path()
    assert path["one_warp_per_item"] and path["warp_items"] == len(DIMS)
    assert not sc.factor_path()["one_warp_per_item"]
    assert (sw.instance_status() == 0).all() and (sc.instance_status() == 0).all()
    worst = 0.0
    for i, x in enumerate(batch.instances):
        seg = min(P, x.N)
        # stages of segment 0: stage 0 and the last N - floor((P-1) N / P) - 1 stages
        b_last = ((seg - 1) * x.N) // seg
        stages = [0] + list(range(b_last + 1, x.N))
        for st in stages[:4]:
            Lw, Lc = sw.stage_factor(i, st), sc.stage_factor(i, st)
            e = np.linalg.norm(Lw - Lc) / np.linalg.norm(Lc)
            worst = max(worst, e)
            assert e <= 2e-5, (i, x.N, x.nx, x.nu, st, e)
    print("worst relative difference of the stored stage factors", worst)
    for x, zi, zj, bi in zip(batch.instances, split_instances(batch, zw), split_instances(batch, zc),
                             split_instances(batch, b)):
        zo = oracle.riccati_solve(x, bi)
        assert rel_err(zi, zo) <= 1e-10, (x.N, x.nx, x.nu)
        assert rel_err(zj, zo) <= 1e-10, (x.N, x.nx, x.nu)
        assert oracle.kkt_residual(x, zi, bi) <= 1e-10


def test_one_warp_factor_reports_a_failed_pivot():
    batch = ragged_batch(72, [(6, 9, 3), (6, 9, 3), (5, 20, 6)], sigma=None)
    nu = 3
    # instance 1, stage 0: R_0 = 0, so the first pivot fails
    o = 1 * 6 * nu * nu
    batch.R[o:o + nu * nu] = 0.0
    batch.instances[1].R[:nu * nu] = 0.0
    torch, cyq = require_gpu()
    s = cyq.Solver(batch.N, batch.nx, batch.nu, precision="fp32_refine", P=1, it_max=2, esc_max=0)
    data, _ = cyq.to_device(batch)
    s.factor(data["Q"], data["R"], data["S"], data["A"], data["B"], data["Sigma"])
    st = s.instance_status()
    assert st[1] == 2 and st[0] == 0 and st[2] == 0
