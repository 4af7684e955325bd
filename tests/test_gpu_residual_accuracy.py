"""The compensated residual entry point (cyq_residual_compensated) against the
oracle's accurate residual, which is itself pinned against exact rational
arithmetic (tests/test_oracle_pins.py).

On the uneven batch's instances whose rows cancel by many orders of magnitude
(nx >= 50, nu <= 4, Sigma up to 1e6) a plain float64 evaluation of
||b - K z|| / ||b|| at the solution is as large as the residual itself; the
compensated rows must still give the residual to many digits.  Away from the
solution (a large residual) both evaluations agree with the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_2512_09058_gb300 import inputs

from gpu_util import oracle_rhs, ragged_batch, require_gpu

pytestmark = pytest.mark.gpu


def _residuals(batch, z_host, b_host):
    torch, cyq = require_gpu()
    s = cyq.Solver(batch.N, batch.nx, batch.nu, precision="fp64", P=1, it_max=0)
    data, _ = cyq.to_device(batch)
    s.factor(data["Q"], data["R"], data["S"], data["A"], data["B"], data["Sigma"])
    b = torch.from_numpy(np.ascontiguousarray(b_host)).cuda()
    z = torch.from_numpy(np.ascontiguousarray(z_host)).cuda()
    comp = s.residual(b, z, compensated=True).cpu().numpy()
    plain = s.residual(b, z).cpu().numpy()
    return comp, plain


def _oracle_solutions(batch):
    bs, zs = [], []
    for x in batch.instances:
        b = oracle.build_rhs(x, *x.rhs[0])
        bs.append(b)
        zs.append(oracle.riccati_solve(x, b))
    return np.concatenate(zs), np.concatenate(bs), bs, zs


def test_compensated_residual_of_noise_limited_instances_matches_the_oracle():
    batch = inputs.make_batch("uneven4096", [31, 586, 1795, 2456])
    z, b, bs, zs = _oracle_solutions(batch)
    comp, plain = _residuals(batch, z, b)
    for i, x in enumerate(batch.instances):
        exact = oracle.kkt_residual(x, zs[i], bs[i])
        print("N %d nx %d nu %d: oracle %.6e compensated %.6e plain float64 %.6e"
              % (x.N, x.nx, x.nu, exact, comp[i], plain[i]))
        assert abs(comp[i] - exact) <= 1e-8 * exact


def test_compensated_and_plain_residuals_agree_away_from_the_solution():
    batch = ragged_batch(75, [(12, 6, 3), (20, 12, 4), (9, 3, 2), (16, 30, 12)], sigma=(1e-2, 1e2))
    b = oracle_rhs(batch)
    rng = np.random.default_rng(5)
    z = rng.standard_normal(b.size)
    comp, plain = _residuals(batch, z, b)
    off = 0
    for i, x in enumerate(batch.instances):
        n = x.kkt_size
        exact = oracle.kkt_residual(x, z[off:off + n], b[off:off + n])
        off += n
        assert abs(comp[i] - exact) <= 1e-13 * exact
        assert abs(plain[i] - exact) <= 1e-12 * exact
