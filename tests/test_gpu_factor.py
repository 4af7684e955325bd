"""The stored factor itself: within segment 0 the Cholesky factor L^Q_s of each
stage matrix satisfies L^Q_s L^Q_s^T = P_s, the Riccati cost-to-go of x^s
(P_N for stage 0, which pairs u^0 with x^N) -- the factorized Riccati recursion
(Sec. 4.1).  P_s comes from the oracle's textbook recursion, a different
algorithm; the stored strict upper triangle holds L^{R-1}."""
import numpy as np
import pytest

import oracle

from gpu_util import ragged_batch, require_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32_refine", 1e-4)])
@pytest.mark.parametrize("P", [1, 3])
def test_segment0_factor_is_the_riccati_cost_to_go(precision, tol, P):
    torch, cyq = require_gpu()
    batch = ragged_batch(51, [(12, 4, 2), (9, 3, 3)], sigma=(1e-1, 1e1))
    s = cyq.Solver(batch.N, batch.nx, batch.nu, precision=precision, P=P, it_max=0)
    data, _ = cyq.to_device(batch)
    s.factor(data["Q"], data["R"], data["S"], data["A"], data["B"], data["Sigma"])
    for i, inst in enumerate(batch.instances):
        N, nx, nu = inst.N, inst.nx, inst.nu
        q, r, c, x0 = inst.rhs[0]
        _, Pk = oracle.riccati_solve(inst, oracle.build_rhs(inst, q, r, c, x0), return_P=True)  # Pk[j-1] = P_j
        # segment 0: stage 0 and stages b_{P-1}+1 .. N-1, with b_c = floor(c N / P)
        seg0 = [0] + list(range((P - 1) * N // P + 1, N))
        for st in seg0:
            L = s.stage_factor(i, st)
            LR, LQ = np.tril(L[:nu, :nu]), np.tril(L[nu:, nu:])
            Pref = Pk[N - 1] if st == 0 else Pk[st - 1]
            assert np.linalg.norm(LQ @ LQ.T - Pref) <= tol * np.linalg.norm(Pref), (i, st)
            # strict upper triangle of the R block: L^{R-1}, transposed
            X = np.tril(np.triu(L[:nu, :nu], 1).T, -1) + np.diag(1.0 / np.diag(LR))
            assert np.linalg.norm(X @ LR - np.eye(nu)) <= 10 * tol * nu, (i, st)
