"""The algorithmic work behind bench.py's residual roofline, pinned against
the oracle's assembled KKT matrix (eq. opt-cond-ocp-eq): one residual r = b - K z
multiplies every nonzero entry of K once, except the identity couplings between
x^{k+1} and lambda^k (a subtraction each), and evaluates Sigma as a term of its
own beside the diagonal of R and Q, so its FMA count is nnz(K) - 2 N nx
(+ N (nu + nx) with Sigma).  Covers S and Sigma present or absent, N = 1 and the
first and last stages, where A, S and their transposes drop out."""
import types

import numpy as np
import pytest

import bench
import oracle
from paper_2512_09058_gb300 import inputs


def _instance(seed, N, nx, nu, S, sigma):
    cfg = dict(batch=1, N=N, nx=nx, nu=nu, S=S, sigma=sigma, nrhs=1, QN_equals_Q0=False, seed=seed)
    inst = inputs.make_instance(cfg, 0)
    if not S:
        inst.S = None   # no S blocks: the kernel and the oracle both skip them
    return inst


@pytest.mark.parametrize("N,nx,nu,S,sigma", [(5, 3, 2, True, (1e-2, 1e2)), (7, 4, 3, False, None),
                                             (1, 3, 2, True, (1e-2, 1e2)), (2, 2, 1, False, (1e-1, 1e1)),
                                             (6, 5, 1, True, None)])
def test_residual_fma_counts_the_products_of_the_kkt_matrix(N, nx, nu, S, sigma):
    inst = _instance(11 + N, N, nx, nu, S, sigma)
    K = oracle.kkt_dense(inst)
    products = np.count_nonzero(K) - 2 * N * nx
    if inst.Sigma is not None:
        products += N * (nu + nx)
    one = types.SimpleNamespace(N=np.array([N]), nx=np.array([nx]), nu=np.array([nu]), S=inst.S,
                                Sigma=inst.Sigma)
    assert bench.residual_fma(one) == products


def test_residual_fma_sums_over_instances():
    insts = [_instance(3, 4, 3, 2, True, (1e-2, 1e2)), _instance(4, 9, 2, 2, True, (1e-2, 1e2))]
    batch = inputs.make_batch(None, instances=insts)
    each = [bench.residual_fma(types.SimpleNamespace(N=np.array([x.N]), nx=np.array([x.nx]), nu=np.array([x.nu]),
                                                     S=x.S, Sigma=x.Sigma)) for x in insts]
    assert bench.residual_fma(batch) == sum(each)
