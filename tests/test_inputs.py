"""The seeded synthetic inputs against the recipe they are drawn by: A_k scaled
to spectral radius 0.95, Q and R symmetric positive definite with eigenvalues
above 0.1, the stage block [R S; S^T Q] kept positive definite with its
smallest eigenvalue at least 0.05 where S is drawn, Sigma inside the
configured range, the uneven workload's dimensions inside theirs, and every
instance reproducible on its own from (config seed, index)."""
import numpy as np
import pytest

from paper_2512_09058_gb300 import inputs


def _blocks(inst):
    N, nx, nu = inst.N, inst.nx, inst.nu
    f = inputs.flat_to_blocks
    return (f(inst.A, N, nx, nx), f(inst.B, N, nx, nu), f(inst.Q, N + 1, nx, nx), f(inst.R, N, nu, nu),
            f(inst.S, N, nu, nx))


@pytest.mark.parametrize("S,sigma", [(True, (1e-6, 1e6)), (False, None)])
def test_instance_follows_the_recipe(S, sigma):
    cfg = dict(batch=4, N=12, nx=6, nu=3, S=S, sigma=sigma, nrhs=2, QN_equals_Q0=False, seed=9)
    for index in range(3):
        inst = inputs.make_instance(cfg, index)
        A, B, Q, R, Sb = _blocks(inst)
        rho = np.abs(np.linalg.eigvals(A)).max(axis=1)
        assert np.allclose(rho, 0.95, rtol=0, atol=1e-12)
        for M in list(Q) + list(R):
            assert np.array_equal(M, M.T)
            assert np.linalg.eigvalsh(M)[0] > 0.1 - 1e-12
        H = np.zeros((inst.N, inst.nu + inst.nx, inst.nu + inst.nx))
        H[:, :inst.nu, :inst.nu], H[:, :inst.nu, inst.nu:] = R, Sb
        H[:, inst.nu:, :inst.nu], H[:, inst.nu:, inst.nu:] = Sb.transpose(0, 2, 1), Q[:inst.N]
        lmin = np.linalg.eigvalsh(H)[:, 0]
        if S:
            assert np.any(Sb != 0.0)
            assert (lmin >= 0.05 - 1e-12).all()
        else:
            assert not np.any(Sb)
        if sigma is None:
            assert inst.Sigma is None
        else:
            assert inst.Sigma.shape == ((inst.N + 1) * (inst.nu + inst.nx),)
            assert (inst.Sigma >= sigma[0]).all() and (inst.Sigma <= sigma[1]).all()
        assert len(inst.rhs) == 2
        q, r, c, x0 = inst.rhs[0]
        assert q.shape == ((inst.N + 1) * inst.nx,) and r.shape == (inst.N * inst.nu,)
        assert c.shape == (inst.N * inst.nx,) and x0.shape == (inst.nx,)
        # B ~ N(0, 1/nx): the scaled entries have unit variance (loose, 216 samples)
        assert 0.6 < np.var(B * np.sqrt(inst.nx)) < 1.5


def test_terminal_cost_equals_the_first_stage_cost_where_configured():
    cfg = dict(inputs.CONFIGS["single_n32_nx8_nu4"])
    inst = inputs.make_instance(cfg, 0)
    Q = inputs.flat_to_blocks(inst.Q, inst.N + 1, inst.nx, inst.nx)
    assert np.array_equal(Q[inst.N], Q[0])


def test_instances_regenerate_alone_and_in_any_subset():
    cfg = dict(batch=6, N=(3, 9), nx=(2, 5), nu=(1, 3), S=True, sigma=(1e-2, 1e2), nrhs=1,
               QN_equals_Q0=False, seed=17)
    whole = inputs.make_batch(cfg, workers=1)
    part = inputs.make_batch(cfg, [4, 1], workers=1)
    for k, i in enumerate([4, 1]):
        a, b = whole.instances[i], part.instances[k]
        for name in ("Q", "R", "S", "A", "B", "Sigma"):
            assert np.array_equal(getattr(a, name), getattr(b, name)), name
        assert all(np.array_equal(x, y) for x, y in zip(a.rhs[0], b.rhs[0]))
    # the batch concatenates its instances in order
    assert np.array_equal(whole.A, np.concatenate([x.A for x in whole.instances]))
    assert list(whole.N) == [x.N for x in whole.instances]


def test_uneven_dimensions_stay_in_their_ranges():
    cfg = inputs.CONFIGS["uneven4096"]
    N, nx, nu = inputs.config_dims(cfg, indices=range(600))
    assert N.min() >= 16 and N.max() <= 256 and nx.min() >= 4 and nx.max() <= 64
    assert nu.min() >= 2 and nu.max() <= 32
    # every value of the small ranges appears (uniform draws)
    assert set(nu.tolist()) == set(range(2, 33))
    again = inputs.config_dims(cfg, indices=[7, 3])
    assert [int(again[0][0]), int(again[0][1])] == [int(N[7]), int(N[3])]
