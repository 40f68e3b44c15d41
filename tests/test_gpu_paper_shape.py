"""The paper's network shape and the Jacobian-order dispatch (GPU).

* Six hidden layers of 400 GELU units, r = 200 DIS, d_y = 25 / 64: the FP64
  path matches the oracle at 1e-10 (surrogate geometry and chains); the BF16
  path meets the Jacobian, forward and proposal-mean bars.  Here d_y < r, so
  the Jacobian runs in reverse mode (50 MFLOP per chain at d_y = 25 against
  324 MFLOP forward, Sec. 4.3's min{d_y, r} rule).
* A surrogate with r < d_y whose forward mode is cheaper: the library
  reports forward mode and matches the oracle at 1e-10 (FP64) and the BF16
  Jacobian bar.
"""
import numpy as np
import pytest

from helpers import gpu_setup, oracle_chains, oracle_setup, rel_err, step_and_compare, variant
from oracle import mmala
from workloads import BASIS_DIS, CONFIGS, SEED_CHAINS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dino():
    import paper_2403_08220_gb300 as d
    return d


@pytest.fixture(scope="module")
def ctx(dino):
    c = dino.dino_init(0)
    yield c
    c.close()


@pytest.mark.parametrize("name", ["paper_ndr_bf16", "paper_hyper_bf16"])
def test_paper_shape_fp64_matches_oracle(dino, ctx, name):
    w = variant(CONFIGS[name], precision="fp64", noise_map="perturbation")
    sid = gpu_setup(dino, ctx, w)
    info = dino.dino_surrogate_query(ctx, sid)
    assert info["jac_forward"] == 0 and info["noise_map"] == "perturbation"
    sur, E, D = oracle_setup(w)
    x = np.random.default_rng(4).standard_normal((3, w.r))
    g = dino.dino_surrogate_eval(ctx, sid, x, w.d_y)
    o = mmala.geometry(sur, x)
    for k, ref in [("f", o.f), ("J", o.J), ("phi", o.phi), ("g", o.g), ("hld", o.hld)]:
        assert rel_err(g[k], ref) <= 1e-10, k
    pool = dino.dino_chains_create(ctx, sid, 6, 1e-3, SEED_CHAINS)
    och = oracle_chains(dino, ctx, sid, w, sur, E, D, 6, 1e-3)
    step_and_compare(dino, ctx, pool, och, w, 6, 3, tol=1e-10)
    dino.dino_chains_destroy(ctx, pool)
    dino.dino_unload_surrogate(ctx, sid)


@pytest.mark.parametrize("name", ["paper_ndr_bf16", "paper_hyper_bf16"])
def test_paper_shape_bf16_bars(dino, ctx, name):
    w = CONFIGS[name]
    sid = gpu_setup(dino, ctx, w)
    sur, E, D = oracle_setup(w)
    x = np.random.default_rng(5).standard_normal((40, w.r))
    g = dino.dino_surrogate_eval(ctx, sid, x, w.d_y)
    o = mmala.geometry(sur, x)
    jrel = np.linalg.norm(g["J"] - o.J, axis=(1, 2)) / np.linalg.norm(o.J, axis=(1, 2))
    assert jrel.max() <= 1e-4
    assert rel_err(g["f"], o.f) <= 1e-4
    C = 24
    pool = dino.dino_chains_create(ctx, sid, C, w.dt, SEED_CHAINS)
    och = oracle_chains(dino, ctx, sid, w, sur, E, D, C, w.dt)
    for _ in range(2):
        dino.dino_chains_step(ctx, pool, 1, stats=False)
        och.step()
        mu = dino.dino_chains_read_last(ctx, pool, C, w.r)["mu"]
        err = np.linalg.norm(mu - och.last["mu"], axis=1) / np.linalg.norm(och.last["mu"], axis=1)
        assert err.max() <= 1e-3
    dino.dino_chains_destroy(ctx, pool)
    dino.dino_unload_surrogate(ctx, sid)


@pytest.mark.parametrize("precision", ["fp64", "bf16"])
def test_forward_mode_jacobian(dino, ctx, precision):
    w = variant(CONFIGS["small_fp64"], widths=[16, 40, 40, 64], precision=precision,
                activation=2, noise_frac=0.05)
    sid = gpu_setup(dino, ctx, w)
    assert dino.dino_surrogate_query(ctx, sid)["jac_forward"] == 1
    sur, E, D = oracle_setup(w)
    x = np.random.default_rng(6).standard_normal((70, w.r))
    g = dino.dino_surrogate_eval(ctx, sid, x, w.d_y)
    o = mmala.geometry(sur, x)
    if precision == "fp64":
        for k, ref in [("f", o.f), ("J", o.J), ("phi", o.phi), ("g", o.g), ("L", o.L)]:
            assert rel_err(g[k], ref) <= 1e-10, k
        pool = dino.dino_chains_create(ctx, sid, 10, 0.002, SEED_CHAINS)
        och = oracle_chains(dino, ctx, sid, w, sur, E, D, 10, 0.002)
        acc, _, _ = step_and_compare(dino, ctx, pool, och, w, 10, 10, tol=1e-10)
        assert np.mean(acc) > 0
        dino.dino_chains_destroy(ctx, pool)
    else:
        jrel = np.linalg.norm(g["J"] - o.J, axis=(1, 2)) / np.linalg.norm(o.J, axis=(1, 2))
        assert jrel.max() <= 1e-4
    dino.dino_unload_surrogate(ctx, sid)


PERT = variant(CONFIGS["small_fp64"], n_grid=9, r=45, widths=[45, 33, 17, 20],
               basis_kind=BASIS_DIS, activation=2, noise_frac=0.2, noise_map="eigen")


@pytest.mark.parametrize("dt", [0.01, 0.5])
def test_eigen_map_fp64_matches_oracle(dino, ctx, dt):
    """The paper's eigen map (symmetric root), per-chain Jacobi eigensolver."""
    w = PERT
    sid = gpu_setup(dino, ctx, w)
    assert dino.dino_surrogate_query(ctx, sid)["noise_map"] == "eigen"
    sur, E, D = oracle_setup(w)
    pool = dino.dino_chains_create(ctx, sid, 16, dt, SEED_CHAINS)
    och = oracle_chains(dino, ctx, sid, w, sur, E, D, 16, dt)
    assert och.noise == "eigen"
    acc, _, _ = step_and_compare(dino, ctx, pool, och, w, 16, 12, tol=1e-10)
    if dt < 0.1:
        assert np.mean(acc) > 0
    dino.dino_chains_destroy(ctx, pool)
    dino.dino_unload_surrogate(ctx, sid)


def test_eigen_map_bf16_paper_shape(dino, ctx):
    """d_y = 25, 6 x 400 GELU on the tensor path with the eigen map."""
    w = variant(CONFIGS["paper_ndr_bf16"], noise_map="eigen")
    sid = gpu_setup(dino, ctx, w)
    sur, E, D = oracle_setup(w)
    C = 24
    pool = dino.dino_chains_create(ctx, sid, C, w.dt, SEED_CHAINS)
    och = oracle_chains(dino, ctx, sid, w, sur, E, D, C, w.dt)
    for _ in range(2):
        dino.dino_chains_step(ctx, pool, 1, stats=False)
        och.step()
        last = dino.dino_chains_read_last(ctx, pool, C, w.r)
        err = np.linalg.norm(last["mu"] - och.last["mu"], axis=1) / np.linalg.norm(
            och.last["mu"], axis=1)
        assert err.max() <= 1e-3
        bdiff = np.linalg.norm(last["b"] - och.last["b"], axis=1) / np.linalg.norm(
            och.last["b"], axis=1)
        assert bdiff.max() <= 1e-3
    dino.dino_chains_destroy(ctx, pool)
    dino.dino_unload_surrogate(ctx, sid)
