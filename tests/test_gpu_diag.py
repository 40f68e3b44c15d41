"""Chain diagnostics on the device against the oracle (GPU).

* Samples pushed from the host (seeded AR(1) series with per-dof
  coefficients and, on some degrees of freedom, chain offsets that the
  between-chain term must catch): ESS% per degree of freedom, MSJ and the
  Wasserstein MPSRF agree with the oracle's on the same array.
* Trajectories recorded on the device from an FP64 pool (reduced
  coordinates and the field) while the oracle runs the same chains: the
  diagnostics of the two trajectories agree.
"""
import numpy as np
import pytest

from helpers import gpu_setup, oracle_chains, oracle_setup
from oracle import diagnostics as dg
from workloads import CONFIGS, SEED_CHAINS

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


def _ar1_samples(n_c, n_s, d, seed):
    rng = np.random.default_rng(seed)
    phi = rng.uniform(0.0, 0.9, d)
    X = np.empty((n_c, n_s, d))
    X[:, 0] = rng.standard_normal((n_c, d)) / np.sqrt(1 - phi ** 2)
    for j in range(1, n_s):
        X[:, j] = phi * X[:, j - 1] + rng.standard_normal((n_c, d))
    X[:, :, : d // 4] += 0.5 * rng.standard_normal((n_c, 1, d // 4))   # chains disagree here
    mix = np.linalg.qr(rng.standard_normal((d, d)))[0]                  # correlated dofs
    return X @ mix.T


@pytest.mark.parametrize("n_c,n_s,d", [(16, 300, 24), (64, 64, 200)])
def test_pushed_samples_match_oracle(dino, ctx, n_c, n_s, d):
    X = _ar1_samples(n_c, n_s, d, 5 + d)
    g = dino.dino_diag_create(ctx, n_c, d, n_s + 3)
    for j in range(n_s):
        dino.dino_diag_push(ctx, g, X[:, j, :])
    out = dino.dino_diag_compute(ctx, g, d, mpsrf=True)
    ess = dg.ess_fractions(X)
    W, V = dg.covariance_estimators(X)
    rw = dg.wasserstein_mpsrf(W, V)
    assert out["n_samples"] == n_s
    assert np.max(np.abs(out["ess"] - ess) / ess) <= 1e-9
    assert abs(out["ess_median"] - np.median(ess)) <= 1e-9 * np.median(ess)
    assert abs(out["msj"] - dg.mean_squared_jump(X)) <= 1e-12 * dg.mean_squared_jump(X)
    assert abs(out["trace_w"] - np.trace(W)) <= 1e-12 * np.trace(W)
    assert abs(out["trace_v"] - np.trace(V)) <= 1e-12 * np.trace(V)
    assert abs(out["mpsrf_w"] - rw) <= 1e-9 * np.trace(V)
    assert rw > 1e-3 * np.trace(V)              # the offsets make W and V differ
    dino.dino_diag_destroy(ctx, g)


def test_recorded_pool_trajectories_match_oracle(dino, ctx):
    w = CONFIGS["small_fp64"]
    sid = gpu_setup(dino, ctx, w)
    sur, E, D = oracle_setup(w)
    C, dt, n_s = 24, 0.002, 60
    pool = dino.dino_chains_create(ctx, sid, C, dt, SEED_CHAINS)
    och = oracle_chains(dino, ctx, sid, w, sur, E, D, C, dt)
    gr = dino.dino_diag_create(ctx, C, w.r, n_s)
    gf = dino.dino_diag_create(ctx, 8, w.N, n_s)        # the field of chains 4 .. 11
    Xr, Xf = [], []
    for _ in range(n_s):
        dino.dino_chains_step(ctx, pool, 1, stats=False)
        och.step()
        dino.dino_diag_record(ctx, gr, pool, dino.DINO_DIAG_REDUCED, 0)
        dino.dino_diag_record(ctx, gf, pool, dino.DINO_DIAG_FIELD, 4)
        Xr.append(och.m_r.copy())
        Xf.append(och.m[4:12].copy())
    Xr = np.stack(Xr, axis=1)
    Xf = np.stack(Xf, axis=1)
    r = dino.dino_diag_compute(ctx, gr, w.r, mpsrf=True)
    ess = dg.ess_fractions(Xr)
    assert np.max(np.abs(r["ess"] - ess) / ess) <= 1e-6
    W, V = dg.covariance_estimators(Xr)
    assert abs(r["mpsrf_w"] - dg.wasserstein_mpsrf(W, V)) <= 1e-8 * np.trace(V)
    assert abs(r["msj"] - dg.mean_squared_jump(Xr)) <= 1e-8 * dg.mean_squared_jump(Xr)
    f = dino.dino_diag_compute(ctx, gf, w.N, mpsrf=False)
    essf = dg.ess_fractions(Xf)
    assert np.max(np.abs(f["ess"] - essf) / essf) <= 1e-6
    assert np.isnan(f["mpsrf_w"])
    for g in (gr, gf):
        dino.dino_diag_destroy(ctx, g)
    dino.dino_chains_destroy(ctx, pool)
    dino.dino_unload_surrogate(ctx, sid)


def test_diag_errors(dino, ctx):
    g = dino.dino_diag_create(ctx, 4, 3, 2)
    with pytest.raises(dino.DinoError) as e:
        dino.dino_diag_compute(ctx, g, 3)
    assert e.value.code == dino.DINO_ESTATE
    dino.dino_diag_push(ctx, g, np.zeros((4, 3)))
    dino.dino_diag_push(ctx, g, np.ones((4, 3)))
    with pytest.raises(dino.DinoError) as e:
        dino.dino_diag_push(ctx, g, np.ones((4, 3)))
    assert e.value.code == dino.DINO_ENOMEM
    dino.dino_diag_destroy(ctx, g)
    with pytest.raises(dino.DinoError) as e:
        dino.dino_diag_create(ctx, 1, 3, 10)
    assert e.value.code == dino.DINO_EINVAL
    g = dino.dino_diag_create(ctx, 2, 1100, 3)
    for _ in range(2):
        dino.dino_diag_push(ctx, g, np.random.default_rng(0).standard_normal((2, 1100)))
    with pytest.raises(dino.DinoError) as e:
        dino.dino_diag_compute(ctx, g, 1100, mpsrf=True)
    assert e.value.code == dino.DINO_EINVAL
    dino.dino_diag_destroy(ctx, g)
