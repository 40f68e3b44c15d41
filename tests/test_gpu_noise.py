"""Caller-supplied noise, the accept rule at its threshold and non-finite log
rho (GPU).

dino_chains_set_noise feeds the next transition's normals and accept uniform
from the host, so the CUDA path and the oracle can be driven with the same
arbitrary (not Philox) draws, including adversarial ones:
  * parity with the oracle under numpy-drawn noise, for both noise maps;
  * log u placed exactly at min(0, log rho): Algorithm 1 rejects only when
    alpha < u, so equality accepts, and the next double above rejects;
  * NaN reduced noise: log rho is not finite, the proposal is rejected and
    counted in nan_rejects, and the chain state is unchanged.
"""
import numpy as np
import pytest

from helpers import gpu_setup, oracle_chains, oracle_setup, rel_err, variant
from workloads import BASIS_DIS, CONFIGS, SEED_CHAINS

pytestmark = pytest.mark.gpu

TOL = 1e-10
SMALL = CONFIGS["small_fp64"]                                   # Cholesky map
PERT = variant(CONFIGS["small_fp64"], n_grid=9, r=45, widths=[45, 33, 17, 20],
               basis_kind=BASIS_DIS, activation=2, noise_frac=0.2)   # perturbation map


@pytest.fixture(scope="module")
def dino():
    import paper_2403_08220_gb300 as d
    return d


@pytest.fixture(scope="module")
def ctx(dino):
    c = dino.dino_init(0)
    yield c
    c.close()


def _noise(rng, C, w, pert):
    return dict(xi=rng.standard_normal((C, w.r)),
                xi2=rng.standard_normal((C, w.d_y)) if pert else None,
                z=rng.standard_normal((C, w.N)),
                log_u=np.log(rng.uniform(size=C)))


@pytest.mark.parametrize("w,dt", [(SMALL, 0.002), (PERT, 0.01)], ids=["cholesky", "perturbation"])
def test_caller_noise_matches_oracle(dino, ctx, w, dt):
    sid = gpu_setup(dino, ctx, w)
    sur, E, D = oracle_setup(w)
    C = 24
    pool = dino.dino_chains_create(ctx, sid, C, dt, SEED_CHAINS)
    och = oracle_chains(dino, ctx, sid, w, sur, E, D, C, dt)
    pert = och.noise == "perturbation"
    assert pert == (w is PERT)
    rng = np.random.default_rng(101)
    for step in range(4):
        nz = _noise(rng, C, w, pert)
        dino.dino_chains_set_noise(ctx, pool, **nz)
        dino.dino_chains_step(ctx, pool, 1, stats=False)
        och.step(noise=nz)
        last = dino.dino_chains_read_last(ctx, pool, C, w.r)
        st = dino.dino_chains_read(ctx, pool, C, w.r, w.N)
        assert np.array_equal(last["log_u"], nz["log_u"])
        assert rel_err(last["b"], och.last["b"]) <= TOL
        scale = np.maximum(1.0, och.last["log_rho_scale"])
        assert np.all(np.abs(last["log_rho"] - och.last["log_rho"]) <= TOL * scale)
        assert np.array_equal(last["accepted"], och.last["accepted"])
        assert rel_err(st["m_r"], och.m_r) <= TOL
        assert rel_err(st["m"], och.m) <= TOL
    # the noise is one-shot: the next step draws Philox again, like the oracle
    dino.dino_chains_step(ctx, pool, 1, stats=False)
    och.step()
    assert rel_err(dino.dino_chains_read_last(ctx, pool, C, w.r)["b"], och.last["b"]) <= TOL
    dino.dino_chains_destroy(ctx, pool)
    dino.dino_unload_surrogate(ctx, sid)


def test_log_u_at_the_threshold_accepts(dino, ctx):
    """Three pools in the same state draw the same proposals; the accept
    uniform is placed at min(0, log rho) and one double above it."""
    w = SMALL
    sid = gpu_setup(dino, ctx, w)
    sur, E, D = oracle_setup(w)
    C, dt = 32, 0.002
    rng = np.random.default_rng(7)
    nz = _noise(rng, C, w, False)
    pools = [dino.dino_chains_create(ctx, sid, C, dt, SEED_CHAINS) for _ in range(3)]
    dino.dino_chains_set_noise(ctx, pools[0], **nz)
    dino.dino_chains_step(ctx, pools[0], 1, stats=False)
    lr = dino.dino_chains_read_last(ctx, pools[0], C, w.r)["log_rho"]
    assert np.all(np.isfinite(lr))
    thr = np.minimum(0.0, lr)
    cases = [(pools[1], thr, True), (pools[2], np.nextafter(thr, np.inf), False)]
    och0 = oracle_chains(dino, ctx, sid, w, sur, E, D, C, dt)
    och0.step(noise=nz)
    othr = np.minimum(0.0, och0.last["log_rho"])
    for (pool, log_u, accept), olog_u in zip(cases, (othr, np.nextafter(othr, np.inf))):
        dino.dino_chains_set_noise(ctx, pool, **{**nz, "log_u": log_u})
        st = dino.dino_chains_step(ctx, pool, 1)
        last = dino.dino_chains_read_last(ctx, pool, C, w.r)
        assert np.array_equal(last["log_rho"], lr)           # same state, same noise
        assert last["accepted"].all() == accept and (~last["accepted"]).all() == (not accept)
        assert st["accepts"] == (C if accept else 0)
        och = oracle_chains(dino, ctx, sid, w, sur, E, D, C, dt)
        och.step(noise={**nz, "log_u": olog_u})
        assert np.array_equal(och.last["accepted"], last["accepted"])
    for p in pools:
        dino.dino_chains_destroy(ctx, p)
    dino.dino_unload_surrogate(ctx, sid)


@pytest.mark.parametrize("w", [SMALL, variant(CONFIGS["r200_dis_bf16"], n_chains=40)],
                         ids=["fp64", "bf16"])
def test_nan_noise_is_a_counted_reject(dino, ctx, w):
    sid = gpu_setup(dino, ctx, w)
    C, dt = 12, 2e-5 if w.r == 200 else 0.002
    pool = dino.dino_chains_create(ctx, sid, C, dt, SEED_CHAINS)
    before = dino.dino_chains_read(ctx, pool, C, w.r, w.N)
    xi = np.random.default_rng(3).standard_normal((C, w.r))
    bad = [1, 5, 11]
    xi[bad, 0] = np.nan
    dino.dino_chains_set_noise(ctx, pool, xi=xi)
    st = dino.dino_chains_step(ctx, pool, 1)
    last = dino.dino_chains_read_last(ctx, pool, C, w.r)
    after = dino.dino_chains_read(ctx, pool, C, w.r, w.N)
    assert st["nan_rejects"] == len(bad) and st["proposals"] == C
    assert not np.isfinite(last["log_rho"][bad]).any() and not last["accepted"][bad].any()
    good = np.setdiff1d(np.arange(C), bad)
    assert np.isfinite(last["log_rho"][good]).all()
    for k in ("m_r", "phi", "m"):
        assert np.array_equal(after[k][bad], before[k][bad]), k
    assert np.isfinite(st["sum_alpha"])
    # the pool goes on normally afterwards
    st2 = dino.dino_chains_step(ctx, pool, 2)
    assert st2["nan_rejects"] == 0
    dino.dino_chains_destroy(ctx, pool)
    dino.dino_unload_surrogate(ctx, sid)


def test_set_noise_errors(dino, ctx):
    sid = gpu_setup(dino, ctx, SMALL)
    pool = dino.dino_chains_create(ctx, sid, 4, 0.1, 1)
    with pytest.raises(dino.DinoError) as e:      # xi2 on a Cholesky-map pool
        dino.dino_chains_set_noise(ctx, pool, xi2=np.zeros((4, SMALL.d_y)))
    assert e.value.code == dino.DINO_EINVAL
    with pytest.raises(dino.DinoError) as e:
        dino.dino_chains_set_noise(ctx, 987654, xi=np.zeros((4, SMALL.r)))
    assert e.value.code == dino.DINO_ENOTFOUND
    with pytest.raises(dino.DinoError) as e:      # a map that does not apply
        gpu_setup(dino, ctx, variant(SMALL, noise_map="perturbation"))
    assert e.value.code == dino.DINO_EINVAL
    dino.dino_chains_destroy(ctx, pool)
    dino.dino_unload_surrogate(ctx, sid)
