"""Parity of the tensor-core (tcgen05, BF16 slices) path with the FP64 oracle (GPU).

Bars (stated for the BF16 path):
  Jacobian       |J - J64|_F / |J64|_F <= 2e-2 per chain (1e-4 with the 2-slice default)
  proposal mean  |mu - mu64|_2 / |mu64|_2 <= 1e-3 from the same state
  forward        f with 3 slices: FP32-level, |f - f64| <= 1e-4 max(1, |f64|)
                 (FP32 accumulation over K = 400 per layer: K u = 2.4e-5, three layers)
  log rho        |log rho - log rho64| <= 1e-3 x (sum of |terms| of log rho).  The
                 Jacobian's FP32-level error (1e-5) is amplified by the cancellation
                 inside the rho_0 terms (w = H m - g with |H m| >> |w|): measured
                 3e-7 of the scale in the mixing runs and 1.3e-4 at dt = 0.5, where
                 chains sit far from the posterior and log rho is about -1e5.
  accept         under shared uniforms a decision may differ from the FP64 one
                 only when log u lies between the two log rho values (or within
                 1e-3 of the FP64 threshold); the flipped fraction is bounded.
The Cholesky factor and its log-determinant are computed in double-float
arithmetic (a 48-bit significand on the FP32 pipe) and log rho in FP64 from
the BF16/FP32 Jacobian, so their error is the Jacobian's, propagated; the
factorisation itself is pinned to FP64 on an exactly representable Hessian
(`test_double_float_cholesky_on_exact_hessian`).
"""
import numpy as np
import pytest

from helpers import gpu_setup, oracle_setup, rel_err, variant
from oracle import mmala
from oracle.chains import OracleChains
from workloads import ACT_IDENTITY, BASIS_DIS, BASIS_KLE, CONFIGS, SEED_CHAINS

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


def _jac_rel(J, J64):
    return np.linalg.norm(J - J64, axis=(-2, -1)) / np.linalg.norm(J64, axis=(-2, -1))


SMALL = variant(CONFIGS["small_fp64"], precision="bf16")


@pytest.mark.parametrize("fs,js,jtol", [(1, 1, 2e-2), (3, 2, 1e-4), (3, 3, 1e-5)])
def test_tensor_core_forward_and_jacobian_small(dino, ctx, fs, js, jtol):
    """16-64-64-49 tanh network, 130 points (a ragged 128-row tile)."""
    sid = gpu_setup(dino, ctx, SMALL, fwd_slices=fs, jac_slices=js)
    sur, _, _ = oracle_setup(SMALL)
    x = np.random.default_rng(5).standard_normal((130, SMALL.r))
    g = dino.dino_surrogate_eval(ctx, sid, x, SMALL.d_y)
    o = mmala.geometry(sur, x)
    assert _jac_rel(g["J"], o.J).max() <= jtol
    ftol = {1: 3e-2, 2: 1e-4, 3: 1e-4}[fs]
    assert rel_err(g["f"], o.f) <= ftol
    dino.dino_unload_surrogate(ctx, sid)


def test_tensor_core_geometry_r200(dino, ctx):
    """r = 200 DIS, GELU 200-400-400-100: default slices (3 forward, 2 Jacobian)."""
    w = CONFIGS["r200_dis_bf16"]
    sid = gpu_setup(dino, ctx, w)
    sur, _, _ = oracle_setup(w)
    x = np.random.default_rng(6).standard_normal((33, w.r))
    g = dino.dino_surrogate_eval(ctx, sid, x, w.d_y)
    o = mmala.geometry(sur, x)
    assert _jac_rel(g["J"], o.J).max() <= 1e-4
    assert rel_err(g["f"], o.f) <= 1e-4
    # geometry in FP64 from the FP32 Jacobian: relative errors of the same order
    assert np.max(np.abs(g["phi"] - o.phi) / np.abs(o.phi)) <= 1e-4
    assert np.max(np.abs(g["hld"] - o.hld) / np.abs(o.hld)) <= 1e-4
    dino.dino_unload_surrogate(ctx, sid)


def _precision_run(dino, ctx, w, C, dt, steps, sample=None, fs=0, js=0):
    sid = gpu_setup(dino, ctx, w, fwd_slices=fs, jac_slices=js)
    sur, E, D = oracle_setup(w)
    ids = np.arange(C) if sample is None else np.asarray(sample)
    pool = dino.dino_chains_create(ctx, sid, C, dt, SEED_CHAINS)
    och = OracleChains(sur, E, D, w.n_grid, w.prior_gamma, w.prior_delta, len(ids), dt,
                       seed=SEED_CHAINS, chain_ids=ids)
    st0 = dino.dino_chains_read(ctx, pool, C, w.r, w.N)
    assert rel_err(st0["m_r"][ids], och.m_r) <= 1e-12          # FP64 encode at init
    out = dict(mu=[], dec_bad=0, dec_flip=0, n=0, log_rho=[], log_rho_rel=[])
    active = np.ones(len(ids), dtype=bool)
    for _ in range(steps):
        dino.dino_chains_step(ctx, pool, 1, stats=False)
        och.step()
        last = dino.dino_chains_read_last(ctx, pool, C, w.r)
        o = och.last
        a = active
        mu_g = last["mu"][ids][a]
        out["mu"].append(np.max(np.linalg.norm(mu_g - o["mu"][a], axis=1) /
                                np.linalg.norm(o["mu"][a], axis=1)))
        lr64 = o["log_rho"][a]
        lrg = last["log_rho"][ids][a]
        dlr = np.abs(lrg - lr64)
        # a flip is explained when log u lies between the two log rho values
        straddle = np.abs(o["log_u"][a] - np.minimum(0.0, lr64)) < dlr + 1e-3
        agree = last["accepted"][ids][a] == o["accepted"][a]
        out["dec_bad"] += int(np.sum(~agree & ~straddle))
        out["dec_flip"] += int(np.sum(~agree))
        out["n"] += int(a.sum())
        fin = np.isfinite(lr64)
        out["log_rho"].append(np.max(dlr[fin], initial=0))
        out["log_rho_rel"].append(np.max(dlr[fin] / np.maximum(1.0, o["log_rho_scale"][a][fin]),
                                         initial=0))
        # only chains that took the same decision stay comparable from the same state
        sub = np.where(a)[0]
        active[sub[~agree]] = False
    st = dino.dino_chains_read(ctx, pool, C, w.r, w.N)
    out["field"] = float(np.max(np.abs(st["m"][ids][active] - och.m[active]), initial=0))
    dino.dino_chains_destroy(ctx, pool)
    dino.dino_unload_surrogate(ctx, sid)
    return out


def _check_bars(out):
    assert max(out["mu"]) <= 1e-3
    assert max(out["log_rho_rel"]) <= 1e-3
    assert out["dec_bad"] == 0
    assert out["dec_flip"] <= max(1, 0.02 * out["n"])
    assert out["field"] <= 1e-4


@pytest.mark.parametrize("dt", [0.5, 2e-5])
def test_bf16_chains_meet_precision_bars(dino, ctx, dt):
    """r = 200 DIS workload, 130 chains: mean error, log rho, decisions, field (FP32)."""
    w = CONFIGS["r200_dis_bf16"]
    out = _precision_run(dino, ctx, w, 130, dt, 3)
    _check_bars(out)


def test_bf16_small_config_mixing(dino, ctx):
    """The small workload on the tensor path with dt = 0.002 (about a third accepted)."""
    out = _precision_run(dino, ctx, SMALL, 64, 0.002, 20)
    _check_bars(out)


def test_bf16_full_size_sampled(dino, ctx):
    """16384 chains at r = 200 (the BF16 workload's launch shape); 8 chains checked."""
    w = CONFIGS["r200_dis_bf16"]
    C = w.n_chains
    sample = [0, 1, 127, 128, 5000, 9999, 16000, C - 1]
    out = _precision_run(dino, ctx, w, C, w.dt, 2, sample=sample)
    _check_bars(out)


@pytest.mark.parametrize("r,h,dy", [(45, 24, 12), (200, 64, 50), (256, 48, 40)])
def test_double_float_cholesky_on_exact_hessian(dino, ctx, r, h, dy):
    """Weights in {-1, 0, 1} and the identity activation make the tensor-core
    Jacobian J = W2 W1 exact (small integers), so I + J^T J (noise variance 1)
    is exact in FP32 and the double-float factor must agree with an FP64
    Cholesky to 1e-10 of max |L| (an FP32 factorisation of the same matrix
    misses by about 4e-8).  r = 256 runs with the factor in its global slot."""
    rng = np.random.default_rng(21)
    W1 = rng.integers(-1, 2, size=(h, r)).astype(float)
    W2 = rng.integers(-1, 2, size=(dy, h)).astype(float)
    n = int(np.ceil(np.sqrt(r))) + 1
    sid = dino.dino_load_surrogate(
        ctx, n_grid=n, prior_gamma=0.1, prior_delta=1.0, r=r, widths=[r, h, dy],
        activation=ACT_IDENTITY, W=[W1, W2], b=[np.zeros(h), np.zeros(dy)],
        basis_kind=BASIS_KLE, y=np.zeros(dy), noise_var=1.0, precision=dino.DINO_PREC_BF16)
    x = rng.standard_normal((3, r))
    g = dino.dino_surrogate_eval(ctx, sid, x, dy)
    J = W2 @ W1
    L = np.linalg.cholesky(np.eye(r) + J.T @ J)
    hld = np.log(np.diag(L)).sum()
    for c in range(3):
        assert np.array_equal(g["J"][c], J)
        assert np.abs(g["L"][c] - L).max() <= 1e-10 * np.abs(L).max()
        assert abs(g["hld"][c] - hld) <= 1e-10 * abs(hld)
        assert rel_err(g["g"][c], J.T @ g["f"][c]) <= 1e-12
    dino.dino_unload_surrogate(ctx, sid)


@pytest.mark.gpu
def test_host_field_read_in_place_matches_copy(dino):
    """A pool created from a host m0 gives the same chains whether the field-init
    kernel reads m0 in place (devices that read pageable host memory) or from a
    device copy (DINO_FLAG_NO_DIRECT_HOST), and its initial m_r is E m0 (FP64)."""
    w = variant(CONFIGS["r200_dis_bf16"], n_chains=96)
    rng = np.random.default_rng(31)
    m0 = 0.05 * rng.standard_normal((w.n_chains, w.N))
    out = []
    for flags in (0, dino.DINO_FLAG_NO_DIRECT_HOST):
        c = dino.dino_init(0, 0, None, flags)
        try:
            sid = gpu_setup(dino, c, w)
            E, _ = dino.dino_read_basis(c, sid, w.r, w.N)
            pool = dino.dino_chains_create(c, sid, w.n_chains, 2e-5, SEED_CHAINS, 0, m0)
            first = dino.dino_chains_read(c, pool, w.n_chains, w.r, w.N, field=False)
            dino.dino_chains_step(c, pool, 2)
            last = dino.dino_chains_read(c, pool, w.n_chains, w.r, w.N, field=True)
            out.append((first, last))
        finally:
            c.close()
    ref = m0 @ E.T
    assert rel_err(out[0][0]["m_r"], ref) <= 1e-10
    assert np.array_equal(out[0][0]["m_r"], out[1][0]["m_r"])
    for k in ("m_r", "phi", "accepts", "m"):
        assert np.array_equal(out[0][1][k], out[1][1][k]), k
