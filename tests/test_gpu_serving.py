"""Serving: continuous batching of chain ensembles of different size (GPU).

Each result must be the same alone and in a mix (bit-identical: the random
numbers are keyed by seed and chain id, and every kernel is deterministic);
admission must respect the HBM budget; errors come back as codes.
"""
import time

import numpy as np
import pytest

from helpers import gpu_setup, variant
from workloads import BASIS_DIS, CONFIGS, SEED_CHAINS

pytestmark = pytest.mark.gpu

SMALL = CONFIGS["small_fp64"]
MID = variant(CONFIGS["small_fp64"], n_grid=9, r=45, widths=[45, 33, 17, 20],
              basis_kind=BASIS_DIS, activation=2, noise_frac=0.2)
BF = variant(CONFIGS["r200_dis_bf16"])


@pytest.fixture(scope="module")
def dino():
    import paper_2403_08220_gb300 as d
    return d


def _solo(dino, w, C, steps, dt, seed, base=0):
    ctx = dino.dino_init(0)
    try:
        sid = gpu_setup(dino, ctx, w)
        t = dino.dino_serve_submit(ctx, sid, C, steps, dt, seed, w.r, w.N, base)
        return dino.dino_serve_wait(ctx, t, 300)
    finally:
        ctx.close()


def test_request_equals_direct_chains_and_is_the_same_in_a_mix(dino):
    C, steps, dt, seed = 37, 25, 0.002, 5
    solo = _solo(dino, SMALL, C, steps, dt, seed)
    # the same transitions through dino_chains_create / dino_chains_step
    ctx = dino.dino_init(0)
    sid = gpu_setup(dino, ctx, SMALL)
    pool = dino.dino_chains_create(ctx, sid, C, dt, seed)
    dino.dino_chains_step(ctx, pool, steps, stats=False)
    direct = dino.dino_chains_read(ctx, pool, C, SMALL.r, SMALL.N, field=False)
    ctx.close()
    assert np.array_equal(solo["m_r"], direct["m_r"])
    assert np.array_equal(solo["phi"], direct["phi"])
    assert np.array_equal(solo["accepts"], direct["accepts"])
    assert solo["stats"]["accepts"] == int(direct["accepts"].sum())

    # now in a mix of different sizes, precisions and surrogates
    ctx = dino.dino_init(0)
    try:
        dino.dino_serve_config(ctx, n_streams=3, steps_per_round=4, max_active=8)
        s_small = gpu_setup(dino, ctx, SMALL)
        s_mid = gpu_setup(dino, ctx, MID)
        s_bf = gpu_setup(dino, ctx, BF)
        tickets = [
            dino.dino_serve_submit(ctx, s_bf, 700, 6, 0.5, 1, BF.r, BF.N),
            dino.dino_serve_submit(ctx, s_mid, 300, 40, 0.01, 2, MID.r, MID.N),
            dino.dino_serve_submit(ctx, s_small, C, steps, dt, seed, SMALL.r, SMALL.N),
            dino.dino_serve_submit(ctx, s_small, 500, 15, 0.002, 3, SMALL.r, SMALL.N),
            dino.dino_serve_submit(ctx, s_bf, 130, 9, 2e-5, 4, BF.r, BF.N),
        ]
        outs = [dino.dino_serve_wait(ctx, t, 300) for t in tickets]
        mix = outs[2]
        assert np.array_equal(mix["m_r"], solo["m_r"])
        assert np.array_equal(mix["phi"], solo["phi"])
        assert np.array_equal(mix["accepts"], solo["accepts"])
        for o in outs:
            assert o["latency_s"] >= o["queue_s"] >= 0
            assert np.all(np.isfinite(o["phi"]))
        st = dino.dino_serve_status(ctx)
        assert st["queued"] == 0 and st["active"] == 0 and st["peak_active"] >= 2
    finally:
        ctx.close()


def test_admission_respects_the_hbm_budget(dino):
    C, steps = 64, 30
    probe = dino.dino_init(0)
    sid = gpu_setup(dino, probe, SMALL)
    base = dino.dino_serve_status(probe)["hbm_used"]
    pool = dino.dino_chains_create(probe, sid, C, 0.002, 1)
    fp = dino.dino_serve_status(probe)["hbm_used"] - base
    probe.close()
    # room for the surrogate and one and a half pools: requests must take turns
    ctx = dino.dino_init(0, hbm_budget_bytes=int(base + 1.5 * fp))
    try:
        sid = gpu_setup(dino, ctx, SMALL)
        ts = [dino.dino_serve_submit(ctx, sid, C, steps, 0.002, 10 + k, SMALL.r, SMALL.N)
              for k in range(3)]
        outs = [dino.dino_serve_wait(ctx, t, 300) for t in ts]
        st = dino.dino_serve_status(ctx)
        assert st["peak_active"] == 1
        assert st["peak_hbm_used"] <= base + 1.5 * fp
        q = [o["queue_s"] for o in outs]
        assert q[0] <= q[1] <= q[2]
        # a request larger than the whole budget is refused at submit
        with pytest.raises(dino.DinoError) as e:
            dino.dino_serve_submit(ctx, sid, 100 * C, 1, 0.1, 1, SMALL.r, SMALL.N)
        assert e.value.code == dino.DINO_ENOMEM
    finally:
        ctx.close()


def test_serving_errors(dino):
    ctx = dino.dino_init(0)
    try:
        with pytest.raises(dino.DinoError) as e:
            dino.dino_serve_submit(ctx, 424242, 4, 1, 0.1, 1, 16, 1089)
        assert e.value.code == dino.DINO_ENOTFOUND
        sid = gpu_setup(dino, ctx, SMALL)
        with pytest.raises(dino.DinoError) as e:
            dino.dino_serve_submit(ctx, sid, 4, 1, -0.1, 1, SMALL.r, SMALL.N)
        assert e.value.code == dino.DINO_EINVAL
        with pytest.raises(dino.DinoError) as e:
            dino.dino_serve_poll(ctx, 99999)
        assert e.value.code == dino.DINO_ENOTFOUND
        t0 = time.perf_counter()
        t = dino.dino_serve_submit(ctx, sid, 4, 2, 0.1, 1, SMALL.r, SMALL.N)
        out = dino.dino_serve_wait(ctx, t, 60)
        elapsed = time.perf_counter() - t0
        assert out["stats"]["proposals"] == 8
        assert 0.0 <= out["queue_s"] <= out["latency_s"] <= elapsed + 1e-3
        with pytest.raises(dino.DinoError) as e:
            dino.dino_serve_config(ctx, 2, 2, 2)
        assert e.value.code == dino.DINO_ESTATE
    finally:
        ctx.close()
