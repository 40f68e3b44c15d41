"""Several pools stepped concurrently, and the measured FP32 peak (GPU).

dino_chains_step_many runs each pool on its own stream; the chains must be
bit-identical to stepping each pool alone (the random numbers are keyed by
seed and chain id, and every kernel is deterministic).
"""
import numpy as np
import pytest

from helpers import gpu_setup, variant
from workloads import BASIS_DIS, CONFIGS, heterogeneous_workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dino():
    import paper_2403_08220_gb300 as d
    return d


def _shapes():
    hw = heterogeneous_workloads()
    return [(variant(hw[0], n_chains=96), 0.5), (variant(hw[2], n_chains=40), 1e-3),
            (variant(CONFIGS["r200_dis_bf16"], n_chains=64), 2e-5),
            (variant(CONFIGS["small_fp64"], n_chains=50), 0.002)]


def test_step_many_equals_separate_steps(dino):
    outs = []
    for together in (False, True):
        ctx = dino.dino_init(0)
        try:
            pools = []
            for w, dt in _shapes():
                sid = gpu_setup(dino, ctx, w)
                pools.append((w, dino.dino_chains_create(ctx, sid, w.n_chains, dt, 15)))
            if together:
                dino.dino_chains_step_many(ctx, [p for _, p in pools], 4)
            else:
                for _, p in pools:
                    dino.dino_chains_step(ctx, p, 4, stats=False)
            outs.append([dino.dino_chains_read(ctx, p, w.n_chains, w.r, w.N) for w, p in pools])
            with pytest.raises(dino.DinoError) as e:
                dino.dino_chains_step_many(ctx, [pools[0][1], pools[0][1]], 1)
            assert e.value.code == dino.DINO_EINVAL
        finally:
            ctx.close()
    for a, b in zip(*outs):
        for k in ("m_r", "phi", "accepts", "m"):
            assert np.array_equal(a[k], b[k]), k


def test_measured_fp32_peak_is_plausible(dino):
    ctx = dino.dino_init(0)
    try:
        t = dino.dino_measure_fp32_peak(ctx)
    finally:
        ctx.close()
    # 152 SMs x 128 lanes x ~2 GHz x 2 flops = ~80 TFLOP/s at the maximum clock
    assert 20.0 < t < 100.0, t
