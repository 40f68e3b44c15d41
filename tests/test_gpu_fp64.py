"""Parity of the FP64 CUDA path with the FP64 oracle (GPU).

Bar: every compared quantity within 1e-10 relative (|a - b| <= 1e-10
max(1, |b|)), accept decisions identical except within 1e-8 of the threshold.
"""
import numpy as np
import pytest

from helpers import (gpu_setup, oracle_chains, oracle_setup, rel_err, step_and_compare,
                     variant)
from oracle import mmala, prior
from oracle.chains import OracleChains
from workloads import (ACT_GELU, ACT_IDENTITY, ACT_TANH, BASIS_DIS, BASIS_KLE, CONFIGS,
                       SEED_CHAINS, surrogate_inputs)

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def dino():
    import paper_2403_08220_gb300 as d
    return d


@pytest.fixture(scope="module")
def ctx(dino):
    c = dino.dino_init(0)
    yield c
    c.close()


def _oracle_chains(dino, ctx, sid, w, sur, E, D, C, dt, ids=None):
    return oracle_chains(dino, ctx, sid, w, sur, E, D, C, dt, chain_ids=ids)


@pytest.mark.parametrize("kind", [BASIS_KLE, BASIS_DIS])
def test_basis_matches_oracle(dino, ctx, kind):
    w = variant(CONFIGS["small_fp64"], basis_kind=kind, n_grid=9 if kind == BASIS_DIS else 33,
                r=5 if kind == BASIS_DIS else 16,
                widths=[5, 8, 3] if kind == BASIS_DIS else [16, 64, 64, 49])
    sid = gpu_setup(dino, ctx, w)
    E, D = dino.dino_read_basis(ctx, sid, w.r, w.N)
    _, Eo, Do = oracle_setup(w)
    assert np.abs(E - Eo).max() <= 1e-12 * np.abs(Eo).max()
    assert np.abs(D - Do).max() <= 1e-12 * np.abs(Do).max()
    dino.dino_unload_surrogate(ctx, sid)


@pytest.mark.parametrize("name", ["small_fp64", "r200_kle_fp64"])
def test_surrogate_geometry_matches_oracle(dino, ctx, name):
    w = CONFIGS[name]
    sid = gpu_setup(dino, ctx, w)
    sur, _, _ = oracle_setup(w)
    x = np.random.default_rng(3).standard_normal((5, w.r))
    g = dino.dino_surrogate_eval(ctx, sid, x, w.d_y)
    o = mmala.geometry(sur, x)
    for k, ref in [("f", o.f), ("J", o.J), ("phi", o.phi), ("g", o.g), ("L", o.L),
                   ("hld", o.hld)]:
        assert rel_err(g[k], ref) <= TOL, k
    dino.dino_unload_surrogate(ctx, sid)


@pytest.mark.parametrize("dt,steps", [(0.5, 200), (0.002, 200)])
def test_chains_small_config_match_oracle(dino, ctx, dt, steps):
    """64 chains, n=33, r=16, tanh 16-64-64-49 (dt=0.5 as configured; dt=0.002 mixes)."""
    w = CONFIGS["small_fp64"]
    sid = gpu_setup(dino, ctx, w)
    sur, E, D = oracle_setup(w)
    pool = dino.dino_chains_create(ctx, sid, w.n_chains, dt, SEED_CHAINS)
    st = dino.dino_chains_read(ctx, pool, w.n_chains, w.r, w.N)
    och = _oracle_chains(dino, ctx, sid, w, sur, E, D, w.n_chains, dt)
    assert rel_err(st["m"], och.m) <= TOL
    assert rel_err(st["m_r"], och.m_r) <= TOL
    assert rel_err(st["phi"], och.geo.phi) <= TOL
    acc, worst, active = step_and_compare(dino, ctx, pool, och, w, w.n_chains, steps, tol=TOL)
    if dt < 0.01:
        assert 0.1 < np.mean(acc) < 0.9          # the mixing case really moves
    assert active.mean() > 0.9
    dino.dino_chains_destroy(ctx, pool)
    dino.dino_unload_surrogate(ctx, sid)


@pytest.mark.parametrize("dt", [0.5, 2e-5])
def test_chains_r200_match_oracle(dino, ctx, dt):
    """r = 200 KLE, GELU 200-400-400-100 on the 65 x 65 grid: 6 chains x 3 steps."""
    w = CONFIGS["r200_kle_fp64"]
    C = 6
    sid = gpu_setup(dino, ctx, w)
    sur, E, D = oracle_setup(w)
    pool = dino.dino_chains_create(ctx, sid, C, dt, SEED_CHAINS)
    och = _oracle_chains(dino, ctx, sid, w, sur, E, D, C, dt)
    step_and_compare(dino, ctx, pool, och, w, C, 3, tol=TOL)
    dino.dino_chains_destroy(ctx, pool)
    dino.dino_unload_surrogate(ctx, sid)


def test_full_size_fp64_sampled_chains(dino, ctx):
    """4096 chains at r = 200 (the FP64 workload's launch shape); 6 chains checked."""
    w = CONFIGS["r200_kle_fp64"]
    C = w.n_chains
    sample = [0, 1, 777, 2048, 4000, C - 1]
    sid = gpu_setup(dino, ctx, w)
    sur, E, D = oracle_setup(w)
    pool = dino.dino_chains_create(ctx, sid, C, w.dt, SEED_CHAINS)
    och = _oracle_chains(dino, ctx, sid, w, sur, E, D, len(sample), w.dt, ids=sample)
    step_and_compare(dino, ctx, pool, och, w, C, 2, tol=TOL, sample=sample)
    dino.dino_chains_destroy(ctx, pool)
    dino.dino_unload_surrogate(ctx, sid)


def test_ragged_sizes_and_single_chain(dino, ctx):
    """r not a multiple of 32, d_y = 1, one chain, DIS basis, 2 hidden layers of odd width."""
    w = variant(CONFIGS["small_fp64"], n_grid=9, r=45, widths=[45, 33, 17, 1],
                basis_kind=BASIS_DIS, activation=ACT_GELU, noise_frac=0.2)
    sid = gpu_setup(dino, ctx, w)
    sur, E, D = oracle_setup(w)
    for C, dt in [(1, 0.05), (37, 0.01)]:
        pool = dino.dino_chains_create(ctx, sid, C, dt, SEED_CHAINS)
        och = _oracle_chains(dino, ctx, sid, w, sur, E, D, C, dt)
        step_and_compare(dino, ctx, pool, och, w, C, 5, tol=TOL)
        dino.dino_chains_destroy(ctx, pool)
    dino.dino_unload_surrogate(ctx, sid)


def test_linear_surrogate_accepts_everything(dino, ctx):
    """Identity activation: log rho == 0 (linear Gaussian target), every proposal accepted."""
    w = variant(CONFIGS["small_fp64"], activation=ACT_IDENTITY, widths=[16, 20, 12])
    sid = gpu_setup(dino, ctx, w)
    C = 50
    pool = dino.dino_chains_create(ctx, sid, C, 0.5, SEED_CHAINS)
    st = dino.dino_chains_step(ctx, pool, 10)
    last = dino.dino_chains_read_last(ctx, pool, C, w.r)
    assert np.abs(last["log_rho"]).max() < 1e-8
    assert st["accepts"] == C * 10 and st["nan_rejects"] == 0
    dino.dino_chains_destroy(ctx, pool)
    dino.dino_unload_surrogate(ctx, sid)


def test_single_layer_surrogate(dino, ctx):
    """One affine layer: J is the weight matrix itself (no Jacobian GEMM)."""
    w = variant(CONFIGS["small_fp64"], activation=ACT_TANH, widths=[16, 9])
    sid = gpu_setup(dino, ctx, w)
    sur, E, D = oracle_setup(w)
    pool = dino.dino_chains_create(ctx, sid, 8, 0.3, SEED_CHAINS)
    och = _oracle_chains(dino, ctx, sid, w, sur, E, D, 8, 0.3)
    step_and_compare(dino, ctx, pool, och, w, 8, 4, tol=TOL)
    dino.dino_chains_destroy(ctx, pool)
    dino.dino_unload_surrogate(ctx, sid)


def test_given_initial_field(dino, ctx):
    w = CONFIGS["small_fp64"]
    sid = gpu_setup(dino, ctx, w)
    sur, E, D = oracle_setup(w)
    C = 5
    m0 = prior.prior_sample(w.n_grid, w.prior_gamma, w.prior_delta,
                            np.random.default_rng(9).standard_normal((C, w.N)))
    pool = dino.dino_chains_create(ctx, sid, C, 0.002, SEED_CHAINS, 0, m0)
    och = oracle_chains(dino, ctx, sid, w, sur, E, D, C, 0.002, m0=m0)
    step_and_compare(dino, ctx, pool, och, w, C, 10, tol=TOL)
    dino.dino_chains_destroy(ctx, pool)
    dino.dino_unload_surrogate(ctx, sid)


def test_chain_ids_make_results_independent_of_grouping(dino, ctx):
    """Chains 0..9 in one pool equal chains 0..4 and 5..9 in two pools (counter-keyed RNG)."""
    w = CONFIGS["small_fp64"]
    sid = gpu_setup(dino, ctx, w)
    pa = dino.dino_chains_create(ctx, sid, 10, 0.002, 77)
    pb = dino.dino_chains_create(ctx, sid, 5, 0.002, 77, 0)
    pc = dino.dino_chains_create(ctx, sid, 5, 0.002, 77, 5)
    for p in (pa, pb, pc):
        dino.dino_chains_step(ctx, p, 20, stats=False)
    A = dino.dino_chains_read(ctx, pa, 10, w.r, w.N)
    B = dino.dino_chains_read(ctx, pb, 5, w.r, w.N)
    Cc = dino.dino_chains_read(ctx, pc, 5, w.r, w.N)
    assert np.array_equal(A["m_r"], np.concatenate([B["m_r"], Cc["m_r"]]))
    assert np.array_equal(A["m"], np.concatenate([B["m"], Cc["m"]]))
    for p in (pa, pb, pc):
        dino.dino_chains_destroy(ctx, p)
    dino.dino_unload_surrogate(ctx, sid)


def test_error_codes(dino, ctx):
    w = CONFIGS["small_fp64"]
    inp = surrogate_inputs(w)
    with pytest.raises(dino.DinoError) as e:
        dino.dino_load_surrogate(ctx, n_grid=3, prior_gamma=0.1, prior_delta=1.0, r=16,
                                 widths=w.widths, activation=w.activation, W=inp["Ws"],
                                 b=inp["bs"], basis_kind=BASIS_KLE)
    assert e.value.code == dino.DINO_EINVAL            # r > N
    sid = gpu_setup(dino, ctx, w)
    with pytest.raises(dino.DinoError) as e:
        dino.dino_chains_create(ctx, sid, 4, 0.0, 1)
    assert e.value.code == dino.DINO_EINVAL            # dt <= 0
    with pytest.raises(dino.DinoError) as e:
        dino.dino_chains_step(ctx, 987654, 1)
    assert e.value.code == dino.DINO_ENOTFOUND
    pool = dino.dino_chains_create(ctx, sid, 4, 0.1, 1)
    with pytest.raises(dino.DinoError) as e:
        dino.dino_set_data(ctx, sid, np.zeros(w.d_y), 1.0)
    assert e.value.code == dino.DINO_ESTATE            # data change under live pools
    with pytest.raises(dino.DinoError) as e:
        dino.dino_chains_create(ctx, sid, 1 << 30, 0.1, 1)
    assert e.value.code == dino.DINO_ENOMEM
    dino.dino_chains_destroy(ctx, pool)
    dino.dino_unload_surrogate(ctx, sid)
    assert dino.dino_last_error(ctx) == ""


def test_r1_and_zero_steps(dino, ctx):
    """Degenerate reduced space (r = 1) and a zero-step call."""
    w = variant(CONFIGS["small_fp64"], n_grid=4, r=1, widths=[1, 6, 3], noise_frac=0.3)
    sid = gpu_setup(dino, ctx, w)
    sur, E, D = oracle_setup(w)
    pool = dino.dino_chains_create(ctx, sid, 9, 0.7, SEED_CHAINS)
    before = dino.dino_chains_read(ctx, pool, 9, w.r, w.N)
    st = dino.dino_chains_step(ctx, pool, 0)
    after = dino.dino_chains_read(ctx, pool, 9, w.r, w.N)
    assert st["proposals"] == 0 and np.array_equal(before["m_r"], after["m_r"])
    och = _oracle_chains(dino, ctx, sid, w, sur, E, D, 9, 0.7)
    acc, _, _ = step_and_compare(dino, ctx, pool, och, w, 9, 40, tol=TOL)
    assert 0.0 < np.mean(acc) <= 1.0
    dino.dino_chains_destroy(ctx, pool)
    dino.dino_unload_surrogate(ctx, sid)


def test_zero_jacobian_reduces_to_pcn(dino, ctx):
    """Zero last-layer weights: H = 0, g = 0, the proposal is pCN and log rho == 0 (Sec. 2.7)."""
    w = variant(CONFIGS["small_fp64"], widths=[16, 12, 7])
    inp = surrogate_inputs(w)
    Ws = [x.copy() for x in inp["Ws"]]
    Ws[-1][:] = 0.0
    sid = dino.dino_load_surrogate(
        ctx, n_grid=w.n_grid, prior_gamma=w.prior_gamma, prior_delta=w.prior_delta, r=w.r,
        widths=w.widths, activation=w.activation, W=Ws, b=inp["bs"], basis_kind=BASIS_KLE,
        y=np.zeros(w.d_y), noise_var=0.01)
    C, dt = 6, 0.8
    s = (4 - dt) / (4 + dt)
    pool = dino.dino_chains_create(ctx, sid, C, dt, SEED_CHAINS)
    a = dino.dino_chains_read(ctx, pool, C, w.r, w.N)["m_r"]
    dino.dino_chains_step(ctx, pool, 1, stats=False)
    last = dino.dino_chains_read_last(ctx, pool, C, w.r)
    from oracle import philox
    xi = philox.normals(SEED_CHAINS, philox.STREAM_XI, 0, np.arange(C), w.r)
    assert rel_err(last["b"], s * a + np.sqrt(1 - s * s) * xi) <= TOL
    assert np.abs(last["log_rho"]).max() <= 1e-12
    assert last["accepted"].all()
    dino.dino_chains_destroy(ctx, pool)
    dino.dino_unload_surrogate(ctx, sid)


@pytest.mark.parametrize("dy", [192, 193])
def test_noise_map_boundary_matches_oracle(dino, ctx, dy):
    """r = 200: d_y = 192 runs the Woodbury path (perturbation noise), d_y = 193
    the r-sized path (Cholesky noise); both follow the oracle's rule at 1e-10."""
    w = variant(CONFIGS["small_fp64"], n_grid=15, r=200, widths=[200, 64, dy],
                activation=ACT_TANH, noise_frac=0.2)
    sid = gpu_setup(dino, ctx, w)
    info = dino.dino_surrogate_query(ctx, sid)
    assert info["noise_map"] == ("perturbation" if dy == 192 else "cholesky")
    assert (info["r"], info["d_y"], info["N"]) == (w.r, dy, w.N)
    sur, E, D = oracle_setup(w)
    pool = dino.dino_chains_create(ctx, sid, 3, 2e-4, SEED_CHAINS)
    och = _oracle_chains(dino, ctx, sid, w, sur, E, D, 3, 2e-4)
    step_and_compare(dino, ctx, pool, och, w, 3, 3, tol=TOL)
    dino.dino_chains_destroy(ctx, pool)
    dino.dino_unload_surrogate(ctx, sid)
