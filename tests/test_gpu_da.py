"""Delayed acceptance: the two-stage transition of Algorithm 1 (GPU).

The true map is G(m) = f_t(E_t m) with E_t the surrogate's encoder stacked
with further KLE rows (each side builds its own) and f_t the surrogate's
network that also reads those extra coordinates (seeded, scaled by EPS); the
data are the surrogate's.
  * FP64 path: every quantity of both stages matches the oracle at 1e-10
    (Cholesky and perturbation noise maps, so that the second stage's commit
    of the Woodbury state J is covered);
  * a true map equal to the surrogate composed with its encoder gives
    rho^(2) = 1: the two-stage chain is the surrogate-only chain, bit for bit;
  * BF16 path at r = 200: the proposal mean meets its bar and the first-
    and second-stage decisions are counted against the oracle's;
  * the surrogate refuses a new true map while pools of it exist.
"""
import numpy as np
import pytest

from helpers import gpu_setup, oracle_chains, oracle_setup, rel_err, variant
from oracle import da, prior
from workloads import (BASIS_DIS, BASIS_KLE, CONFIGS, SEED_CHAINS, surrogate_inputs,
                       true_model_weights)

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


EPS = 0.05


def _library_kle(dino, ctx, w, r_k):
    """The library's own rank-r_k KLE encoder (through a throwaway surrogate)."""
    Ws = [np.zeros((2, r_k)), np.zeros((2, 2))]
    sid = dino.dino_load_surrogate(
        ctx, n_grid=w.n_grid, prior_gamma=w.prior_gamma, prior_delta=w.prior_delta, r=r_k,
        widths=[r_k, 2, 2], activation=1, W=Ws, b=[np.zeros(2), np.zeros(2)],
        basis_kind=BASIS_KLE)
    E, _ = dino.dino_read_basis(ctx, sid, r_k, w.N)
    dino.dino_unload_surrogate(ctx, sid)
    return E


def _setup(dino, ctx, w, r_c):
    """Surrogate of `w` with the true map f_t(E_t m), E_t = [E; KLE rows r .. r + r_c - 1]
    (each side its own encoder and KLE rows), f_t the surrogate's network with
    the extra coordinates entering its first layer through EPS V."""
    sid = gpu_setup(dino, ctx, w)
    E_lib, _ = dino.dino_read_basis(ctx, sid, w.r, w.N)
    Et_lib = np.vstack([E_lib, _library_kle(dino, ctx, w, w.r + r_c)[w.r:]])
    Ws, bs = true_model_weights(w, r_c, EPS)
    dino.dino_set_true_model(ctx, sid, E_t=Et_lib, W=Ws, b=bs, activation=w.activation)
    assert dino.dino_surrogate_query(ctx, sid)["true_model_rank"] == w.r + r_c
    sur, E, D = oracle_setup(w)
    Ek, _ = prior.kle_basis(w.n_grid, w.prior_gamma, w.prior_delta, w.r + r_c)
    tm = da.TrueModel(Et=np.vstack([E, Ek[w.r:]]), Ws=Ws, bs=bs, act=w.activation)
    return sid, sur, E, D, tm


def _compare(dino, ctx, pool, och, w, C, steps, tol):
    counts = np.zeros(2, dtype=int)
    active = np.ones(C, dtype=bool)
    for _ in range(steps):
        st = dino.dino_chains_step(ctx, pool, 1)
        och.step()
        last = dino.dino_chains_read_last(ctx, pool, C, w.r)
        dd = dino.dino_chains_read_da(ctx, pool, C)
        s = dino.dino_chains_read(ctx, pool, C, w.r, w.N)
        o = och.last
        a = active
        assert rel_err(last["b"][a], o["b"][a]) <= tol
        assert np.array_equal(dd["stage1"][a], o["stage1"][a])
        assert np.array_equal(last["accepted"][a], o["accepted"][a])
        assert st["stage1_accepts"] == int(dd["stage1"].sum())
        assert st["accepts"] == int(last["accepted"].sum())
        s1 = o["stage1"] & a
        scale = np.maximum(1.0, np.abs(och.phi_true) + np.abs(o["phi_true_b"]) + np.abs(o["phi_b"]))
        assert np.all(np.abs(dd["log_rho2"][s1] - o["log_rho2"][s1]) <= tol * scale[s1])
        assert np.isnan(dd["log_rho2"][~dd["stage1"]]).all()
        assert rel_err(dd["log_u2"], o["log_u2"]) <= 1e-14
        assert rel_err(dd["phi_true"][a], och.phi_true[a]) <= tol
        assert rel_err(s["m_r"][a], och.m_r[a]) <= tol
        assert rel_err(s["m"][a], och.m[a]) <= tol
        counts += [int(o["stage1"].sum()), int(o["accepted"].sum())]
    return counts


@pytest.mark.parametrize("w,dt", [
    (CONFIGS["small_fp64"], 0.002),
    (variant(CONFIGS["small_fp64"], n_grid=9, r=45, widths=[45, 33, 17, 20],
             basis_kind=BASIS_DIS, activation=2, noise_frac=0.2), 0.01)],
    ids=["cholesky", "perturbation"])
def test_fp64_two_stage_chains_match_oracle(dino, ctx, w, dt):
    sid, sur, E, D, tm = _setup(dino, ctx, w, 8)
    C = 32
    pool = dino.dino_chains_create(ctx, sid, C, dt, SEED_CHAINS)
    och = oracle_chains(dino, ctx, sid, w, sur, E, D, C, dt, true_model=tm)
    assert rel_err(dino.dino_chains_read_da(ctx, pool, C)["phi_true"], och.phi_true) <= TOL
    s1, acc = _compare(dino, ctx, pool, och, w, C, 12, TOL)
    assert s1 > acc > 0                     # both stages accept and the second rejects
    dino.dino_chains_destroy(ctx, pool)
    with pytest.raises(dino.DinoError) as e:      # a live pool pins the true model
        p2 = dino.dino_chains_create(ctx, sid, 2, dt, 1)
        dino.dino_set_true_model(ctx, sid)
    assert e.value.code == dino.DINO_ESTATE
    dino.dino_chains_destroy(ctx, p2)
    dino.dino_set_true_model(ctx, sid)            # detach: the surrogate-only chain again
    assert dino.dino_surrogate_query(ctx, sid)["true_model_rank"] == 0
    dino.dino_unload_surrogate(ctx, sid)


def test_true_map_equal_to_surrogate_is_the_one_stage_chain(dino, ctx):
    """G = f o Psi_r^* (FP64): rho^(2) = 1 up to rounding, so every first-stage
    accept is final and the chain equals the surrogate-only one bit for bit."""
    w = CONFIGS["small_fp64"]
    plain = gpu_setup(dino, ctx, w)
    sid = gpu_setup(dino, ctx, w)
    E, _ = dino.dino_read_basis(ctx, sid, w.r, w.N)
    inp = surrogate_inputs(w)
    dino.dino_set_true_model(ctx, sid, E_t=E, W=inp["Ws"], b=inp["bs"], activation=w.activation)
    C, dt = 48, 0.002
    pa = dino.dino_chains_create(ctx, plain, C, dt, SEED_CHAINS)
    pb = dino.dino_chains_create(ctx, sid, C, dt, SEED_CHAINS)
    acc = 0
    for _ in range(6):
        sa = dino.dino_chains_step(ctx, pa, 1)
        sb = dino.dino_chains_step(ctx, pb, 1)
        assert sb["stage1_accepts"] == sb["accepts"] == sa["accepts"]
        acc += sa["accepts"]
        dd = dino.dino_chains_read_da(ctx, pb, C)
        s1 = dd["stage1"]
        phi = dino.dino_chains_read(ctx, pb, C, w.r, w.N, field=False)["phi"]
        assert np.all(np.abs(dd["log_rho2"][s1]) <= 1e-9 * np.maximum(1.0, phi[s1]))
    A = dino.dino_chains_read(ctx, pa, C, w.r, w.N)
    B = dino.dino_chains_read(ctx, pb, C, w.r, w.N)
    for k in ("m_r", "phi", "accepts", "m"):
        assert np.array_equal(A[k], B[k]), k
    assert acc > 0
    for p in (pa, pb):
        dino.dino_chains_destroy(ctx, p)
    dino.dino_unload_surrogate(ctx, sid)
    dino.dino_unload_surrogate(ctx, plain)


def test_bf16_two_stage_chains_r200(dino, ctx):
    """r = 200 DIS surrogate, true map on a 400-dimensional encoding (the DIS
    coordinates and 200 KLE coordinates); 64 chains from the truth at dt = 2e-5."""
    w = CONFIGS["r200_dis_bf16"]
    sid, sur, E, D, tm = _setup(dino, ctx, w, 200)
    C, dt = 64, 2e-5
    m0 = D @ surrogate_inputs(w)["m_true_r"]
    pool = dino.dino_chains_create(ctx, sid, C, dt, SEED_CHAINS, 0,
                                   np.ascontiguousarray(np.broadcast_to(m0, (C, w.N))))
    och = oracle_chains(dino, ctx, sid, w, sur, E, D, C, dt, m0=m0, true_model=tm)
    pt = dino.dino_chains_read_da(ctx, pool, C)["phi_true"]
    # FP32-level forward pass at 1% noise: the misfit moves by ~1e-4 of itself
    # (0.012 at 82 measured), like the surrogate's misfit (test_gpu_bf16)
    assert np.max(np.abs(pt - och.phi_true) / np.maximum(1.0, och.phi_true)) <= 1e-3
    active = np.ones(C, dtype=bool)
    flips = n = s1_tot = acc_tot = 0
    for _ in range(4):
        dino.dino_chains_step(ctx, pool, 1, stats=False)
        och.step()
        last = dino.dino_chains_read_last(ctx, pool, C, w.r)
        dd = dino.dino_chains_read_da(ctx, pool, C)
        o = och.last
        a = active
        mu = np.linalg.norm(last["mu"][a] - o["mu"][a], axis=1) / np.linalg.norm(o["mu"][a], axis=1)
        assert mu.max() <= 1e-3
        agree = (dd["stage1"] == o["stage1"]) & (last["accepted"] == o["accepted"])
        flips += int((~agree & a).sum())
        n += int(a.sum())
        s1_tot += int(o["stage1"][a].sum())
        acc_tot += int(o["accepted"][a].sum())
        active &= agree
    # the decision bar of the BF16 path is not met (see test_gpu_bf16); pinned here
    assert flips <= 0.02 * n
    assert s1_tot > 0 and acc_tot > 0
    dino.dino_chains_destroy(ctx, pool)
    dino.dino_unload_surrogate(ctx, sid)
