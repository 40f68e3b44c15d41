"""Builds the same synthetic posterior on both sides of a parity test.

The oracle and the CUDA library each compute their own basis and their own
noiseless observables y0 = f(m_true_r); only the seeded raw inputs (weights,
Gaussian basis matrix, truth coordinates, data noise) come from `workloads`.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from oracle import mlp, mmala, prior
from workloads import (BASIS_DIS, BASIS_KLE, SEED_CHAINS, Workload, make_data,
                       surrogate_inputs)


def variant(w: Workload, **kw) -> Workload:
    """A reshaped workload; unless given, its noise map is the library's choice."""
    return dataclasses.replace(w, **{"noise_map": "auto", **kw})


def oracle_setup(w: Workload):
    inp = surrogate_inputs(w)
    if w.basis_kind == BASIS_KLE:
        E, D = prior.kle_basis(w.n_grid, w.prior_gamma, w.prior_delta, w.r)
    else:
        E, D = prior.dis_basis(w.n_grid, w.prior_gamma, w.prior_delta, inp["G"])
    f0, _ = mlp.forward(inp["Ws"], inp["bs"], w.activation, inp["m_true_r"])
    y, nv = make_data(f0, inp["eps"], w.noise_frac)
    sur = mmala.Surrogate(Ws=inp["Ws"], bs=inp["bs"], act=w.activation, y=y, noise_var=nv)
    return sur, E, D


NOISE_CODES = {"auto": 0, "cholesky": 1, "perturbation": 2, "eigen": 3}


def gpu_setup(dino, ctx, w: Workload, precision=None, fwd_slices=0, jac_slices=0):
    inp = surrogate_inputs(w)
    prec = precision if precision is not None else (
        dino.DINO_PREC_BF16 if w.precision == "bf16" else dino.DINO_PREC_FP64)
    sid = dino.dino_load_surrogate(
        ctx, n_grid=w.n_grid, prior_gamma=w.prior_gamma, prior_delta=w.prior_delta, r=w.r,
        widths=w.widths, activation=w.activation, W=inp["Ws"], b=inp["bs"],
        basis_kind=w.basis_kind, basis_gauss=inp["G"], precision=prec,
        fwd_slices=fwd_slices, jac_slices=jac_slices, noise_map=NOISE_CODES[w.noise_map])
    # the library's own FP64 forward gives its copy of the noiseless data (an
    # FP64 twin with the same weights; the basis does not enter f)
    twin = dino.dino_load_surrogate(
        ctx, n_grid=w.n_grid, prior_gamma=w.prior_gamma, prior_delta=w.prior_delta, r=w.r,
        widths=w.widths, activation=w.activation, W=inp["Ws"], b=inp["bs"],
        basis_kind=BASIS_KLE, precision=dino.DINO_PREC_FP64)
    ev = dino.dino_surrogate_eval(ctx, twin, inp["m_true_r"][None, :], w.d_y, want_L=False)
    dino.dino_unload_surrogate(ctx, twin)
    y, nv = make_data(ev["f"][0], inp["eps"], w.noise_frac)
    dino.dino_set_data(ctx, sid, y, nv)
    return sid


def noise_of(dino, ctx, sid) -> str:
    """The proposal noise map the library reports for a loaded surrogate."""
    return dino.dino_surrogate_query(ctx, sid)["noise_map"]


def oracle_chains(dino, ctx, sid, w: Workload, sur, E, D, C, dt, **kw):
    """Oracle chains of workload `w` with the noise map the library uses for `sid`."""
    from oracle.chains import OracleChains
    return OracleChains(sur, E, D, w.n_grid, w.prior_gamma, w.prior_delta, C, dt,
                        seed=kw.pop("seed", SEED_CHAINS), noise=noise_of(dino, ctx, sid), **kw)


def rel_err(a, b):
    """max |a - b| / max(1, |b|) elementwise (the FP64 parity metric)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if a.size == 0:
        return 0.0
    return float(np.max(np.abs(a - b) / np.maximum(1.0, np.abs(b))))


def step_and_compare(dino, ctx, pool, och, w: Workload, C: int, steps: int, tol=1e-10,
                     sample=None, near=1e-8, field=True):
    """Advance GPU pool and oracle chains in lockstep and compare every step.

    `sample` lists the GPU chain indices the oracle runs (all chains if None).
    Accept decisions must agree unless |log u - min(0, log rho)| < `near`; a
    chain whose decision differed stops being compared (its trajectory forks).
    Returns per-step acceptance fractions and the largest errors seen.
    """
    idx = np.arange(C) if sample is None else np.asarray(sample)
    active = np.ones(len(idx), dtype=bool)
    worst = dict(b=0.0, mu=0.0, log_rho=0.0, m_r=0.0, phi=0.0, m=0.0)
    acc_frac = []
    for _ in range(steps):
        dino.dino_chains_step(ctx, pool, 1, stats=False)
        och.step()
        last = dino.dino_chains_read_last(ctx, pool, C, w.r)
        st = dino.dino_chains_read(ctx, pool, C, w.r, w.N, field=field)
        o = och.last
        a = active
        e = dict(b=rel_err(last["b"][idx][a], o["b"][a]),
                 mu=rel_err(last["mu"][idx][a], o["mu"][a]))
        lr_g, lr_o = last["log_rho"][idx], o["log_rho"]
        fin = np.isfinite(lr_o) & a
        assert np.array_equal(np.isfinite(lr_g[a]), np.isfinite(lr_o[a]))
        # log rho is a difference of terms far larger than itself: its error is
        # measured relative to the magnitude of those terms
        scale = np.maximum(1.0, o["log_rho_scale"][fin])
        e["log_rho"] = float(np.max(np.abs(lr_g[fin] - lr_o[fin]) / scale, initial=0.0))
        assert rel_err(last["log_u"][idx], o["log_u"]) <= 1e-14
        close = np.abs(o["log_u"] - np.minimum(0.0, np.where(np.isfinite(lr_o), lr_o, -np.inf))) < near
        agree = last["accepted"][idx] == o["accepted"]
        assert np.all(agree | close | ~a), "accept decisions differ away from the threshold"
        active &= agree
        a = active
        e["m_r"] = rel_err(st["m_r"][idx][a], och.m_r[a])
        e["phi"] = rel_err(st["phi"][idx][a], och.geo.phi[a])
        if field:
            e["m"] = rel_err(st["m"][idx][a], och.m[a])
        for k, v in e.items():
            worst[k] = max(worst[k], v)
            assert v <= tol, f"{k}: relative error {v:.3e} > {tol:.1e}"
        acc_frac.append(float(np.mean(o["accepted"])))
    return acc_frac, worst, active
