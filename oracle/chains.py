"""Many independent chains of surrogate-only DINO-mMALA (oracle driver).

TEST INFRASTRUCTURE ONLY (see `oracle/__init__.py`).

One step is one transition of every chain: the surrogate stage of
Algorithm 1 (reduced proposal, surrogate evaluation, first-stage acceptance
with rho_r^(1)) with the complement drawn as in Prop. 5.1, so that an
accepted chain moves its full field m to m^dagger.  There is no second stage:
the target is the surrogate posterior.

Random numbers (see `philox`): step j of chain c uses XI(j, c) for the r
reduced normals, U(j, c) for the accept uniform and Z(j, c) for the N normals
of the complement prior draw; the initial prior draw uses INIT(0, c).  With
the perturbation noise map the d_y further normals come from XI2(j, c).
The noise map ("cholesky" or "perturbation", see `mmala.NOISE_MAPS`) is an
explicit argument.  `step(noise=...)` replaces the draws of one transition by
given arrays (xi, xi2, z, log_u, log_u2), any of which may be absent.

With a `true_model` (see `da.TrueModel`) every transition is the two-stage
delayed-acceptance step of Algorithm 1: a first-stage acceptance is followed
by the true misfit at the full proposal m^dagger and the test with rho^(2)
(eq:da_dino_trr_2) against its own uniform U2(j, c); only a second-stage
acceptance moves the chain.
"""
from __future__ import annotations

import numpy as np

from . import da, mmala, philox, prior


class OracleChains:
    def __init__(self, sur: mmala.Surrogate, E, D, n_grid: int, gamma: float, delta: float,
                 n_chains: int, dt: float, seed: int, m0=None, chain_ids=None, *,
                 noise: str, true_model=None):
        if noise not in mmala.NOISE_MAPS:
            raise ValueError(f"noise map must be one of {mmala.NOISE_MAPS}, got {noise!r}")
        self.sur, self.E, self.D = sur, np.asarray(E), np.asarray(D)
        self.n_grid, self.gamma, self.delta = n_grid, gamma, delta
        self.dt, self.seed = float(dt), int(seed)
        self.noise = noise
        self.ids = (np.arange(n_chains, dtype=np.uint64) if chain_ids is None
                    else np.asarray(chain_ids, dtype=np.uint64))
        C = len(self.ids)
        N = n_grid * n_grid
        if m0 is None:
            z = philox.normals(seed, philox.STREAM_INIT, 0, self.ids, N)
            m0 = prior.prior_sample(n_grid, gamma, delta, z)
        self.m = np.array(np.broadcast_to(np.asarray(m0, dtype=np.float64), (C, N)))
        self.m_r = self.m @ self.E.T                     # m_r = Psi_r^* m (eq:projector)
        self.geo = mmala.geometry(sur, self.m_r)
        # delayed acceptance (Algorithm 1's second stage) when a true model is given
        self.tm = true_model
        self.phi_true = (true_model.misfit(self.m, sur.y, sur.noise_var)
                         if true_model is not None else None)
        self.step_index = 0
        self.accepts = np.zeros(C, dtype=np.int64)
        self.last = None

    def step(self, n_steps: int = 1, noise=None):
        for k in range(n_steps):
            self._step(noise if k == 0 else None)

    def _step(self, given=None):
        j = self.step_index
        sur, dt, r = self.sur, self.dt, self.sur.r
        N = self.m.shape[1]
        given = given or {}

        def draw(name, stream, width):
            if given.get(name) is not None:
                return np.asarray(given[name], dtype=np.float64)
            return philox.normals(self.seed, stream, j, self.ids, width)

        xi = draw("xi", philox.STREAM_XI, r)
        if given.get("log_u") is not None:
            log_u = np.asarray(given["log_u"], dtype=np.float64)
        else:
            log_u = np.log(philox.uniform(self.seed, philox.STREAM_U, j, self.ids))
        a, geo_a = self.m_r, self.geo
        if self.noise == "perturbation":
            xi2 = draw("xi2", philox.STREAM_XI2, sur.d_y)
            mu, b = mmala.reduced_proposal_perturbation(a, geo_a, xi, xi2, sur.noise_var, dt)
        elif self.noise == "eigen":
            mu, b = mmala.reduced_proposal_sqrt(a, geo_a, xi, dt)
        else:
            mu, b = mmala.reduced_proposal(a, geo_a, xi, dt)
        geo_b = mmala.geometry(sur, b)
        lr = mmala.log_rho(a, geo_a, b, geo_b, dt)
        # magnitude of the terms log rho sums (the scale its rounding error lives on)
        lr_scale = (np.abs(geo_a.phi) + np.abs(geo_b.phi)
                    + np.abs(mmala.log_rho0(a, b, geo_a, dt))
                    + np.abs(mmala.log_rho0(b, a, geo_b, dt)))
        acc = mmala.accept(log_u, lr)
        z = draw("z", philox.STREAM_Z, N)
        M = prior.prior_sample(self.n_grid, self.gamma, self.delta, z)
        m_new = mmala.field_proposal(self.m, b, M, self.E, self.D, dt)
        extra = {}
        if self.tm is not None:
            # second stage: the true misfit at the full proposal, rho^(2) and
            # its own uniform; a first-stage rejection never reaches it
            acc1 = acc
            phi_t_new = self.tm.misfit(m_new, sur.y, sur.noise_var)
            lr2 = da.log_rho2(self.phi_true, phi_t_new, geo_a.phi, geo_b.phi)
            if given.get("log_u2") is not None:
                log_u2 = np.asarray(given["log_u2"], dtype=np.float64)
            else:
                log_u2 = np.log(philox.uniform(self.seed, philox.STREAM_U2, j, self.ids))
            acc = acc1 & mmala.accept(log_u2, lr2)
            extra = dict(stage1=acc1.copy(), log_rho2=np.where(acc1, lr2, np.nan),
                         log_u2=log_u2, phi_true_b=phi_t_new)
            self.phi_true = np.where(acc, phi_t_new, self.phi_true)
        self.last = dict(mu=mu, b=b, log_rho=lr, log_rho_scale=lr_scale, log_u=log_u, accepted=acc.copy(),
                         phi_b=geo_b.phi, hld_b=geo_b.hld, J_b=geo_b.J, f_b=geo_b.f,
                         g_b=geo_b.g, L_b=geo_b.L, m_new=m_new, **extra)
        self.m = np.where(acc[:, None], m_new, self.m)
        self.m_r = np.where(acc[:, None], b, a)
        g = self.geo
        self.geo = mmala.Geometry(
            f=np.where(acc[:, None], geo_b.f, g.f),
            J=np.where(acc[:, None, None], geo_b.J, g.J),
            phi=np.where(acc, geo_b.phi, g.phi),
            g=np.where(acc[:, None], geo_b.g, g.g),
            H=np.where(acc[:, None, None], geo_b.H, g.H),
            L=np.where(acc[:, None, None], geo_b.L, g.L),
            hld=np.where(acc, geo_b.hld, g.hld))
        self.accepts += acc
        self.step_index += 1
