"""Second (true-model) stage of delayed-acceptance DINO-mMALA (oracle).

TEST INFRASTRUCTURE ONLY (see `oracle/__init__.py`).

Algorithm 1, once the first stage (surrogate-only, eq:da_dino_trr_1) has
accepted the reduced proposal: assemble the full proposal m^dagger (Prop.
5.1), evaluate the data misfit of the true parameter-to-observable map there,
and accept with probability min(1, rho^(2)), where (eq:da_dino_trr_2)

    rho^(2)(m_j, m^dagger) = exp(-Phi~(m_r,j)) exp(-Phi(m^dagger))
                             / (exp(-Phi~(m_r^dagger)) exp(-Phi(m_j))),

i.e. log rho^(2) = Phi(m_j) - Phi(m^dagger) + Phi~(m_r^dagger) - Phi~(m_r,j).
A first-stage rejection returns m_j without touching the true model.

The paper's true maps are PDE solves; a stand-in of the same role is used
here: a larger MLP acting on an encoding of the FULL field, G(m) = f_t(E_t m)
with E_t an r_t x N matrix (r_t >= r, so G sees directions that the
surrogate's reduced basis leaves out).  Its data misfit uses the surrogate's
data and noise, Phi(m) = |G(m) - y|^2 / (2 noise_var).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import mlp


@dataclass
class TrueModel:
    Et: np.ndarray      # (r_t, N) encoder of the true map
    Ws: list            # MLP r_t -> ... -> d_y
    bs: list
    act: int

    def observe(self, m):
        """G(m) = f_t(E_t m) for fields m of shape (..., N)."""
        f, _ = mlp.forward(self.Ws, self.bs, self.act, np.asarray(m) @ self.Et.T)
        return f

    def misfit(self, m, y, noise_var: float):
        """Phi(m) = |G(m) - y|^2 / (2 noise_var) (the data misfit of Sec. 2.2, Gamma = noise_var I)."""
        res = self.observe(m) - y
        return 0.5 * np.sum(res * res, axis=-1) / noise_var


def log_rho2(phi_true_cur, phi_true_prop, phi_sur_cur, phi_sur_prop):
    """log rho^(2) of eq:da_dino_trr_2 from the four misfit values."""
    return phi_true_cur - phi_true_prop + phi_sur_prop - phi_sur_cur
