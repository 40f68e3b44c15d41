"""Derivative-informed subspace from surrogate Jacobians (oracle).

TEST INFRASTRUCTURE ONLY (see `oracle/__init__.py`).

The DIS basis solves the eigenproblem of the expected prior-preconditioned
Gauss-Newton Hessian (eq:jtj_eigenvalue) estimated by Monte Carlo over prior
draws (eq:mc_ppgnh).  A reduced-basis surrogate sees a parameter only through
its coordinates m_r = Psi_r^* m in a C_pr^-1-orthonormal basis, and there the
ppGNH is J^T Gamma^-1 J (eq:surrogate_rppgnh).  Encoded prior draws are
N(0, I_r) (Lemma on encoded white noise, Sec. 5.3), so the Monte Carlo
estimate over n prior draws is

    H_mc = (1/n) sum_i J(m_r,i)^T J(m_r,i) / noise_var,    m_r,i ~ N(0, I_r),

its eigenpairs (decreasing) H_mc = P diag(lam) P^T give the surrogate's DIS
within span(Psi_r): decoder D' = D P_r', encoder E' = P_r'^T E, which are
again C_pr^-1-orthonormal (P is orthogonal) and satisfy E' D' = I.

The draws m_r,i are Philox normals of stream DIS (6), step 0, "chain" i.
"""
from __future__ import annotations

import numpy as np

from . import mmala, philox

STREAM_DIS = 6


def mc_draws(seed: int, n: int, r: int):
    """The n encoded prior draws m_r,i ~ N(0, I_r) (Philox stream DIS)."""
    return philox.normals(seed, STREAM_DIS, 0, np.arange(n, dtype=np.uint64), r)


def expected_gnh(sur: mmala.Surrogate, samples):
    """H_mc = (1/n) sum_i J_i^T J_i / noise_var (eq:mc_ppgnh in reduced coordinates)."""
    J = mmala.geometry(sur, np.asarray(samples)).J
    return np.einsum("nki,nkj->ij", J, J) / (len(samples) * sur.noise_var)


def surrogate_dis(sur: mmala.Surrogate, E, D, samples, r_new: int):
    """Eigenvalues (decreasing), P (r x r_new), E' (r_new x N), D' (N x r_new)."""
    H = expected_gnh(sur, samples)
    lam, P = np.linalg.eigh(H)
    order = np.argsort(-lam, kind="stable")
    lam, P = lam[order], P[:, order]
    Pr = P[:, :r_new]
    return lam, Pr, Pr.T @ E, D @ Pr
