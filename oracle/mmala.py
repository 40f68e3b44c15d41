"""Surrogate mMALA transition in reduced coordinates (oracle).

TEST INFRASTRUCTURE ONLY (see `oracle/__init__.py`).

Target.  The surrogate posterior (eq:surrogate_posterior, Sec. 2.8) in the
whitened reduced coordinates m_r = Psi_r^* m has density
    pi(m_r) ∝ exp(-Phi(m_r) - |m_r|^2 / 2),
the complement staying at its prior (Lemma on encoded white noise, Sec. 5.3).

Readings of the paper taken here (each also listed in the design notes):
* Gamma = noise_var * I and the observable basis V = sqrt(noise_var) I, so the
  MLP outputs observables in data units and Gamma^-1 is written explicitly:
  Phi = |f - y|^2 / (2 noise_var), H = J^T J / noise_var (eq:surrogate_rppgnh).
* The reduced ppg is printed as J^T (V^* y - f) in eq:surrogate_rppg; the
  drift of eq:mmala, eq:ppg and rho_{0,r} all need the gradient of Phi, so
  g = J^T (f - y) / noise_var.
* In rho_{0,r} (Sec. 5.4) the factor prod_j (d_j + 1)^{1/2} multiplies the
  exponential (it is the determinant factor of eq:mmala_trr); its weight
  is (I + H)^-1.  In logs: + (1/2) log det(I + H).
* The proposal noise map is L^-T xi with L L^T = I + H (lower Cholesky
  factor).  It has the law of the eigen form of eq:reduced_space_sampling
  (covariance (1 - s^2)(I + H)^-1); `reduced_proposal_eigen` keeps the
  paper's map for distribution checks.
* The paper's own eigen map, in its symmetric form P diag((d+1)^-1/2) P^T xi
  (`reduced_proposal_sqrt`), is a third choice with the same law.
* The noise may instead be drawn as zeta = (I + H)^-1 (xi1 + K^T xi2) with
  K = J / sqrt(noise_var) and d_y further normals xi2: the same law
  (`reduced_proposal_perturbation`), which needs only the d_y x d_y matrix
  I + K K^T to be factored.  Which of the two maps a chain uses is an explicit
  argument of the chain driver (`NOISE_MAPS`); both give the proposal law of
  eq:reduced_space_sampling, so the choice is a property of the sampler being
  compared against, not of the method.
* Accept iff log u <= min(0, log rho) (Alg. 1 rejects iff alpha < u);
  a non-finite log rho is a reject.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import mlp


def s_of_dt(dt: float) -> float:
    """s = (4 - dt)/(4 + dt) (eq:mmala)."""
    return (4.0 - dt) / (4.0 + dt)


@dataclass
class Surrogate:
    Ws: list
    bs: list
    act: int
    y: np.ndarray
    noise_var: float
    jac_mode: str = "reverse"

    @property
    def r(self) -> int:
        return self.Ws[0].shape[1]

    @property
    def d_y(self) -> int:
        return self.Ws[-1].shape[0]


@dataclass
class Geometry:
    """Surrogate quantities at a reduced point ("Known at m_j" in Alg. 1)."""
    f: np.ndarray       # (..., d_y)
    J: np.ndarray       # (..., d_y, r)
    phi: np.ndarray     # (...)
    g: np.ndarray       # (..., r)
    H: np.ndarray       # (..., r, r)
    L: np.ndarray       # (..., r, r) lower Cholesky factor of I + H
    hld: np.ndarray     # (...) half log det(I + H)


def geometry(sur: Surrogate, m_r) -> Geometry:
    """Misfit, gradient, Gauss-Newton Hessian and its factor at m_r (Sec. 5.1; the geometry step of Algorithm 1)."""
    m_r = np.asarray(m_r, dtype=np.float64)
    f, zs = mlp.forward(sur.Ws, sur.bs, sur.act, m_r)
    if len(sur.Ws) == 1:
        J = np.broadcast_to(sur.Ws[0], m_r.shape[:-1] + sur.Ws[0].shape).copy()
    elif sur.jac_mode == "forward":
        J = mlp.jacobian_forward(sur.Ws, sur.act, zs)
    else:
        J = mlp.jacobian_reverse(sur.Ws, sur.act, zs)
    res = f - sur.y
    phi = 0.5 * np.sum(res * res, axis=-1) / sur.noise_var
    g = np.einsum("...ij,...i->...j", J, res) / sur.noise_var
    H = np.einsum("...ki,...kj->...ij", J, J) / sur.noise_var
    r = m_r.shape[-1]
    L = np.linalg.cholesky(np.eye(r) + H)
    hld = np.sum(np.log(np.diagonal(L, axis1=-2, axis2=-1)), axis=-1)
    return Geometry(f=f, J=J, phi=phi, g=g, H=H, L=L, hld=hld)


def _solve(A, b):
    return np.linalg.solve(A, b[..., None])[..., 0]


def proposal_mean(a, geo: Geometry, dt: float):
    """mu = s a + (1 - s) A~(a) with A~(a) = a - (I + H)^-1 (a + g) (eq:mmala, Sec. 5.3)."""
    s = s_of_dt(dt)
    r = a.shape[-1]
    v = _solve(np.eye(r) + geo.H, a + geo.g)
    return a - (1.0 - s) * v


def reduced_proposal(a, geo: Geometry, xi, dt: float):
    """m_r^dagger = mu + sqrt(1 - s^2) L^-T xi (Prop. 5.1, Cholesky noise map).  Returns (mu, b)."""
    s = s_of_dt(dt)
    mu = proposal_mean(a, geo, dt)
    LT = np.swapaxes(geo.L, -1, -2)
    eta = _solve(LT, np.asarray(xi, dtype=np.float64))
    return mu, mu + np.sqrt(1.0 - s * s) * eta


NOISE_MAPS = ("cholesky", "perturbation", "eigen")


def reduced_proposal_perturbation(a, geo: Geometry, xi1, xi2, noise_var: float, dt: float):
    """m_r^dagger = mu + sqrt(1 - s^2) zeta, zeta = (I + H)^-1 (xi1 + K^T xi2), K = J / sqrt(noise_var).

    With xi1 ~ N(0, I_r) and xi2 ~ N(0, I_{d_y}) independent, zeta is Gaussian
    with covariance (I + H)^-1 (I + K^T K) (I + H)^-1 = (I + H)^-1, because
    H = K^T K (eq:surrogate_rppgnh, Gamma = noise_var I): the law of the noise
    of eq:reduced_space_sampling.  The mean is `proposal_mean`.  Returns (mu, b).
    """
    s = s_of_dt(dt)
    mu = proposal_mean(a, geo, dt)
    r = a.shape[-1]
    K = geo.J / np.sqrt(noise_var)
    rhs = (np.asarray(xi1, dtype=np.float64)
           + np.einsum("...ij,...i->...j", K, np.asarray(xi2, dtype=np.float64)))
    zeta = _solve(np.eye(r) + geo.H, rhs)
    return mu, mu + np.sqrt(1.0 - s * s) * zeta


def reduced_proposal_sqrt(a, geo: Geometry, xi, dt: float):
    """m_r^dagger = mu + sqrt(1 - s^2) (I + H)^-1/2 xi with the symmetric root
    (I + H)^-1/2 = P diag((d + 1)^-1/2) P^T, H = P diag(d) P^T.

    This is the eigen form of eq:reduced_space_sampling written so that it
    does not depend on the signs or the order of the eigenvectors: the
    paper's P diag(...) Xi with Xi = P^T xi (the same law, since P^T xi is
    again standard normal).  Returns (mu, b).
    """
    s = s_of_dt(dt)
    mu = proposal_mean(a, geo, dt)
    d, P = np.linalg.eigh(geo.H)
    Pt = np.swapaxes(P, -1, -2)
    y = np.einsum("...ij,...j->...i", Pt, np.asarray(xi, dtype=np.float64))
    zeta = np.einsum("...ij,...j->...i", P, y / np.sqrt(d + 1.0))
    return mu, mu + np.sqrt(1.0 - s * s) * zeta


def reduced_proposal_eigen(a, H, g, xi, dt: float):
    """The paper's eigen form of eq:reduced_space_sampling with H = P diag(d) P^T."""
    s = s_of_dt(dt)
    d, P = np.linalg.eigh(H)
    Pt = np.swapaxes(P, -1, -2)

    def apply(diag, v):
        return np.einsum("...ij,...j->...i", P, diag * np.einsum("...ij,...j->...i", Pt, v))

    return (apply((d + s) / (d + 1.0), a) - apply((1.0 - s) / (d + 1.0), g)
            + np.einsum("...ij,...j->...i", P, np.sqrt((1.0 - s * s) / (d + 1.0)) * xi))


def log_rho0(m1, m2, geo1: Geometry, dt: float):
    """log of rho_{0,r}(m1, m2): surrogate mMALA vs pCN proposal density (Sec. 5.4, eq:mmala_trr).

    -dt/8 w^T (I+H)^-1 w + sqrt(dt)/2 mhat^T w + (1/2) log det(I+H) - (1/2) mhat^T H mhat,
    w = H m1 - g, mhat = (m2 - s m1)/sqrt(1 - s^2), all at m1.
    """
    s = s_of_dt(dt)
    r = m1.shape[-1]
    H, g = geo1.H, geo1.g
    w = np.einsum("...ij,...j->...i", H, m1) - g
    Kw = _solve(np.eye(r) + H, w)
    mhat = (m2 - s * m1) / np.sqrt(1.0 - s * s)
    Hm = np.einsum("...ij,...j->...i", H, mhat)
    return (-dt / 8.0 * np.sum(w * Kw, -1) + np.sqrt(dt) / 2.0 * np.sum(mhat * w, -1)
            + geo1.hld - 0.5 * np.sum(mhat * Hm, -1))


def log_rho(a, geo_a: Geometry, b, geo_b: Geometry, dt: float):
    """log rho_r^(1)(a, b) = Phi(a) - Phi(b) + log rho_0(b, a) - log rho_0(a, b) (eq:da_dino_trr_1)."""
    return geo_a.phi - geo_b.phi + log_rho0(b, a, geo_b, dt) - log_rho0(a, b, geo_a, dt)


def accept(log_u, log_rho_val):
    """The accept test of Algorithm 1: accept iff alpha >= u, i.e. log u <= min(0, log rho); NaN rejects."""
    lr = np.asarray(log_rho_val)
    return np.isfinite(lr) & (np.asarray(log_u) <= np.minimum(0.0, lr))


def log_target(geo: Geometry, m):
    """log pi(m_r) up to a constant: -Phi - |m_r|^2 / 2."""
    return -geo.phi - 0.5 * np.sum(m * m, -1)


def log_q(a, geo_a: Geometry, b, dt: float):
    """Gaussian log density of the reduced proposal N(mu_a, (1 - s^2)(I + H_a)^-1) at b."""
    s = s_of_dt(dt)
    r = a.shape[-1]
    mu = proposal_mean(a, geo_a, dt)
    prec = (np.eye(r) + geo_a.H) / (1.0 - s * s)
    d = b - mu
    _, logdet_prec = np.linalg.slogdet(prec)
    return (-0.5 * np.einsum("...i,...ij,...j->...", d, prec, d)
            + 0.5 * logdet_prec - 0.5 * r * np.log(2.0 * np.pi))


def field_proposal(m, b, M, E, D, dt: float):
    """Full proposal of Prop. 5.1: (I - Psi Psi^*) M_perp + Psi b with M_perp = s m + sqrt(1-s^2) M.

    m, M: (..., N) field and prior draw; b: (..., r) reduced proposal;
    E: (r, N) encoder Psi_r^*; D: (N, r) decoder Psi_r.
    """
    s = s_of_dt(dt)
    M_perp = s * m + np.sqrt(1.0 - s * s) * M
    return M_perp - (M_perp @ E.T) @ D.T + b @ D.T
