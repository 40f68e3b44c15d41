"""Reduced MLP f: R^r -> R^{d_y} and its Jacobian (oracle).

TEST INFRASTRUCTURE ONLY (see `oracle/__init__.py`).

The reduced-basis neural operator evaluates f_NN on the encoded parameter
m_r = Psi_r^* m (eq:rb_dino, Sec. 4); its reduced Jacobian is
J = d f_NN / d m_r (Sec. 4, "surrogate reduced Jacobian").  The network is
    z_l = W_l a_{l-1} + b_l,   a_l = sigma(z_l)   (hidden layers),
    f   = W_L a_{L-1} + b_L                        (linear output layer),
with sigma = identity, tanh or GELU.  GELU is read as the exact
x Phi(x) (the paper names GELU without a variant, Sec. 7.4).

J = W_L D_{L-1} W_{L-1} ... D_1 W_1 with D_l = diag(sigma'(z_l)).  Reverse mode
multiplies from the left, forward mode from the right; the cheaper order has
the min(d_y, r) dimension on the outside (the paper's min{d_y, r} count of
Jacobian actions, Sec. 4.3).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

ACT_IDENTITY = 0
ACT_TANH = 1
ACT_GELU = 2

_INV_SQRT2 = 1.0 / math.sqrt(2.0)
_INV_SQRT2PI = 1.0 / math.sqrt(2.0 * math.pi)


def act(kind: int, z):
    if kind == ACT_IDENTITY:
        return np.array(z, dtype=np.float64, copy=True)
    if kind == ACT_TANH:
        return np.tanh(z)
    if kind == ACT_GELU:
        return 0.5 * z * (1.0 + erf(z * _INV_SQRT2))
    raise ValueError(kind)


def act_deriv(kind: int, z):
    if kind == ACT_IDENTITY:
        return np.ones_like(z)
    if kind == ACT_TANH:
        return 1.0 - np.tanh(z) ** 2
    if kind == ACT_GELU:
        # d/dz [z Phi(z)] = Phi(z) + z phi(z)
        return 0.5 * (1.0 + erf(z * _INV_SQRT2)) + z * np.exp(-0.5 * z * z) * _INV_SQRT2PI
    raise ValueError(kind)


def forward(Ws, bs, kind: int, x):
    """f(x) and the hidden pre-activations z_1..z_{L-1}.  x: (..., r)."""
    a = np.asarray(x, dtype=np.float64)
    zs = []
    L = len(Ws)
    for l in range(L - 1):
        z = a @ Ws[l].T + bs[l]
        zs.append(z)
        a = act(kind, z)
    f = a @ Ws[L - 1].T + bs[L - 1]
    return f, zs


def jacobian_reverse(Ws, kind: int, zs):
    """J = W_L D_{L-1} W_{L-1} ... D_1 W_1, accumulated from the output side: (..., d_y, r)."""
    L = len(Ws)
    batch = zs[0].shape[:-1] if zs else ()
    P = np.broadcast_to(Ws[L - 1], batch + Ws[L - 1].shape)
    for l in range(L - 2, -1, -1):
        P = P * act_deriv(kind, zs[l])[..., None, :]
        P = P @ Ws[l]
    return np.array(P)


def jacobian_forward(Ws, kind: int, zs):
    """The same J accumulated from the input side: T = W_1, T <- W_{l+1} D_l T."""
    L = len(Ws)
    batch = zs[0].shape[:-1] if zs else ()
    T = np.broadcast_to(Ws[0], batch + Ws[0].shape)
    for l in range(L - 1):
        T = act_deriv(kind, zs[l])[..., :, None] * T
        T = Ws[l + 1] @ T
    return np.array(T)
