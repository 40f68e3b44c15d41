"""Markov-chain diagnostics of a pool of chains (oracle).

TEST INFRASTRUCTURE ONLY (see `oracle/__init__.py`).

Samples are an array X of shape (n_c, n_s, d): n_c chains, n_s samples each
(after burn-in), d degrees of freedom (the reduced coordinates m_r or the
nodal values of the field).  Following the diagnostics section of the paper
(Sec. 6.2):

* covariance estimators (eq:covariance_estimator): the within-chain W and
  the pooled V = (n_s - 1)/n_s W + (n_c + 1)/(n_c (n_c - 1)) sum_k (mbar_k -
  mbar)(mbar_k - mbar)^T;
* Wasserstein MPSRF: Tr(W + V - 2 (W^1/2 V W^1/2)^1/2), the 2-Wasserstein
  distance between N(0, W) and N(0, V);
* ESS% per degree of freedom (eq:ess): 1 / (1 + 2 sum_{t=1}^{2n'+1} MACT(t))
  with MACT(t) = 1 - (w - mean_k AC(t, k)) / v, w and v the 1D versions of W
  and V;
* acceptance rate and mean squared jump (the step-size tuning appendix):
  MSJ = 1/(n_s - 1) sum_j |m_{j+1} - m_j|^2, averaged over chains.

Readings (the section does not fix them):
* AC(t, k) is the lag-t autocovariance of chain k, (1/n_s) sum_{j < n_s - t}
  (x_j - xbar_k)(x_{j+t} - xbar_k): MACT subtracts it from the variance w,
  which only balances if AC carries the variance's units;
* n' is the last index of the initial positive sequence: with MACT(0) = 1
  and P_i = MACT(2i) + MACT(2i+1), n' is the largest n such that P_0 ... P_n
  are all positive (lags beyond n_s - 1 are not formed);
* ESS% is returned as a fraction (1 = as many effective as actual samples).
"""
from __future__ import annotations

import numpy as np


def covariance_estimators(X):
    """W and V of eq:covariance_estimator for X of shape (n_c, n_s, d)."""
    X = np.asarray(X, dtype=np.float64)
    n_c, n_s, d = X.shape
    mk = X.mean(axis=1)                     # (n_c, d) chain means
    m = mk.mean(axis=0)
    Xc = X - mk[:, None, :]
    W = np.einsum("kji,kjl->il", Xc, Xc) / (n_c * (n_s - 1))
    B = (mk - m).T @ (mk - m)
    V = (n_s - 1) / n_s * W + (n_c + 1) / (n_c * (n_c - 1)) * B
    return W, V


def sqrt_psd(A):
    """Symmetric square root of a symmetric positive semidefinite matrix."""
    lam, Q = np.linalg.eigh(0.5 * (A + A.T))
    return (Q * np.sqrt(np.clip(lam, 0.0, None))) @ Q.T


def wasserstein_mpsrf(W, V):
    """Tr(W + V - 2 (W^1/2 V W^1/2)^1/2) (Sec. 6.2.1)."""
    Wh = sqrt_psd(W)
    return float(np.trace(W) + np.trace(V) - 2.0 * np.trace(sqrt_psd(Wh @ V @ Wh)))


def mact(x):
    """MACT(t) for t = 0 .. n_s - 1 of one degree of freedom, x of shape (n_c, n_s)."""
    x = np.asarray(x, dtype=np.float64)
    n_c, n_s = x.shape
    mk = x.mean(axis=1)
    xc = x - mk[:, None]
    w = np.mean(np.sum(xc * xc, axis=1) / (n_s - 1))
    v = (n_s - 1) / n_s * w + (n_c + 1) / (n_c * (n_c - 1)) * np.sum((mk - mk.mean()) ** 2)
    out = np.empty(n_s)
    out[0] = 1.0
    for t in range(1, n_s):
        ac = np.sum(xc[:, :n_s - t] * xc[:, t:], axis=1) / n_s     # AC(t, k)
        out[t] = 1.0 - (w - ac.mean()) / v
    return out


def ess_fraction(x):
    """ESS% (as a fraction) of one degree of freedom, x of shape (n_c, n_s)."""
    rho = mact(x)
    n_s = len(rho)
    total = 0.0                             # sum_{t=1}^{2n'+1} MACT(t)
    i = 0
    while 2 * i + 1 < n_s:
        pair = rho[2 * i] + rho[2 * i + 1]
        if not pair > 0.0:
            break
        total += pair
        i += 1
    # the pairs P_0 .. P_n' summed include MACT(0) = 1
    return 1.0 / (1.0 + 2.0 * (total - 1.0)) if i > 0 else 1.0


def ess_fractions(X):
    """ESS% per degree of freedom for X of shape (n_c, n_s, d)."""
    X = np.asarray(X, dtype=np.float64)
    return np.array([ess_fraction(X[:, :, i]) for i in range(X.shape[2])])


def mean_squared_jump(X):
    """MSJ averaged over chains: 1/(n_s - 1) sum_j |x_{j+1} - x_j|^2."""
    X = np.asarray(X, dtype=np.float64)
    D = np.diff(X, axis=1)
    return float(np.mean(np.sum(D * D, axis=2).sum(axis=1) / (X.shape[1] - 1)))
