"""Pins of the oracle's chain diagnostics (CPU only).

* W and V on a hand-computed two-chain example;
* Wasserstein MPSRF: 0 for W = V; sum_i (sqrt(w_i) - sqrt(v_i))^2 for
  commuting W, V (the closed form of the Gaussian 2-Wasserstein distance),
  also after a common rotation;
* ESS%: about 1 for independent draws, (1 - phi)/(1 + phi) for an AR(1)
  process (its integrated autocorrelation time is (1 + phi)/(1 - phi));
* MSJ of a known sequence.
"""
import numpy as np

from oracle import diagnostics as dg


def test_covariance_estimators_by_hand():
    # chain 1: 1, 2, 3 (mean 2, s^2 = 1); chain 2: 3, 5, 7 (mean 5, s^2 = 4)
    X = np.array([[[1.0], [2.0], [3.0]], [[3.0], [5.0], [7.0]]])
    W, V = dg.covariance_estimators(X)
    assert W[0, 0] == (1.0 + 4.0) / 2
    # V = (2/3) W + (3 / 2) ((2 - 3.5)^2 + (5 - 3.5)^2)
    assert abs(V[0, 0] - (2.0 / 3.0 * 2.5 + 1.5 * 4.5)) < 1e-14


def test_wasserstein_closed_forms():
    rng = np.random.default_rng(1)
    w = rng.uniform(0.5, 2.0, 6)
    v = rng.uniform(0.5, 2.0, 6)
    ref = np.sum((np.sqrt(w) - np.sqrt(v)) ** 2)
    assert abs(dg.wasserstein_mpsrf(np.diag(w), np.diag(v)) - ref) < 1e-12
    Q, _ = np.linalg.qr(rng.standard_normal((6, 6)))
    assert abs(dg.wasserstein_mpsrf(Q @ np.diag(w) @ Q.T, Q @ np.diag(v) @ Q.T) - ref) < 1e-12
    A = rng.standard_normal((6, 6))
    A = A @ A.T
    assert abs(dg.wasserstein_mpsrf(A, A)) < 1e-10 * np.trace(A)


def test_ess_of_independent_draws_and_ar1():
    rng = np.random.default_rng(2)
    n_c, n_s = 64, 2000
    iid = rng.standard_normal((n_c, n_s))
    assert abs(dg.ess_fraction(iid) - 1.0) < 0.08
    for phi in (0.5, 0.8):
        x = np.empty((n_c, n_s))
        x[:, 0] = rng.standard_normal(n_c) / np.sqrt(1 - phi * phi)
        for j in range(1, n_s):
            x[:, j] = phi * x[:, j - 1] + rng.standard_normal(n_c)
        ref = (1 - phi) / (1 + phi)
        assert abs(dg.ess_fraction(x) / ref - 1.0) < 0.1
    # chains stuck at different values: the between-chain term dominates
    stuck = np.repeat(rng.standard_normal((n_c, 1)), n_s, axis=1) + 1e-3 * iid
    assert dg.ess_fraction(stuck) < 0.01


def test_mean_squared_jump():
    X = np.zeros((2, 4, 2))
    X[0, :, 0] = [0, 1, 3, 6]          # jumps 1, 2, 3 -> (1 + 4 + 9) / 3
    X[1, :, 1] = [0, 0, 2, 2]          # jumps 0, 2, 0 -> 4 / 3
    assert abs(dg.mean_squared_jump(X) - (14 / 3 + 4 / 3) / 2) < 1e-14
