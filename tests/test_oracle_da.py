"""Pins of the oracle's delayed-acceptance second stage (CPU only).

p-da1  A true model that IS the surrogate composed with the encoder gives
       rho^(2) = 1 up to rounding (eq:da_dino_trr_2 with Phi = Phi~ o Psi_r^*
       and Psi_r^* m^dagger = m_r^dagger, Prop. 5.1): the two-stage chain is
       the surrogate-only chain, transition for transition.
p-da2  Linear surrogate and a linear true model that also sees directions
       outside the reduced basis: the stationary law of the two-stage chain is
       the TRUE posterior, a Gaussian with closed-form mean and covariance
       (prior N(0, C_pr), C_pr = A^-2; y = G m + c + noise), which differs
       from the surrogate posterior; the ensemble moments after burn-in must
       match the former and miss the latter.  A wrong sign or a missing term
       in rho^(2) makes the chain sample something else.
"""
import numpy as np

from oracle import da, mlp, mmala, prior
from oracle.chains import OracleChains

GAMMA, DELTA = 0.1, 1.0


def _mlp(widths, act, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    Ws = [scale * rng.standard_normal((widths[l + 1], widths[l])) / np.sqrt(widths[l])
          for l in range(len(widths) - 1)]
    bs = [0.1 * rng.standard_normal(widths[l + 1]) for l in range(len(widths) - 1)]
    return Ws, bs


def test_da1_true_model_equal_to_surrogate_gives_rho2_one():
    n, r = 4, 5
    Ws, bs = _mlp([r, 7, 3], mlp.ACT_TANH, 3)
    y = np.random.default_rng(4).standard_normal(3)
    sur = mmala.Surrogate(Ws=Ws, bs=bs, act=mlp.ACT_TANH, y=y, noise_var=0.2)
    E, D = prior.kle_basis(n, GAMMA, DELTA, r)
    tm = da.TrueModel(Et=E, Ws=Ws, bs=bs, act=mlp.ACT_TANH)
    C, dt = 40, 0.3
    a = OracleChains(sur, E, D, n, GAMMA, DELTA, C, dt, seed=9, noise="cholesky")
    b = OracleChains(sur, E, D, n, GAMMA, DELTA, C, dt, seed=9, noise="cholesky", true_model=tm)
    assert np.allclose(b.phi_true, a.geo.phi, rtol=1e-12, atol=1e-12)
    n_acc = 0
    for _ in range(30):
        a.step()
        b.step()
        s1 = b.last["stage1"]
        assert np.array_equal(s1, a.last["accepted"])
        assert np.all(np.abs(b.last["log_rho2"][s1]) <= 1e-9 * np.maximum(1.0, b.last["phi_b"][s1]))
        assert np.array_equal(b.last["accepted"], a.last["accepted"])
        assert np.array_equal(a.m, b.m) and np.array_equal(a.m_r, b.m_r)
        n_acc += int(s1.sum())
    assert n_acc > 0


def _gauss_posterior(G, c, y, nv, Cpr):
    Cpost = np.linalg.inv(np.linalg.inv(Cpr) + G.T @ G / nv)
    return Cpost @ G.T @ (y - c) / nv, Cpost


def test_da2_linear_models_sample_the_true_posterior():
    n, r, rc = 3, 3, 2
    N = n * n
    E5, D5 = prior.kle_basis(n, GAMMA, DELTA, r + rc)
    E, D = E5[:r], D5[:, :r]
    dy, nv = 2, 0.5
    Ws, bs = _mlp([r, 4, dy], mlp.ACT_IDENTITY, 21)
    Wsur = Ws[1] @ Ws[0]
    csur = Ws[1] @ bs[0] + bs[1]
    V = 0.8 * np.random.default_rng(22).standard_normal((dy, rc))
    tm = da.TrueModel(Et=E5, Ws=[np.hstack([Wsur, V])], bs=[csur], act=mlp.ACT_IDENTITY)
    y = np.array([2.1, -3.3])
    sur = mmala.Surrogate(Ws=Ws, bs=bs, act=mlp.ACT_IDENTITY, y=y, noise_var=nv)
    A = prior.prior_operator(n, GAMMA, DELTA).toarray()
    Cpr = np.linalg.inv(A @ A)
    m_true, C_true = _gauss_posterior(tm.Ws[0] @ E5, csur, y, nv, Cpr)
    m_sur, C_sur = _gauss_posterior(Wsur @ E, csur, y, nv, Cpr)
    # the two targets differ by many Monte Carlo standard errors
    Lt = np.linalg.cholesky(C_true)
    assert np.abs(np.linalg.solve(Lt, m_sur - m_true)).max() > 0.4
    C, dt = 4000, 0.5
    ch = OracleChains(sur, E, D, n, GAMMA, DELTA, C, dt, seed=33, m0=np.zeros(N),
                      noise="cholesky", true_model=tm)
    s1, s2 = [], []
    for _ in range(80):
        ch.step()
        s1.append(ch.last["stage1"].mean())
        s2.append(ch.last["accepted"].mean())
    assert min(s1) == 1.0                                      # linear surrogate: rho^(1) = 1
    assert 0.2 < np.mean(s2) < 0.95                            # the second stage rejects some
    w = np.linalg.solve(Lt, (ch.m - m_true).T).T
    assert np.all(np.abs(w.mean(0)) < 5 / np.sqrt(C))
    assert np.abs(np.cov(w.T) - np.eye(N)).max() < 7 / np.sqrt(C)
    ws = np.linalg.solve(np.linalg.cholesky(C_sur), (ch.m - m_sur).T).T
    assert np.abs(ws.mean(0)).max() > 10 / np.sqrt(C)          # not the surrogate posterior
