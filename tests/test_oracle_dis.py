"""Pins of the surrogate-DIS construction (CPU only).

* linear surrogate f(x) = W x + c: J = W everywhere, so H_mc = W^T W /
  noise_var for any draws, and its eigenvalues are the squared singular
  values of W / sigma (a library SVD);
* the new basis satisfies E' D' = I and stays C_pr^-1-orthonormal
  (D'^T A^2 D' = I with C_pr = A^-2);
* a nonlinear surrogate: H_mc is the plain average of per-draw J^T J (brute
  force over the draws) and its leading eigenvector captures more of the
  average misfit curvature than any other unit vector tried.
"""
import numpy as np

from oracle import dis, mlp, mmala, prior

GAMMA, DELTA = 0.1, 1.0


def _sur(widths, act, seed, nv=0.3):
    rng = np.random.default_rng(seed)
    Ws = [rng.standard_normal((widths[l + 1], widths[l])) / np.sqrt(widths[l])
          for l in range(len(widths) - 1)]
    bs = [0.1 * rng.standard_normal(widths[l + 1]) for l in range(len(widths) - 1)]
    return mmala.Surrogate(Ws=Ws, bs=bs, act=act, y=np.zeros(widths[-1]), noise_var=nv)


def test_linear_surrogate_gives_singular_values():
    sur = _sur([6, 9, 4], mlp.ACT_IDENTITY, 1)
    W = sur.Ws[1] @ sur.Ws[0]
    x = dis.mc_draws(3, 17, 6)
    H = dis.expected_gnh(sur, x)
    assert np.allclose(H, W.T @ W / sur.noise_var, atol=1e-13)
    n, r = 4, 6
    E, D = prior.kle_basis(n, GAMMA, DELTA, r)
    lam, P, E2, D2 = dis.surrogate_dis(sur, E, D, x, 3)
    sv = np.linalg.svd(W / np.sqrt(sur.noise_var), compute_uv=False)
    assert np.allclose(lam[:4], sv ** 2, rtol=1e-12)
    assert np.allclose(lam[4:], 0.0, atol=1e-12)
    assert np.allclose(E2 @ D2, np.eye(3), atol=1e-12)
    A = prior.prior_operator(n, GAMMA, DELTA).toarray()
    assert np.allclose(D2.T @ A @ A @ D2, np.eye(3), atol=1e-10)


def test_nonlinear_average_and_leading_direction():
    sur = _sur([5, 12, 12, 3], mlp.ACT_GELU, 2)
    x = dis.mc_draws(7, 40, 5)
    H = dis.expected_gnh(sur, x)
    brute = np.zeros((5, 5))
    for xi in x:
        J = mmala.geometry(sur, xi[None, :]).J[0]
        brute += J.T @ J
    assert np.allclose(H, brute / (40 * sur.noise_var), rtol=1e-12)
    E, D = prior.kle_basis(3, GAMMA, DELTA, 5)
    lam, P, _, _ = dis.surrogate_dis(sur, E, D, x, 2)
    assert np.all(np.diff(lam) <= 0)
    v = P[:, 0]
    rng = np.random.default_rng(0)
    for _ in range(50):
        u = rng.standard_normal(5)
        u /= np.linalg.norm(u)
        assert u @ H @ u <= v @ H @ v + 1e-12
