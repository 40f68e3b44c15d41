"""Pins of the oracle's prior, reduced bases and prior draws (CPU only).

Each check compares the closed forms against the sparse stencil operator, a
dense eigensolver or an exact identity of the paper (Lemma in Sec. 5.3).
"""
import numpy as np
import pytest

from oracle import prior
from workloads import dis_gaussian

GAMMA, DELTA = 0.1, 1.0


def _dense_A(n):
    return prior.prior_operator(n, GAMMA, DELTA).toarray()


def test_laplacian_stencil_values():
    n = 4
    Lap = prior.laplacian(n).toarray()
    h2 = prior.mesh_width(n) ** 2
    # corner node 0 has two neighbours (1 and n); interior diagonal is -4/h^2
    assert Lap[0, 0] == pytest.approx(-4 / h2)
    assert Lap[0, 1] == pytest.approx(1 / h2) and Lap[0, n] == pytest.approx(1 / h2)
    assert np.count_nonzero(Lap[0]) == 3
    p = 1 + n * 1
    assert np.count_nonzero(Lap[p]) == 5
    assert np.allclose(Lap, Lap.T)


@pytest.mark.parametrize("n", [3, 7, 12])
def test_sine_modes_are_eigenvectors_of_stencil(n):
    A = _dense_A(n)
    kappa, lam = prior.spectrum(n, GAMMA, DELTA)
    S = prior.sine_matrix(n)
    assert np.allclose(S @ S.T, np.eye(n), atol=1e-13)
    for kx in range(1, n + 1):
        for ky in range(1, n + 1):
            e = prior.eta(n, kx, ky)
            ev = DELTA + GAMMA * kappa[ky - 1, kx - 1]
            assert np.linalg.norm(A @ e - ev * e) < 1e-10 * ev
            assert lam[ky - 1, kx - 1] == pytest.approx(ev ** -2)


def test_kle_eigenvalues_match_dense_eigensolver():
    n, r = 7, 12
    A = _dense_A(n)
    Cpr = np.linalg.inv(A) @ np.linalg.inv(A)
    w = np.sort(np.linalg.eigvalsh(Cpr))[::-1]
    kx, ky = prior.kle_order(n, GAMMA, DELTA)
    _, lam = prior.spectrum(n, GAMMA, DELTA)
    lam_kle = lam[ky - 1, kx - 1]
    assert np.allclose(lam_kle, w, rtol=1e-10)
    # the first r modes span the dominant eigenspace when the cut does not split a tie
    if not np.isclose(lam_kle[r - 1], lam_kle[r], rtol=1e-12):
        _, V = np.linalg.eigh(Cpr)
        Vr = V[:, ::-1][:, :r]
        E, D = prior.kle_basis(n, GAMMA, DELTA, r)
        Pk = D @ E
        assert np.allclose(Pk @ Vr, Vr, atol=1e-10)


def test_kle_tie_rule_is_smaller_kx_first():
    # at n = 33 the pair (kx, ky) = (1, 5) / (5, 1) is tied and straddles r = 16
    kx, ky = prior.kle_order(33, GAMMA, DELTA)
    kappa, _ = prior.spectrum(33, GAMMA, DELTA)
    k = kappa[ky - 1, kx - 1]
    ties = [(i, i + 1) for i in range(len(k) - 1) if k[i] == k[i + 1]]
    assert ties
    for i, j in ties:
        assert kx[i] < kx[j]
    assert (kx[15], ky[15]) == (1, 5) and (kx[16], ky[16]) == (5, 1)


@pytest.mark.parametrize("kind", ["kle", "dis"])
def test_basis_is_cm_orthonormal_and_encoder_is_adjoint(kind):
    n, r = 6, 5
    A = _dense_A(n)
    if kind == "kle":
        E, D = prior.kle_basis(n, GAMMA, DELTA, r)
    else:
        E, D = prior.dis_basis(n, GAMMA, DELTA, dis_gaussian(n * n, r, 3))
    A2 = A @ A                                  # C_pr^-1
    assert np.allclose(E @ D, np.eye(r), atol=1e-12)                  # Psi^* Psi = I_r
    assert np.allclose(D.T @ A2 @ D, np.eye(r), atol=1e-10)           # <psi_j, psi_k>_{C^-1}
    assert np.allclose(E, D.T @ A2, atol=1e-9 * np.abs(E).max())       # encoder = <., psi>_{C^-1}


def test_dis_orthonormalisation_has_positive_R():
    n, r = 5, 4
    G = dis_gaussian(n * n, r, 8)
    E, D = prior.dis_basis(n, GAMMA, DELTA, G)
    Q = _dense_A(n) @ D
    assert np.allclose(Q.T @ Q, np.eye(r), atol=1e-12)
    R = Q.T @ G
    assert np.allclose(np.tril(R, -1), 0, atol=1e-12)
    assert np.all(np.diag(R) > 0)


def _prior_map(n):
    N = n * n
    return prior.prior_sample(n, GAMMA, DELTA, np.eye(N)).T   # column q = draw from e_q


def test_prior_draw_has_prior_covariance():
    n = 5
    T = _prior_map(n)
    Ainv = np.linalg.inv(_dense_A(n))
    assert np.allclose(T @ T.T, Ainv @ Ainv, atol=1e-14)


@pytest.mark.parametrize("kind", ["kle", "dis"])
def test_lemma_encoded_prior_is_white_and_complement_independent(kind):
    # Lemma (Sec. 5.3, eq:encoded_white_noise): Psi^* M ~ N(0, I_r) and
    # (I - Psi Psi^*) M is independent of Psi Psi^* M.
    n, r = 5, 4
    T = _prior_map(n)
    if kind == "kle":
        E, D = prior.kle_basis(n, GAMMA, DELTA, r)
    else:
        E, D = prior.dis_basis(n, GAMMA, DELTA, dis_gaussian(n * n, r, 5))
    C = T @ T.T
    assert np.allclose(E @ C @ E.T, np.eye(r), atol=1e-10)
    P = D @ E
    cross = (np.eye(n * n) - P) @ C @ P.T
    assert np.abs(cross).max() < 1e-12


def test_kle_encoding_of_prior_draw_is_leading_normals():
    n, r = 6, 7
    E, _ = prior.kle_basis(n, GAMMA, DELTA, r)
    z = np.random.default_rng(0).standard_normal(n * n)
    M = prior.prior_sample(n, GAMMA, DELTA, z)
    kx, ky = prior.kle_order(n, GAMMA, DELTA)
    q = (kx[:r] - 1) + n * (ky[:r] - 1)
    assert np.allclose(E @ M, z[q], atol=1e-12)
