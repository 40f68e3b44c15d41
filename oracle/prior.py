"""Gaussian prior, reduced bases and prior draws on a 2D grid (oracle).

TEST INFRASTRUCTURE ONLY (see `oracle/__init__.py`).

Discretisation (a reading: the paper's experiments use FEM with Robin
conditions, Secs. 7.1 and 8.2; the workloads here use the finite-difference
form below):

* n x n interior nodes of the unit square, h = 1/(n+1), node p = i + n j with
  x = (i+1) h, y = (j+1) h;
* Lap_h = the 5-point Dirichlet stencil divided by h^2;
* A = delta I - gamma Lap_h, the prior covariance C_pr = A^-2 (Assumption 2,
  Sec. 2.2), Euclidean inner product on R^N.

The eigenpairs of C_pr are closed-form: the 1D sine vectors
v_k(i) = sqrt(2/(n+1)) sin(k (i+1) pi/(n+1)) diagonalise the 1D stencil with
eigenvalue -s_k, s_k = (4/h^2) sin^2(k pi h/2); eta_{kx,ky} = v_kx (x) v_ky and
lambda = (delta + gamma (s_kx + s_ky))^-2.  The KLE order (Sec. 4.2) is by
decreasing lambda; ties (which the cut at r can split) are broken by the
smaller kx first.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def mesh_width(n: int) -> float:
    return 1.0 / (n + 1)


def laplacian(n: int) -> sp.csr_matrix:
    """5-point Dirichlet Laplacian on the n x n interior grid, scaled by 1/h^2."""
    h = mesh_width(n)
    T = sp.diags([np.ones(n - 1), -2.0 * np.ones(n), np.ones(n - 1)], [-1, 0, 1])
    I = sp.identity(n)
    # node p = i + n j: x varies fastest
    return ((sp.kron(I, T) + sp.kron(T, I)) / (h * h)).tocsr()


def prior_operator(n: int, gamma: float, delta: float) -> sp.csr_matrix:
    """A = delta I - gamma Lap_h; the prior covariance is A^-2."""
    return (delta * sp.identity(n * n) - gamma * laplacian(n)).tocsr()


def sine_matrix(n: int) -> np.ndarray:
    """S[k-1, i] = sqrt(2/(n+1)) sin(k (i+1) pi / (n+1)); symmetric and orthogonal."""
    k = np.arange(1, n + 1)[:, None]
    i = np.arange(1, n + 1)[None, :]
    return np.sqrt(2.0 / (n + 1)) * np.sin(k * i * np.pi / (n + 1))


def lap1d_eigs(n: int) -> np.ndarray:
    """s_k = (4/h^2) sin^2(k pi h / 2), k = 1..n: minus the eigenvalues of the 1D stencil."""
    h = mesh_width(n)
    k = np.arange(1, n + 1)
    return 4.0 / (h * h) * np.sin(k * np.pi * h / 2.0) ** 2


def spectrum(n: int, gamma: float, delta: float):
    """kappa[ky-1, kx-1] = s_kx + s_ky and lambda = (delta + gamma kappa)^-2 (2D arrays)."""
    s = lap1d_eigs(n)
    kappa = s[None, :] + s[:, None]          # [ky-1, kx-1]
    lam = (delta + gamma * kappa) ** -2
    return kappa, lam


def kle_order(n: int, gamma: float, delta: float):
    """Modes (kx, ky) by decreasing lambda (increasing kappa), ties -> smaller kx first."""
    kappa, _ = spectrum(n, gamma, delta)
    ky, kx = np.meshgrid(np.arange(1, n + 1), np.arange(1, n + 1), indexing="ij")
    kx = kx.ravel()
    ky = ky.ravel()
    kap = kappa.ravel()
    order = np.lexsort((kx, kap))            # primary key kappa, secondary kx
    return kx[order], ky[order]


def eta(n: int, kx: int, ky: int) -> np.ndarray:
    """Euclidean-normalised eigenvector eta_{kx,ky}(p = i + n j) = v_kx(i) v_ky(j)."""
    S = sine_matrix(n)
    return np.outer(S[ky - 1], S[kx - 1]).ravel()     # row j, column i


def kle_basis(n: int, gamma: float, delta: float, r: int):
    """KLE reduced basis of rank r (Sec. 4.2): psi_j = sqrt(lambda_j) eta_j.

    Returns (E, D): the encoder Psi_r^* (r x N), whose rows are
    <., psi_j>_{C_pr^-1} = eta_j^T / sqrt(lambda_j), and the decoder Psi_r
    (N x r) with columns psi_j (eq:projector, Sec. 4).
    """
    kx, ky = kle_order(n, gamma, delta)
    _, lam = spectrum(n, gamma, delta)
    N = n * n
    E = np.empty((r, N))
    D = np.empty((N, r))
    for j in range(r):
        e = eta(n, kx[j], ky[j])
        l = lam[ky[j] - 1, kx[j] - 1]
        E[j] = e / np.sqrt(l)
        D[:, j] = np.sqrt(l) * e
    return E, D


def dis_basis(n: int, gamma: float, delta: float, G: np.ndarray):
    """Stand-in for a derivative-informed basis: C_pr^-1-orthonormalised Gaussian vectors.

    Q = thin QR factor of G with positive diag(R); psi_j = A^-1 q_j so that
    <psi_j, psi_k>_{C_pr^-1} = q_j^T q_k = delta_jk (the orthonormality that
    eq:jtj_eigenvalue imposes).  Encoder E = Psi^T C_pr^-1 = Q^T A, decoder
    D = A^-1 Q.
    """
    Q, R = np.linalg.qr(G, mode="reduced")
    Q = Q * np.sign(np.diag(R))[None, :]
    A = prior_operator(n, gamma, delta)
    D = spla.splu(A.tocsc()).solve(np.ascontiguousarray(Q))
    E = np.asarray((A @ Q).T)
    return E, D


def prior_sample(n: int, gamma: float, delta: float, z: np.ndarray) -> np.ndarray:
    """Prior draw M ~ N(0, C_pr) from the full Karhunen-Loeve expansion (Sec. 4.2).

    M = sum_{kx,ky} sqrt(lambda_{kx,ky}) z_{kx,ky} eta_{kx,ky}, with the
    standard normal z indexed q = (kx-1) + n (ky-1).  In matrix form
    M[j, i] = (S^T (sqrt(Lambda) * Z) S)[j, i].  `z` has shape (..., N).
    """
    S = sine_matrix(n)
    _, lam = spectrum(n, gamma, delta)
    Z = np.asarray(z, dtype=np.float64).reshape(z.shape[:-1] + (n, n))   # [.., ky-1, kx-1]
    M = S.T @ (np.sqrt(lam) * Z) @ S                                     # [.., j, i]
    return M.reshape(z.shape)
