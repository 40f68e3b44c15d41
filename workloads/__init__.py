"""Seeded synthetic inputs shared by the oracle and the CUDA library's tests.

This module holds shapes and random numbers only: no step of the sampler's
arithmetic lives here.  It produces

* the MLP weights of a reduced-basis surrogate (LeCun-normal W, N(0, 0.1^2) b),
* the Gaussian matrix G that the DIS stand-in basis orthonormalises,
* the reduced coordinates of a synthetic truth and the data-noise draw,
* the recipe that turns a noiseless observable vector into data
  (noise standard deviation = a fraction of its RMS).

Seeds follow one convention: basis=11, weights=12, truth=13, data noise=14,
chains=15, true-model weights=16 (plus a request index for serving workloads).

The workloads mirror the shapes of the paper's experiments (Secs. 7-8: a
reduced basis of rank 200, GELU MLPs of width 400, tens to hundreds of
observations) on a synthetic 2D prior of (delta I - gamma Laplacian)^-2 type,
since the paper's PDE data and trained weights are not available.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Tuple

import numpy as np

ACT_IDENTITY = 0
ACT_TANH = 1
ACT_GELU = 2

BASIS_KLE = 0
BASIS_DIS = 1
BASIS_EXPLICIT = 2

SEED_BASIS = 11
SEED_WEIGHTS = 12
SEED_TRUTH = 13
SEED_DATA_NOISE = 14
SEED_CHAINS = 15
SEED_TRUE = 16


@dataclass
class Workload:
    """One synthetic posterior plus the chain ensemble that samples it."""
    name: str
    n_grid: int                 # interior nodes per side; N = n_grid**2
    r: int                      # reduced dimension
    widths: List[int]           # widths[0] = r, widths[-1] = d_y
    activation: int
    basis_kind: int
    n_chains: int
    n_steps: int
    dt: float = 0.5
    prior_gamma: float = 0.1
    prior_delta: float = 1.0
    noise_frac: float = 0.01    # sigma = noise_frac * RMS(noiseless observables)
    precision: str = "fp64"
    seed_offset: int = 0        # added to every seed (serving requests)
    # proposal noise map the chains use: "cholesky" (L^-T xi), "perturbation"
    # ((I + H)^-1 (xi + K^T xi2)) or "auto" (the library's choice, reported by
    # dino_surrogate_query); both are the same proposal law
    noise_map: str = "auto"

    @property
    def N(self) -> int:
        return self.n_grid * self.n_grid

    @property
    def d_y(self) -> int:
        return self.widths[-1]


# The five workloads: shapes follow the paper's experiments scaled to a 2D grid.
CONFIGS = {
    "small_fp64": Workload("small_fp64", n_grid=33, r=16, widths=[16, 64, 64, 49],
                           activation=ACT_TANH, basis_kind=BASIS_KLE,
                           n_chains=64, n_steps=200, noise_map="cholesky"),
    "r200_kle_fp64": Workload("r200_kle_fp64", n_grid=65, r=200, widths=[200, 400, 400, 100],
                              activation=ACT_GELU, basis_kind=BASIS_KLE,
                              n_chains=4096, n_steps=1000, noise_map="perturbation"),
    "r200_dis_bf16": Workload("r200_dis_bf16", n_grid=65, r=200, widths=[200, 400, 400, 100],
                              activation=ACT_GELU, basis_kind=BASIS_DIS,
                              n_chains=16384, n_steps=1000, precision="bf16",
                              noise_map="perturbation"),
    # the paper's network shape (Sec. 7-8: six hidden layers of 400 GELU units,
    # r = 200 DIS; d_y = 25 and 64 observations, N of about 1681 and 2145)
    "paper_ndr_bf16": Workload("paper_ndr_bf16", n_grid=41, r=200,
                               widths=[200] + [400] * 6 + [25], activation=ACT_GELU,
                               basis_kind=BASIS_DIS, n_chains=16384, n_steps=1000,
                               precision="bf16", noise_map="perturbation"),
    "paper_hyper_bf16": Workload("paper_hyper_bf16", n_grid=46, r=200,
                                 widths=[200] + [400] * 6 + [64], activation=ACT_GELU,
                                 basis_kind=BASIS_DIS, n_chains=16384, n_steps=1000,
                                 precision="bf16", noise_map="perturbation"),
}


def heterogeneous_workloads() -> List[Workload]:
    """Eight posteriors of different size batched together (r from 32 to 400)."""
    rs = [32, 64, 100, 128, 200, 256, 320, 400]
    chains = [8192, 8192, 4096, 4096, 2048, 2048, 1024, 512]
    out = []
    for i, (r, c) in enumerate(zip(rs, chains)):
        d_y = 50 * (i + 1)
        out.append(Workload(f"hetero_{i}", n_grid=65, r=r, widths=[r, 2 * r, 2 * r, d_y],
                            activation=ACT_GELU, basis_kind=BASIS_DIS, n_chains=c,
                            n_steps=1000, precision="bf16", seed_offset=100 * i))
    return out


def mlp_weights(widths, seed: int) -> Tuple[List[np.ndarray], List[np.ndarray]]:
    """W_l ~ N(0, 1/fan_in) of shape (widths[l+1], widths[l]); b_l ~ N(0, 0.1^2)."""
    rng = np.random.default_rng(seed)
    Ws, bs = [], []
    for l in range(len(widths) - 1):
        fan_in, fan_out = widths[l], widths[l + 1]
        Ws.append(rng.standard_normal((fan_out, fan_in)) / np.sqrt(fan_in))
        bs.append(0.1 * rng.standard_normal(fan_out))
    return Ws, bs


def dis_gaussian(N: int, r: int, seed: int) -> np.ndarray:
    """The N x r standard-normal matrix whose orthonormalisation gives the DIS stand-in."""
    return np.random.default_rng(seed).standard_normal((N, r))


def truth_reduced(r: int, seed: int) -> np.ndarray:
    """Reduced coordinates of the synthetic truth: N(0, I_r), the law of an encoded prior draw."""
    return np.random.default_rng(seed).standard_normal(r)


def data_noise(d_y: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(d_y)


def make_data(y0: np.ndarray, eps: np.ndarray, noise_frac: float) -> Tuple[np.ndarray, float]:
    """Data = noiseless observables + sigma * eps with sigma = noise_frac * RMS(y0).

    Returns (y, noise_var) with noise_var = sigma^2 (Gamma = sigma^2 I).
    """
    sigma = noise_frac * float(np.sqrt(np.mean(np.asarray(y0) ** 2)))
    return np.asarray(y0) + sigma * np.asarray(eps), sigma * sigma


def surrogate_inputs(w: Workload):
    """Everything random a surrogate of workload `w` needs, from the seed convention."""
    Ws, bs = mlp_weights(w.widths, SEED_WEIGHTS + w.seed_offset)
    G = dis_gaussian(w.N, w.r, SEED_BASIS + w.seed_offset) if w.basis_kind == BASIS_DIS else None
    m_true_r = truth_reduced(w.r, SEED_TRUTH + w.seed_offset)
    eps = data_noise(w.d_y, SEED_DATA_NOISE + w.seed_offset)
    return dict(Ws=Ws, bs=bs, G=G, m_true_r=m_true_r, eps=eps)


def true_model_weights(w: Workload, r_c: int, eps: float):
    """Weights of the true-map stand-in f_t of delayed acceptance for workload
    `w`: the surrogate's network whose first layer also reads r_c further
    coordinates (the encoder's extra rows) through eps V, V seeded
    N(0, 1/r_c), so that f_t(x, x_c) = f(x) + O(eps)."""
    inp = surrogate_inputs(w)
    V = np.random.default_rng(SEED_TRUE + w.seed_offset).standard_normal(
        (w.widths[1], r_c)) / np.sqrt(r_c)
    Ws = [np.hstack([inp["Ws"][0], eps * V])] + [x.copy() for x in inp["Ws"][1:]]
    return Ws, [x.copy() for x in inp["bs"]]
