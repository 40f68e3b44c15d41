"""Philox4x32-10 counter-based generator and the normals drawn from it (oracle).

TEST INFRASTRUCTURE ONLY (see `oracle/__init__.py`).

The paper does not fix a random number generator.  Both the oracle and the
CUDA library implement the same counter-based generator from its published
definition -- Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, "Parallel
random numbers: as easy as 1, 2, 3", SC'11) -- so that every random number a
chain draws is a pure function of (seed, stream, step, chain, index):

    key     = (seed mod 2^32, seed >> 32)
    counter = (block, step, chain, stream)

One block yields four 32-bit words x0..x3.  A word maps to a uniform on (0, 1)
by u = (x + 1/2) 2^-32 (exact in float64); (u0, u1) and (u2, u3) give two
pairs of standard normals by the Box-Muller transform, so block k carries the
normals 4k .. 4k+3.

Streams: XI (reduced proposal noise of Algorithm 1), U (the uniform of its
accept test), Z (prior draw for the complement, Prop. 5.1), INIT (prior draw
of the initial state), XI2 (the d_y observation-space normals of the
perturbation noise map, see `mmala.reduced_proposal_perturbation`), U2 (the
uniform of the second, true-model stage of delayed acceptance, Algorithm 1).
"""
from __future__ import annotations

import numpy as np

STREAM_XI = 0
STREAM_U = 1
STREAM_Z = 2
STREAM_INIT = 3
STREAM_XI2 = 4
STREAM_U2 = 5

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)
_SH = np.uint64(32)


def philox4x32_10(counter, key):
    """Ten Philox rounds on `counter` (..., 4) uint32 under `key` (..., 2) uint32.

    Each round multiplies words 0 and 2 by the two Philox multipliers, splits the
    64-bit products into high and low halves, and permutes/xors them with words
    1 and 3 and the round key; the key is bumped by the two Weyl constants
    between rounds (SC'11, Sec. 3.2).
    """
    counter = np.asarray(counter, dtype=np.uint32)
    key = np.asarray(key, dtype=np.uint32)
    c0, c1, c2, c3 = (counter[..., i].astype(np.uint64) for i in range(4))
    k0 = key[..., 0].astype(np.uint64)
    k1 = key[..., 1].astype(np.uint64)
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
        p0 = c0 * _M0
        p1 = c2 * _M1
        c0, c1, c2, c3 = ((p1 >> _SH) ^ c1 ^ k0, p1 & _MASK,
                          (p0 >> _SH) ^ c3 ^ k1, p0 & _MASK)
    return np.stack([c0, c1, c2, c3], axis=-1).astype(np.uint32)


def _key(seed: int):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32)


def blocks(seed: int, stream: int, step: int, chains, n_blocks: int) -> np.ndarray:
    """Words of blocks 0..n_blocks-1 for each chain id: shape (C, n_blocks, 4) uint32."""
    chains = np.asarray(chains, dtype=np.uint64).reshape(-1)
    C = chains.shape[0]
    ctr = np.zeros((C, n_blocks, 4), dtype=np.uint32)
    ctr[..., 0] = np.arange(n_blocks, dtype=np.uint32)[None, :]
    ctr[..., 1] = np.uint32(int(step) & 0xFFFFFFFF)
    ctr[..., 2] = chains.astype(np.uint32)[:, None]
    ctr[..., 3] = np.uint32(stream)
    return philox4x32_10(ctr, _key(seed))


def word_to_uniform(x) -> np.ndarray:
    """u = (x + 1/2) 2^-32 in (0, 1), exact in float64."""
    return (np.asarray(x, dtype=np.float64) + 0.5) * 2.0 ** -32


def normals(seed: int, stream: int, step: int, chains, count: int) -> np.ndarray:
    """`count` standard normals per chain via Box-Muller: shape (C, count) float64."""
    nb = (count + 3) // 4
    u = word_to_uniform(blocks(seed, stream, step, chains, nb))   # (C, nb, 4)
    rad01 = np.sqrt(-2.0 * np.log(u[..., 0]))
    rad23 = np.sqrt(-2.0 * np.log(u[..., 2]))
    th01 = 2.0 * np.pi * u[..., 1]
    th23 = 2.0 * np.pi * u[..., 3]
    out = np.stack([rad01 * np.cos(th01), rad01 * np.sin(th01),
                    rad23 * np.cos(th23), rad23 * np.sin(th23)], axis=-1)
    return out.reshape(out.shape[0], nb * 4)[:, :count]


def uniform(seed: int, stream: int, step: int, chains) -> np.ndarray:
    """One uniform per chain: word 0 of block 0.  Shape (C,)."""
    return word_to_uniform(blocks(seed, stream, step, chains, 1)[:, 0, 0])
