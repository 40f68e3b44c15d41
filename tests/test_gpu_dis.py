"""Surrogate-driven DIS basis on the device against the oracle (GPU).

The Monte Carlo Gauss-Newton average over encoded prior draws, its
eigenvalues, the leading eigenvectors (compared up to sign, where the
spectrum separates them) and the rotated basis E' = P^T E, D' = D P.
"""
import numpy as np
import pytest

from helpers import gpu_setup, oracle_setup
from oracle import dis
from workloads import CONFIGS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dino():
    import paper_2403_08220_gb300 as d
    return d


@pytest.fixture(scope="module")
def ctx(dino):
    c = dino.dino_init(0)
    yield c
    c.close()


@pytest.mark.parametrize("name,n,r_new,tol", [("small_fp64", 100, 6, 1e-10),
                                              ("r200_kle_fp64", 48, 20, 1e-10),
                                              ("r200_dis_bf16", 48, 20, 1e-4)])
def test_dis_from_surrogate_matches_oracle(dino, ctx, name, n, r_new, tol):
    w = CONFIGS[name]
    sid = gpu_setup(dino, ctx, w)
    sur, E, D = oracle_setup(w)
    out = dino.dino_dis_from_surrogate(ctx, sid, n, 77, r_new, w.r, w.N)
    lam, P, E2, D2 = dis.surrogate_dis(sur, E, D, dis.mc_draws(77, n, w.r), r_new)
    assert np.all(np.diff(out["eigvals"]) <= 0)
    assert np.max(np.abs(out["eigvals"] - lam)) <= tol * lam[0]
    # leading eigenvectors, up to sign, where the gap to both neighbours is clear
    gaps = np.minimum(np.abs(np.diff(lam, prepend=np.inf)), np.abs(np.diff(lam, append=-np.inf)))
    sep = np.where(gaps[:r_new] > 1e-3 * lam[0])[0]
    assert len(sep) >= r_new // 2
    sgn = np.sign(np.sum(out["P"] * P, axis=0))
    vt = 10 * np.sqrt(tol) if tol > 1e-9 else 1e-7
    assert np.max(np.abs(out["P"][:, sep] * sgn[sep] - P[:, sep])) <= vt
    assert np.max(np.abs(out["D"][:, sep] * sgn[sep] - D2[:, sep])) <= vt * np.abs(D2).max()
    assert np.max(np.abs(out["E"][sep] * sgn[sep, None] - E2[sep])) <= vt * np.abs(E2).max()
    # the new basis is a basis pair: E' D' = I
    assert np.max(np.abs(out["E"] @ out["D"] - np.eye(r_new))) <= 1e-9
    dino.dino_unload_surrogate(ctx, sid)
