"""Pins of the oracle's MLP, activations and Jacobians (CPU only)."""
import math

import numpy as np
import pytest

from oracle import mlp
from workloads import mlp_weights

# Standard normal CDF values: Phi(1) and Phi(-1)
PHI_1 = 0.8413447460685429
PHI_M1 = 0.15865525393145707


def test_gelu_known_values():
    z = np.array([0.0, 1.0, -1.0, 2.0])
    g = mlp.act(mlp.ACT_GELU, z)
    assert g[0] == 0.0
    assert g[1] == pytest.approx(PHI_1, abs=1e-15)
    assert g[2] == pytest.approx(-PHI_M1, abs=1e-15)
    assert g[3] == pytest.approx(2 * 0.5 * (1 + math.erf(2 / math.sqrt(2))), abs=1e-15)
    assert mlp.act_deriv(mlp.ACT_GELU, np.array([0.0]))[0] == 0.5


@pytest.mark.parametrize("kind", [mlp.ACT_IDENTITY, mlp.ACT_TANH, mlp.ACT_GELU])
def test_activation_derivative_by_central_difference(kind):
    z = np.linspace(-4, 4, 41)
    h = 1e-6
    fd = (mlp.act(kind, z + h) - mlp.act(kind, z - h)) / (2 * h)
    assert np.allclose(mlp.act_deriv(kind, z), fd, atol=1e-8)


@pytest.mark.parametrize("kind", [mlp.ACT_TANH, mlp.ACT_GELU])
@pytest.mark.parametrize("widths", [[3, 7, 5], [6, 8, 8, 4], [4, 5, 9]])
def test_jacobian_matches_central_finite_differences(kind, widths):
    Ws, bs = mlp_weights(widths, 21)
    x = np.random.default_rng(1).standard_normal(widths[0])
    f, zs = mlp.forward(Ws, bs, kind, x)
    J = mlp.jacobian_reverse(Ws, kind, zs)
    fd = np.empty_like(J)
    for k in range(widths[0]):
        h = 1e-5 * max(1.0, abs(x[k]))
        e = np.zeros_like(x)
        e[k] = h
        fp, _ = mlp.forward(Ws, bs, kind, x + e)
        fm, _ = mlp.forward(Ws, bs, kind, x - e)
        fd[:, k] = (fp - fm) / (2 * h)
    assert np.linalg.norm(J - fd) / np.linalg.norm(fd) < 1e-7


def test_forward_and_reverse_modes_agree_batched():
    widths = [5, 9, 9, 7]
    Ws, bs = mlp_weights(widths, 2)
    x = np.random.default_rng(4).standard_normal((6, 5))
    _, zs = mlp.forward(Ws, bs, mlp.ACT_GELU, x)
    Jr = mlp.jacobian_reverse(Ws, mlp.ACT_GELU, zs)
    Jf = mlp.jacobian_forward(Ws, mlp.ACT_GELU, zs)
    assert Jr.shape == (6, 7, 5)
    assert np.allclose(Jr, Jf, rtol=0, atol=1e-13 * np.abs(Jr).max())


def test_identity_network_is_composed_affine_map():
    widths = [4, 6, 3]
    Ws, bs = mlp_weights(widths, 9)
    x = np.random.default_rng(3).standard_normal(4)
    f, zs = mlp.forward(Ws, bs, mlp.ACT_IDENTITY, x)
    W = Ws[1] @ Ws[0]
    c = Ws[1] @ bs[0] + bs[1]
    assert np.allclose(f, W @ x + c, atol=1e-14)
    assert np.allclose(mlp.jacobian_reverse(Ws, mlp.ACT_IDENTITY, zs), W, atol=1e-14)
