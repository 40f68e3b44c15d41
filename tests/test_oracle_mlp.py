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


# Known values of a hand-written 2 -> 2 -> 1 network: W1 = [[1, -1], [0.5, 2]],
# b1 = [0.1, -0.2], W2 = [[2, -3]], b2 = [0.25] at x = (0.3, 0.7), so the hidden
# pre-activations are z = (-0.3, 1.35) and f = 2 s(-0.3) - 3 s(1.35) + 0.25,
# J = W2 diag(s'(z)) W1.  The numbers were evaluated once from these closed
# forms at 30 significant digits (arbitrary-precision tanh and erf); a bias
# added after the activation, a dropped bias or a transposed weight changes
# them in the second digit.
_KNOWN = {
    mlp.ACT_TANH: (-2.954785088561202874551505, [1.47622764874976700790838,
                                                 -3.246459023267223999740097]),
    mlp.ACT_GELU: (-3.670795781365150178026406, [-1.156669784365503845580935,
                                                 -7.303401469190916752434359]),
}


@pytest.mark.parametrize("kind", [mlp.ACT_TANH, mlp.ACT_GELU])
def test_nonlinear_forward_and_jacobian_known_values(kind):
    Ws = [np.array([[1.0, -1.0], [0.5, 2.0]]), np.array([[2.0, -3.0]])]
    bs = [np.array([0.1, -0.2]), np.array([0.25])]
    x = np.array([[0.3, 0.7]])
    f, zs = mlp.forward(Ws, bs, kind, x)
    f_ref, J_ref = _KNOWN[kind]
    assert abs(f[0, 0] - f_ref) <= 1e-15 * abs(f_ref)
    assert np.allclose(zs[0][0], [-0.3, 1.35], rtol=0, atol=1e-15)
    for J in (mlp.jacobian_reverse(Ws, kind, zs), mlp.jacobian_forward(Ws, kind, zs)):
        assert np.allclose(J[0, 0], J_ref, rtol=1e-15, atol=0)
