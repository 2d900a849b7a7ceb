"""Planted mistakes in the learned-warm-start oracle (oracle/unet.py) must be caught
by its pins (tests/test_oracle_unet.py).  Each case swaps one function for a copy
with a plausible mistake, on the CPU and inside this process only, and runs the
pin that should catch it."""
import numpy as np
import pytest

from oracle import unet
from tests import test_oracle_unet as pins

ORIG = {name: getattr(unet, name) for name in
        ("shifted", "conv3_backward", "silu_grad", "pool_backward", "up_backward",
         "subspace_loss", "adam_step")}


def shifted_wrong_direction(X, N, tap):
    dx, dy, dz = unet.TAPS[tap]  # reads X[m - off]: a convolution, not a correlation
    Xp = np.pad(X.reshape(N, N, N, X.shape[1]), ((1, 1), (1, 1), (1, 1), (0, 0)))
    return Xp[1 - dz:1 - dz + N, 1 - dy:1 - dy + N, 1 - dx:1 - dx + N, :].reshape(N ** 3, -1)


def conv3_backward_wrong_direction(X, N, W, dZ):
    dW = np.stack([unet.shifted(X, N, t).T @ dZ for t in range(27)])
    db = dZ.sum(axis=0)
    dXp = np.zeros((N + 2, N + 2, N + 2, X.shape[1]))
    for t, (dx, dy, dz) in enumerate(unet.TAPS):  # scattered to m - off instead of m + off
        dXp[1 - dz:1 - dz + N, 1 - dy:1 - dy + N, 1 - dx:1 - dx + N, :] += \
            (dZ @ W[t].T).reshape(N, N, N, -1)
    return dXp[1:-1, 1:-1, 1:-1, :].reshape(N ** 3, -1), dW, db


def silu_grad_missing_term(z):
    return 1.0 / (1.0 + np.exp(-z))  # dropped the z s (1 - s) term


def pool_backward_unscaled(dY, N):
    return ORIG["pool_backward"](dY, N) * 8.0


def up_backward_dropped(dY, M):
    return np.zeros((M ** 3, dY.shape[1]))  # the decoder's gradient never reaches the encoder


def loss_missing_y_term(Y, Ustar, gamma):
    L, dY = ORIG["subspace_loss"](Y, Ustar, gamma)
    G = Y.T @ Y
    P = Ustar.T @ Y
    b = np.trace(G)
    return L, dY - Y * (2.0 * np.sum(P * P) / b ** 2)  # dropped 2 ||P||^2 / b^2 Y


def adam_without_bias_correction(theta, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    return theta - lr * m / (np.sqrt(v) + eps), m, v


CASES = [
    ("shifted", shifted_wrong_direction,
     pins.test_conv3_single_channel_is_zero_padded_correlation),
    ("conv3_backward", conv3_backward_wrong_direction, pins.test_conv3_backward_is_the_adjoint),
    ("silu_grad", silu_grad_missing_term, pins.test_silu_and_its_derivative),
    ("pool_backward", pool_backward_unscaled, pins.test_pool_and_up_definitions_and_adjoints),
    ("up_backward", up_backward_dropped, pins.test_network_gradient_matches_central_differences),
    ("subspace_loss", loss_missing_y_term, pins.test_subspace_loss_value_invariances_and_gradient),
    ("adam_step", adam_without_bias_correction, pins.test_adam_first_step_closed_form),
]


@pytest.mark.parametrize("name,mutant,pin", CASES, ids=[c[0] for c in CASES])
def test_unet_mutant_is_caught(monkeypatch, name, mutant, pin):
    monkeypatch.setattr(unet, name, mutant)
    with pytest.raises(AssertionError):
        pin()


def test_unmutated_pins_pass():
    for _, _, pin in CASES:
        pin()
