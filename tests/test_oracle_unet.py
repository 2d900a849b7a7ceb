"""Pins of the learned-warm-start oracle (oracle/unet.py) against things other than itself.

- conv3 against scipy.ndimage.correlate (zero padding) and against plain loops;
- every backward against the adjoint (dot-product) identity or central finite
  differences;
- pool and up against their definitions;
- the subspace loss against a direct projection formula and its invariances;
- the first Adam step against its closed form.
"""
import itertools

import numpy as np
import pytest

from oracle import unet
import synthetic as syn

scipy_ndimage = pytest.importorskip("scipy.ndimage")


def rng(seed):
    return np.random.default_rng(seed)


def test_conv3_single_channel_is_zero_padded_correlation():
    N = 5
    X = rng(0).standard_normal((N ** 3, 1))
    K = rng(1).standard_normal((3, 3, 3))  # [dz][dy][dx]
    W = np.zeros((27, 1, 1))
    for t, (dx, dy, dz) in enumerate(unet.TAPS):
        W[t, 0, 0] = K[dz + 1, dy + 1, dx + 1]
    out = unet.conv3(X, N, W, np.array([0.25]))
    ref = scipy_ndimage.correlate(X.reshape(N, N, N), K, mode="constant", cval=0.0) + 0.25
    np.testing.assert_allclose(out.reshape(N, N, N), ref, atol=1e-13)


def test_conv3_multichannel_matches_plain_loops():
    N, ci, co = 4, 2, 3
    X = rng(2).standard_normal((N ** 3, ci))
    W = rng(3).standard_normal((27, ci, co))
    b = rng(4).standard_normal(co)
    out = unet.conv3(X, N, W, b)
    for iz, iy, ix in itertools.product(range(N), repeat=3):
        m = ix + N * (iy + N * iz)
        for o in range(co):
            s = b[o]
            for t, (dx, dy, dz) in enumerate(unet.TAPS):
                jx, jy, jz = ix + dx, iy + dy, iz + dz
                if 0 <= jx < N and 0 <= jy < N and 0 <= jz < N:
                    s += X[jx + N * (jy + N * jz)] @ W[t, :, o]
            assert out[m, o] == pytest.approx(s, abs=1e-12)


def test_conv3_backward_is_the_adjoint():
    N, ci, co = 6, 3, 2
    X = rng(5).standard_normal((N ** 3, ci))
    W = rng(6).standard_normal((27, ci, co))
    dZ = rng(7).standard_normal((N ** 3, co))
    dX, dW, db = unet.conv3_backward(X, N, W, dZ)
    zero = np.zeros(co)
    # <conv(X), dZ> = <X, dX> (linear in X) and = <W, dW> (linear in W)
    lhs = np.sum(unet.conv3(X, N, W, zero) * dZ)
    assert np.sum(X * dX) == pytest.approx(lhs, rel=1e-12)
    assert np.sum(W * dW) == pytest.approx(lhs, rel=1e-12)
    np.testing.assert_allclose(db, dZ.sum(axis=0), rtol=1e-13)


def test_pool_and_up_definitions_and_adjoints():
    N, c = 4, 2
    X = rng(8).standard_normal((N ** 3, c))
    Pm = unet.pool(X, N)
    G = X.reshape(N, N, N, c)
    for kz, ky, kx in itertools.product(range(N // 2), repeat=3):
        blk = G[2 * kz:2 * kz + 2, 2 * ky:2 * ky + 2, 2 * kx:2 * kx + 2].reshape(8, c)
        m = kx + (N // 2) * (ky + (N // 2) * kz)
        np.testing.assert_allclose(Pm[m], blk.mean(axis=0), atol=1e-14)
    Yc = rng(9).standard_normal(((N // 2) ** 3, c))
    U = unet.up(Yc, N // 2)
    for iz, iy, ix in itertools.product(range(N), repeat=3):
        np.testing.assert_array_equal(U[ix + N * (iy + N * iz)],
                                      Yc[ix // 2 + (N // 2) * (iy // 2 + (N // 2) * (iz // 2))])
    np.testing.assert_allclose(unet.pool(U, N), Yc, atol=1e-14)
    Yf = rng(10).standard_normal((N ** 3, c))
    assert np.sum(Pm * Yc) == pytest.approx(np.sum(X * unet.pool_backward(Yc, N)), rel=1e-12)
    assert np.sum(U * Yf) == pytest.approx(np.sum(Yc * unet.up_backward(Yf, N // 2)), rel=1e-12)


def test_silu_and_its_derivative():
    z = np.linspace(-8, 8, 41)
    np.testing.assert_allclose(unet.silu(z), z * (1 / (1 + np.exp(-z))), rtol=1e-15)
    assert unet.silu(np.array([0.0]))[0] == 0.0
    h = 1e-6
    fd = (unet.silu(z + h) - unet.silu(z - h)) / (2 * h)
    np.testing.assert_allclose(unet.silu_grad(z), fd, atol=1e-8)


def test_features_are_scaled_potential_and_box_coordinates():
    P = syn.warm_start_problem(1, N=8, p=4)
    F = unet.features(P.V, 8, P.lo, P.hi)
    np.testing.assert_allclose(F[:, 0], P.V / unet.V_SCALE)
    X = syn._mesh(P.shape, P.lo, P.hi)
    for d in range(3):
        np.testing.assert_allclose(F[:, 1 + d], X[d] / 8.0, atol=1e-14)  # box [-8, 8]


def small_net(seed=0, N=8, widths=(3, 4, 5), p=3):
    table = unet.layer_table(*widths, p)
    theta = syn.uniform_init(seed, unet.fans(table))
    P = syn.warm_start_problem(seed + 11, N=N, p=p)
    return theta, P, widths


def test_parameter_count_and_layout():
    table = unet.layer_table(24, 48, 96, 64)
    n = sum(t * ci * co + co for _, t, ci, co in table)
    # 27 x 32928 conv3 weights + 48 x 64 output weights + 592 biases: the ~1M-parameter
    # network of the 48^3 workload
    assert n == 27 * 32928 + 48 * 64 + 592 == 892720
    theta = np.arange(n, dtype=float)
    assert np.array_equal(unet.pack(unet.unpack(theta, table)), theta)


def test_network_gradient_matches_central_differences():
    theta, P, widths = small_net()
    p = 3
    R = rng(12).standard_normal((P.n, p))  # loss = <Y, R>

    def loss(th):
        return np.sum(unet.forward(th, P.V, 8, P.lo, P.hi, widths, p)[0] * R)

    Y, cache = unet.forward(theta, P.V, 8, P.lo, P.hi, widths, p)
    g = unet.backward(cache, R)
    eps = 1e-6
    for k in range(6):
        d = rng(100 + k).standard_normal(theta.size)
        fd = (loss(theta + eps * d) - loss(theta - eps * d)) / (2 * eps)
        assert np.dot(g, d) == pytest.approx(fd, rel=2e-7, abs=1e-9)
    # single coordinates in the first, a middle and the last layer
    for idx in (0, theta.size // 2, theta.size - 1):
        e = np.zeros(theta.size)
        e[idx] = 1.0
        fd = (loss(theta + eps * e) - loss(theta - eps * e)) / (2 * eps)
        assert g[idx] == pytest.approx(fd, rel=1e-6, abs=1e-8)


def test_subspace_loss_value_invariances_and_gradient():
    n, p, gamma = 200, 5, 0.1
    Us, _ = np.linalg.qr(rng(13).standard_normal((n, p)))
    Y = rng(14).standard_normal((n, p))
    L, dY = unet.subspace_loss(Y, Us, gamma)
    # L1 by explicit projection
    Rperp = Y - Us @ (Us.T @ Y)
    L1 = np.sum(Rperp ** 2) / np.sum(Y ** 2)
    G = Y.T @ Y
    L2 = np.sum((p * G / np.trace(G) - np.eye(p)) ** 2) / p ** 2
    assert L == pytest.approx(L1 + gamma * L2, rel=1e-13)
    Q, _ = np.linalg.qr(rng(15).standard_normal((p, p)))
    assert unet.subspace_loss(3.7 * Y @ Q, Us, gamma)[0] == pytest.approx(L, rel=1e-12)
    assert unet.subspace_loss(2.0 * Us @ Q, Us, gamma)[0] == pytest.approx(0.0, abs=1e-14)
    eps = 1e-6
    for k in range(4):
        D = rng(20 + k).standard_normal((n, p))
        fd = (unet.subspace_loss(Y + eps * D, Us, gamma)[0]
              - unet.subspace_loss(Y - eps * D, Us, gamma)[0]) / (2 * eps)
        assert np.sum(dY * D) == pytest.approx(fd, rel=1e-6, abs=1e-10)


def test_adam_first_step_closed_form():
    theta = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    th, m, v = unet.adam_step(theta, g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    # bias-corrected first step: m_hat = g, v_hat = g^2
    np.testing.assert_allclose(th, theta - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-14)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)
