"""FP64 CPU oracle of the learned warm start: a 3-level convolutional U-Net that
maps the potential V to an n x p block, a rotation-invariant subspace loss
against a converged block U*, the hand-derived backward pass and Adam.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  The paper has no
network; this is the learned-warm-start extension of the scheme.  The network
only has to put U^0 in the basin of the scheme's fixed point.  The basin
condition on the energy, E(U^0) below the excited-state level (§3), is what a
good warm start buys; the scheme itself is unchanged and decides the result.

Tensors are channels-last, [grid point][channel], on an N^3 grid (N % 4 == 0).
Point (ix, iy, iz) has index ix + N (iy + N iz), the orbital-block ordering.

  x0  = [V / v_scale, xhat, yhat, zhat]          xhat in (-1, 1): box coordinate
  e0a = silu(conv3(x0))          4      -> c0     N^3
  e0  = silu(conv3(e0a))         c0     -> c0
  e1a = silu(conv3(pool(e0)))    c0     -> c1     (N/2)^3
  e1  = silu(conv3(e1a))         c1     -> c1
  b2a = silu(conv3(pool(e1)))    c1     -> c2     (N/4)^3
  b2  = silu(conv3(b2a))         c2     -> c2
  d1a = silu(conv3([up(b2), e1]))  c2+c1 -> c1    (N/2)^3
  d1  = silu(conv3(d1a))         c1     -> c1
  d0a = silu(conv3([up(d1), e0]))  c1+c0 -> c1    N^3
  d0  = silu(conv3(d0a))         c1     -> c1
  Y   = conv1(d0)                c1     -> p      (linear output)

- conv3 is the 3x3x3 cross-correlation with zero padding plus a bias:
  out[m] = b + sum over taps t of in[m + off_t] W[t], where W[t] is Cin x Cout and
  tap t = (dz+1)*9 + (dy+1)*3 + (dx+1).
- pool is the 2x2x2 mean; up is nearest-neighbour (x2); [a, b] concatenates
  channels.
- silu(z) = z / (1 + exp(-z)).

Parameters are one flat vector: per layer in the table order, W (taps x Cin x
Cout, row-major) and then b (Cout).
"""
from __future__ import annotations

import numpy as np

TAPS = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
CIN = 4          # input features: V / v_scale and the three box coordinates
V_SCALE = 6.0    # depth scale of the potential


def layer_table(c0: int, c1: int, c2: int, p: int):
    """(name, taps, Cin, Cout) of every layer, in parameter order."""
    return [("e0a", 27, CIN, c0), ("e0", 27, c0, c0), ("e1a", 27, c0, c1), ("e1", 27, c1, c1),
            ("b2a", 27, c1, c2), ("b2", 27, c2, c2), ("d1a", 27, c2 + c1, c1),
            ("d1", 27, c1, c1), ("d0a", 27, c1 + c0, c1), ("d0", 27, c1, c1),
            ("out", 1, c1, p)]


def fans(table):
    """(fan_in, weights, biases) per layer: the input of synthetic.uniform_init."""
    return [(t * ci, t * ci * co, co) for _, t, ci, co in table]


def unpack(theta: np.ndarray, table):
    out, off = [], 0
    for _, t, ci, co in table:
        W = theta[off:off + t * ci * co].reshape(t, ci, co)
        off += t * ci * co
        b = theta[off:off + co]
        off += co
        out.append((W, b))
    assert off == theta.size
    return out


def pack(parts) -> np.ndarray:
    return np.concatenate([np.concatenate([W.reshape(-1), b]) for W, b in parts])


# ---------------------------------------------------------------------------
# Layers and their adjoints
# ---------------------------------------------------------------------------
def features(V: np.ndarray, N: int, lo, hi) -> np.ndarray:
    """[V / V_SCALE, xhat, yhat, zhat] per grid point; xhat = 2 (x - lo) / (hi - lo) - 1."""
    hats = []
    for d in range(3):
        h = (hi[d] - lo[d]) / (N + 1)
        x = lo[d] + (np.arange(N) + 1.0) * h
        hats.append(2.0 * (x - lo[d]) / (hi[d] - lo[d]) - 1.0)
    iz, iy, ix = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    return np.stack([V.reshape(-1) / V_SCALE, hats[0][ix.reshape(-1)],
                     hats[1][iy.reshape(-1)], hats[2][iz.reshape(-1)]], axis=1)


def _grid(X, N):
    return X.reshape(N, N, N, X.shape[1])  # [iz][iy][ix][c]


def shifted(X: np.ndarray, N: int, tap: int) -> np.ndarray:
    """Rows X[m + off_tap] (zero outside the grid), as an N^3 x C array."""
    dx, dy, dz = TAPS[tap]
    Xp = np.pad(_grid(X, N), ((1, 1), (1, 1), (1, 1), (0, 0)))
    return Xp[1 + dz:1 + dz + N, 1 + dy:1 + dy + N, 1 + dx:1 + dx + N, :].reshape(N ** 3, -1)


def conv3(X, N, W, b):
    out = np.zeros((N ** 3, W.shape[2])) + b
    for t in range(27):
        out += shifted(X, N, t) @ W[t]
    return out


def conv3_backward(X, N, W, dZ):
    """(dX, dW, db) of out = conv3(X) given dZ = d loss / d out."""
    dW = np.stack([shifted(X, N, t).T @ dZ for t in range(27)])
    db = dZ.sum(axis=0)
    dXp = np.zeros((N + 2, N + 2, N + 2, X.shape[1]))
    for t, (dx, dy, dz) in enumerate(TAPS):
        # out[m] used X[m + off]: the adjoint scatters dZ[m] W[t]^T to m + off
        dXp[1 + dz:1 + dz + N, 1 + dy:1 + dy + N, 1 + dx:1 + dx + N, :] += \
            _grid(dZ @ W[t].T, N)
    return dXp[1:-1, 1:-1, 1:-1, :].reshape(N ** 3, -1), dW, db


def pool(X, N):
    M = N // 2
    return X.reshape(M, 2, M, 2, M, 2, -1).mean(axis=(1, 3, 5)).reshape(M ** 3, -1)


def pool_backward(dY, N):
    M = N // 2
    g = dY.reshape(M, 1, M, 1, M, 1, -1) / 8.0
    return np.broadcast_to(g, (M, 2, M, 2, M, 2, dY.shape[1])).reshape(N ** 3, -1)


def up(X, M):
    """Nearest-neighbour upsampling of an M^3 grid to (2M)^3."""
    g = X.reshape(M, 1, M, 1, M, 1, -1)
    return np.broadcast_to(g, (M, 2, M, 2, M, 2, X.shape[1])).reshape(8 * M ** 3, -1)


def up_backward(dY, M):
    return dY.reshape(M, 2, M, 2, M, 2, -1).sum(axis=(1, 3, 5)).reshape(M ** 3, -1)


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


# ---------------------------------------------------------------------------
# Network
# ---------------------------------------------------------------------------
def forward(theta, V, N, lo, hi, widths, p):
    """Y (N^3 x p) and the cache for backward()."""
    c0, c1, c2 = widths
    table = layer_table(c0, c1, c2, p)
    P = dict(zip([t[0] for t in table], unpack(theta, table)))
    cache = {"N": N, "table": table, "P": P}
    grids = {"e0a": N, "e0": N, "e1a": N // 2, "e1": N // 2, "b2a": N // 4, "b2": N // 4,
             "d1a": N // 2, "d1": N // 2, "d0a": N, "d0": N}

    def layer(name, X):
        Z = conv3(X, grids[name], *P[name])
        cache[name] = (X, Z)
        return silu(Z)

    x0 = features(V, N, lo, hi)
    e0 = layer("e0", layer("e0a", x0))
    e1 = layer("e1", layer("e1a", pool(e0, N)))
    b2 = layer("b2", layer("b2a", pool(e1, N // 2)))
    d1 = layer("d1", layer("d1a", np.concatenate([up(b2, N // 4), e1], axis=1)))
    d0 = layer("d0", layer("d0a", np.concatenate([up(d1, N // 2), e0], axis=1)))
    Wo, bo = P["out"]
    cache["out"] = d0
    return d0 @ Wo[0] + bo, cache


def backward(cache, dY):
    """Gradient of the loss with respect to the flat parameter vector, given dY."""
    N, table, P = cache["N"], cache["table"], cache["P"]
    c1 = P["e1"][0].shape[2]
    grads = {}
    grids = {"e0a": N, "e0": N, "e1a": N // 2, "e1": N // 2, "b2a": N // 4, "b2": N // 4,
             "d1a": N // 2, "d1": N // 2, "d0a": N, "d0": N}

    def layer_back(name, dA):
        X, Z = cache[name]
        dZ = dA * silu_grad(Z)
        dX, dW, db = conv3_backward(X, grids[name], P[name][0], dZ)
        grads[name] = (dW, db)
        return dX

    d0 = cache["out"]
    Wo = P["out"][0]
    grads["out"] = ((d0.T @ dY)[None], dY.sum(axis=0))
    g = layer_back("d0a", layer_back("d0", dY @ Wo[0].T))        # d [up(d1), e0]
    g_d1 = up_backward(g[:, :c1], N // 2)
    g_e0 = g[:, c1:].copy()
    g = layer_back("d1a", layer_back("d1", g_d1))                 # d [up(b2), e1]
    c2 = P["b2"][0].shape[2]
    g_b2 = up_backward(g[:, :c2], N // 4)
    g_e1 = g[:, c2:].copy()
    g = layer_back("b2a", layer_back("b2", g_b2))                 # d pool(e1)
    g_e1 += pool_backward(g, N // 2)
    g = layer_back("e1a", layer_back("e1", g_e1))                 # d pool(e0)
    g_e0 += pool_backward(g, N)
    layer_back("e0a", layer_back("e0", g_e0))
    return pack([grads[name] for name, *_ in table])


# ---------------------------------------------------------------------------
# Subspace loss
# ---------------------------------------------------------------------------
def subspace_loss(Y, Ustar, gamma):
    """Rotation- and scale-invariant distance of span(Y) from span(U*), U* orthonormal.

    With G = Y^T Y, P = U*^T Y, b = tr G and Gh = p G / b:
      L1 = 1 - ||P||_F^2 / b        (share of ||Y||^2 outside span U*)
      L2 = ||Gh - I||_F^2 / p^2     (columns orthogonal and of equal norm)
      L  = L1 + gamma L2
    L = 0 exactly when Y = c U* Q, Q orthogonal.  Returns (L, dL/dY) with
      dL/dY = Y [2 ||P||^2 / b^2 I + gamma 4 / (p b) ((Gh - I) - tr((Gh - I) G) / b I)]
              - U* (2 / b) P.
    """
    p = Y.shape[1]
    G = Y.T @ Y
    P = Ustar.T @ Y
    b = np.trace(G)
    pp = np.sum(P * P)
    Gh = p * G / b
    E = Gh - np.eye(p)
    L1 = 1.0 - pp / b
    L2 = np.sum(E * E) / p ** 2
    KY = (2.0 * pp / b ** 2) * np.eye(p) + gamma * (4.0 / (p * b)) * (
        E - (np.sum(E * G) / b) * np.eye(p))
    KU = -(2.0 / b) * P
    return L1 + gamma * L2, Y @ KY + Ustar @ KU


# ---------------------------------------------------------------------------
# Adam (Kingma and Ba, ICLR 2015, Algorithm 1)
# ---------------------------------------------------------------------------
def adam_step(theta, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update at step t >= 1; returns (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
