"""op_gram_noalloc: the Gram matrices without any device allocation.

Some callers cannot let this library allocate device memory or give it a
workspace (all device memory belongs to another allocator with a hard budget,
or the calling loop may not enter the driver's allocator).  op_gram_noalloc
keeps its reduction partials in a fixed library-owned device array instead.
These tests call it through the C ABI and compare it with op_gram on the same
inputs, twice in a row with different data (the array keeps the previous
call's contents, which must not leak into the next result).  This file is
named to be collected last.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2511_06788_gb300 as pkg  # noqa: E402

DEV = torch.device("cuda:0")


def _blocks(seed, n, p, ld, dtype):
    g = torch.Generator(device=DEV).manual_seed(seed)
    U = torch.zeros(n, ld, dtype=dtype, device=DEV)
    W = torch.zeros(n, ld, dtype=dtype, device=DEV)
    U[:, :p] = torch.randn(n, p, dtype=torch.float64, device=DEV, generator=g).to(dtype)
    W[:, :p] = 0.3 * torch.randn(n, p, dtype=torch.float64, device=DEV, generator=g).to(dtype)
    return U, W


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["fp64", "fp32"])
def test_noalloc_gram_matches_op_gram_twice(dtype):
    n, p, ld = 50021, 100, 104
    for call, seed in enumerate((11, 12)):
        U, W = _blocks(seed, n, p, ld, dtype)
        ref = pkg.gram(U, W, p)
        got = pkg.binding.gram_noalloc(U, W, p)
        Uh, Wh = U.double().cpu().numpy(), W.double().cpu().numpy()
        # both are within the dot-product rounding bound of the exact result; the two
        # differ only in how the grid points are split into chunks
        if dtype == torch.float64:
            scale = 2.0 * 2.2e-16 * math.sqrt(n)
        else:
            scale = 4.0 * 6e-8 * math.sqrt(2048) + 2.0 ** -21
        for a, b, (X, Y) in zip(ref, got, ((Wh, Uh), (Wh, Wh), (Uh, Uh))):
            bound = 2.0 * scale * (np.abs(X).T @ np.abs(Y)) + 1e-300
            diff = np.abs(a.cpu().numpy() - b.cpu().numpy())
            assert np.all(diff <= bound), (call, float(diff.max()))
            exact = X.T @ Y
            assert np.all(np.abs(b.cpu().numpy() - exact) <= bound)


def test_noalloc_gram_subset_of_products():
    n, p, ld = 7001, 40, 40
    U, W = _blocks(3, n, p, ld, torch.float32)
    C_ref, _, _ = pkg.gram(U, W, p, want=("C",))
    C, S, D = pkg.binding.gram_noalloc(U, W, p, want=("C",))
    assert S is None and D is None
    assert torch.allclose(C, C_ref, rtol=0, atol=1e-3)


def test_noalloc_gram_rejects_sizes_beyond_its_scratch():
    n, p, ld = 1000, 1024, 1024
    U = torch.zeros(n, ld, dtype=torch.float32, device=DEV)
    with pytest.raises(pkg.OpError) as e:
        pkg.binding.gram_noalloc(U, U, p)
    assert e.value.status == pkg.binding.OP_ERR_ARG
    assert "fixed scratch" in str(e.value)


def test_noalloc_gram_allocates_nothing():
    # after a first call (which may load the library's module and its array), a further
    # call leaves the device's free memory unchanged
    n, p, ld = 20011, 64, 64
    U, W = _blocks(5, n, p, ld, torch.float32)
    pkg.binding.gram_noalloc(U, W, p)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    pkg.binding.gram_noalloc(U, W, p)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_gram_fp64_size_limit():
    # FP64: 64 x 64 tiles; with all three products ld = 960 fits the array, 968 does not
    n = 300
    U = torch.zeros(n, 960, dtype=torch.float64, device=DEV)
    U[:, :960] = torch.randn(n, 960, dtype=torch.float64, device=DEV)
    C, S, D = pkg.binding.gram_noalloc(U, U, 960)
    Uh = U.cpu().numpy()
    assert np.abs(D.cpu().numpy() - Uh.T @ Uh).max() <= 1e-12 * n
    V = torch.zeros(n, 968, dtype=torch.float64, device=DEV)
    with pytest.raises(pkg.OpError) as e:
        pkg.binding.gram_noalloc(V, V, 968)
    assert e.value.status == pkg.binding.OP_ERR_ARG


def test_noalloc_gram_fp32_widest_blocks_over_a_million_points():
    """ld = 896 (the widest FP32 blocks that fit) over n > 10^6 grid points: the chunks
    are op_gram's (here 5 chunks of 200032 points per output tile), so every entry is
    within the FP32 rounding bound of that run length, (64 + 200032 / 32) 2^-24 sum |x y|
    (a 32-point slab on the tensor cores, then one FP32 addition per slab), checked
    against FP64 sums on sampled entries, and equal to op_gram's up to the order of the
    FP64 chunk sums."""
    n, p, ld = 1_000_003, 896, 896
    U, W = _blocks(21, n, p, ld, torch.float32)
    got = pkg.binding.gram_noalloc(U, W, p)
    ref = pkg.gram(U, W, p)
    run = 200032 // 32
    bound_scale = (64 + run) * 2.0 ** -24
    rng = np.random.default_rng(3)
    for M, R, (X, Y) in zip(got, ref, ((W, U), (W, W), (U, U))):
        Mh, Rh = M.cpu().numpy(), R.cpu().numpy()
        assert np.abs(Mh - Rh).max() <= 1e-9 * np.abs(Rh).max()
        for i, j in rng.integers(0, p, (48, 2)):
            x, y = X[:, i].double(), Y[:, j].double()
            exact = float((x * y).sum())
            mag = float((x.abs() * y.abs()).sum())
            assert abs(Mh[i, j] - exact) <= bound_scale * mag, (i, j, Mh[i, j], exact)
