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
