"""FP64 Gram and update on the tensor cores (exact digit products, op_fp64_gemm =
OP_GEMM_TC) against the oracle's products of the same FP64 data, through the C ABI.

Expected accuracy (from the arithmetic, see tests/test_fp64_digits.py): every term of a
contraction is exact up to 2^-53.4 |a| |b| and the digits round a by at most 2^-56 of the
largest |a| of its row, so an entry of a K-term product is within
c K 2^-53 max|a| max|b| of the exact sum (the error class of an FP64 dot product; the
oracle's numpy product adds its own FP64 rounding).  Small-integer operands give exact
products.  Sizes span several 128 x 64 tiles, ragged tails in both dimensions, one and
several K chunks of 256, and the p = 1024 width.
"""
import numpy as np
import pytest

import oracle as o
import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2511_06788_gb300 as pkg  # noqa: E402

DEV = torch.device("cuda:0")


def padded(A, ld):
    n, p = A.shape
    out = torch.zeros(n, ld, dtype=torch.float64, device=DEV)
    out[:, :p] = torch.from_numpy(np.ascontiguousarray(A)).to(DEV)
    return out


def ld_of(p):
    return (p + 7) // 8 * 8


def bound(X, Y, K):
    # c K 2^-53 max_k |x_ik| max_k |y_jk| per entry (rows i of X^T, j of Y^T)
    return 8.0 * K * 2.0 ** -53 * np.outer(np.abs(X).max(axis=0), np.abs(Y).max(axis=0)) + 1e-300


@pytest.mark.parametrize("n,p", [(1, 1), (257, 5), (3001, 72), (20011, 130), (50021, 257),
                                 (4099, 1024)])
def test_gram_fp64tc_matches_oracle(n, p):
    rng = np.random.default_rng(n + p)
    U = rng.standard_normal((n, p))
    W = rng.standard_normal((n, p)) * np.exp(rng.uniform(-4, 4, p))  # unequal column scales
    if p > 3:
        U[:, 1] = 0.0                                                # an all-zero column
        U[:, 2] *= 1e-30                                             # a tiny column
    ld = ld_of(p)
    Cm, Sm, Dm = pkg.binding.gram_fp64tc(padded(U, ld), padded(W, ld), p)
    for got, (X, Y) in ((Cm, (W, U)), (Sm, (W, W)), (Dm, (U, U))):
        g = got.cpu().numpy()
        ref = o.inner(X, Y)
        err = np.abs(g[:p, :p] - ref)
        assert np.all(err <= bound(X, Y, n)), float((err / bound(X, Y, n)).max())
        assert np.all(g[p:, :] == 0.0) and np.all(g[:, p:] == 0.0)
    assert np.array_equal(Dm.cpu().numpy(), Dm.cpu().numpy().T)


def test_gram_fp64tc_d_only_and_exact_integers():
    n, p = 9000, 40
    rng = np.random.default_rng(1)
    U = rng.integers(-9, 10, (n, p)).astype(np.float64)
    W = rng.integers(-9, 10, (n, p)).astype(np.float64)
    Cm, Sm, Dm = pkg.binding.gram_fp64tc(padded(U, 40), padded(W, 40), p)
    Ui, Wi = U.astype(np.int64), W.astype(np.int64)
    assert np.array_equal(Cm.cpu().numpy(), (Wi.T @ Ui).astype(np.float64))
    assert np.array_equal(Sm.cpu().numpy(), (Wi.T @ Wi).astype(np.float64))
    assert np.array_equal(Dm.cpu().numpy(), (Ui.T @ Ui).astype(np.float64))
    C2, S2, D2 = pkg.binding.gram_fp64tc(padded(U, 40), None, p, want=("D",))
    assert C2 is None and S2 is None and torch.equal(D2, Dm)


@pytest.mark.parametrize("n,p", [(1, 1), (1000, 8), (4097, 72), (20011, 130), (3001, 1024)])
def test_update_fp64tc_matches_oracle(n, p):
    rng = np.random.default_rng(n * p)
    U = rng.standard_normal((n, p))
    W = rng.standard_normal((n, p)) * 0.05
    KU = np.eye(p) + 0.1 * rng.standard_normal((p, p))
    KW = 3.0 * rng.standard_normal((p, p))
    ld = ld_of(p)
    sq = lambda K: padded(np.pad(K, ((0, ld - p), (0, 0))), ld)  # noqa: E731
    out = pkg.binding.update_fp64tc(padded(U, ld), padded(W, ld), sq(KU), sq(KW), p)
    got = out.cpu().numpy()
    ref = U @ KU + W @ KW
    # per output: 2p terms; rows of [U W] carry one exponent, columns of [KU - I; KW] one
    row = np.maximum(np.abs(U).max(axis=1), np.abs(W).max(axis=1))
    col = np.maximum(np.abs(KU - np.eye(p)).max(axis=0), np.abs(KW).max(axis=0))
    tol = 8.0 * 2 * p * 2.0 ** -53 * np.outer(row, col) + 4 * 2.0 ** -53 * np.abs(U)
    assert np.all(np.abs(got[:, :p] - ref) <= tol), float((np.abs(got[:, :p] - ref) / tol).max())
    assert np.all(got[:, p:] == 0.0)
    # W = None: Unew = U KU
    out2 = pkg.binding.update_fp64tc(padded(U, ld), None, sq(KU), None, p)
    ref2 = U @ KU
    tol2 = 8.0 * p * 2.0 ** -53 * np.outer(np.abs(U).max(axis=1),
                                          np.abs(KU - np.eye(p)).max(axis=0)) + \
        4 * 2.0 ** -53 * np.abs(U)
    assert np.all(np.abs(out2.cpu().numpy()[:, :p] - ref2) <= tol2)


def test_update_fp64tc_exact_for_integers():
    n, p = 5000, 24
    rng = np.random.default_rng(2)
    U = rng.integers(-20, 21, (n, p)).astype(np.float64)
    W = rng.integers(-20, 21, (n, p)).astype(np.float64)
    KU = rng.integers(-3, 4, (p, p)).astype(np.float64)
    KW = rng.integers(-3, 4, (p, p)).astype(np.float64)
    out = pkg.binding.update_fp64tc(padded(U, 24), padded(W, 24), padded(KU, 24), padded(KW, 24), p)
    ref = (U.astype(np.int64) @ KU.astype(np.int64) + W.astype(np.int64) @ KW.astype(np.int64))
    assert np.array_equal(out.cpu().numpy(), ref.astype(np.float64))


@pytest.mark.parametrize("geom", [((32, 32), (0.0, 0.0), (1.0, 1.0), 8),
                                  ((20, 22, 18), (-8.0,) * 3, (8.0,) * 3, 40)],
                         ids=["laplace2d_p8", "3d_p40"])
def test_fp64_steps_tc_and_fma_agree_with_oracle(geom):
    """Ten FP64 steps with the tensor-core products (and the mixed-precision Step 1 they
    select) and with FP64 FMA (plain FP64 CG), against the oracle's steps (exact Step 1) from
    the same U0: U within 1e-11 of max|U| and E within 1e-12 relative (each Step 1 stops at a
    relative residual of 1e-13 per column, so each step carries ~tau ||B|| 1e-13)."""
    shape, lo, hi, p = geom
    n = int(np.prod(shape))
    V = syn.potential(shape, lo, hi, 0.5, syn.draw_wells(3, 4, lo, hi)) if len(shape) == 3 \
        else np.zeros(n)
    U0 = syn.gaussian_block(5, n, p)
    H = o.hamiltonian(shape, lo, hi, V)
    sigma = o.default_sigma(shape, lo, hi, V)
    tau = o.default_tau(shape, lo, hi, V, sigma)
    U = o.householder_orthonormalize(U0)
    G = o.SourceSolver(H, sigma)
    for _ in range(10):
        U = o.scheme_step(U, G.solve(U), tau)
    res = {}
    for gemm in ("tc", "fma"):
        with pkg.Solver(shape, lo, hi, V, U0, p, prec="fp64", cg_rtol=1e-13, fp64_gemm=gemm) as s:
            st = s.step(10)
            res[gemm] = (s.get_U(), st)
    for gemm, (Ug, st) in res.items():
        assert np.abs(Ug - U).max() <= 1e-11 * np.abs(U).max(), gemm
        assert np.linalg.norm(Ug.T @ Ug - np.eye(p)) < 1e-13, gemm
        assert st["energy"] == pytest.approx(o.energy(H, U), rel=1e-12), gemm
