"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances.  FP64 kernels: the same arithmetic up to summation order, so
entries agree to a few ulps of the magnitudes involved (1e-13 relative to the
operand scale).  FP32 kernels are compared with the FP64 oracle evaluated on
the same FP32-rounded inputs, to FP32 rounding of the operand scale (a few
1e-6 relative; error analysis: one stencil row is a 7-term FP32 sum, a Gram or
update entry an FP32 sum over <= 256 terms flushed to FP64).  Whole solves:
eigenvalues to 1e-10 relative in FP64 (the target of the FP64 mode) and to
1e-5 in FP32.
"""
import math

import numpy as np
import pytest

import oracle as o
import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU runs deselect -m gpu anyway
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2511_06788_gb300 as pkg  # noqa: E402

DEV = torch.device("cuda:0")
DT = {"fp64": torch.float64, "fp32": torch.float32, "mix_bf16x3": torch.float32}


def padded(A, ld, dtype):
    n, p = A.shape
    out = torch.zeros(n, ld, dtype=dtype, device=DEV)
    out[:, :p] = torch.from_numpy(np.ascontiguousarray(A)).to(DEV, dtype)
    return out


def ld_of(p):
    return (p + 7) // 8 * 8


def rounded(A, prec):
    return A.astype(np.float32).astype(np.float64) if prec != "fp64" else A


def mode_of(prec):
    """The prec argument of pkg.gram / pkg.update (None: by the dtype)."""
    return prec if prec == "mix_bf16x3" else None


GEOMS = [
    ((32, 32), (0.0, 0.0), (1.0, 1.0), 8),                   # the 2D Laplace workload
    ((7, 5, 3), (-1.0, -1.0, -1.0), (1.3, 0.9, 1.1), 5),     # tiny, anisotropic, ragged ld
    ((33, 17), (0.0, -1.0), (2.0, 1.0), 13),                 # 2D, ragged
    ((20, 22, 18), (-8.0,) * 3, (8.0,) * 3, 40),             # 3D, several row blocks
    ((9, 8, 7), (-2.0,) * 3, (2.0,) * 3, 300),               # wide rows (p > 256)
]


def random_potential(shape, lo, hi, seed):
    rng = np.random.default_rng(seed)
    wells = syn.draw_wells(seed, 3, lo, hi) if len(shape) == 3 else []
    V = syn.potential(shape, lo, hi, 0.5, wells) if wells else rng.uniform(-1, 2, int(np.prod(shape)))
    return V


# ----------------------------------------------------------------------------
# Kernel-level parity
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("geom", GEOMS, ids=lambda g: "x".join(map(str, g[0])) + f"_p{g[3]}")
def test_apply_H_matches_oracle(prec, geom):
    shape, lo, hi, p = geom
    n = int(np.prod(shape))
    V = random_potential(shape, lo, hi, 1)
    X = rounded(np.random.default_rng(2).standard_normal((n, p)), prec)
    Vr = rounded(V, prec)
    sigma = 0.75
    H = o.hamiltonian(shape, lo, hi, Vr)
    ref = H @ X + sigma * X
    ld = ld_of(p)
    Y = pkg.apply_H(shape, lo, hi, torch.from_numpy(Vr).to(DEV, DT[prec]), sigma,
                    padded(X, ld, DT[prec]))
    Yh = Y.double().cpu().numpy()
    scale = o.gershgorin_norm(shape, lo, hi, Vr, sigma) * np.abs(X).max()
    tol = 1e-14 if prec == "fp64" else 4e-7
    assert np.abs(Yh[:, :p] - ref).max() <= tol * scale
    assert np.all(Yh[:, p:] == 0.0)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "mix_bf16x3"])
@pytest.mark.parametrize("n,p", [(1, 3), (100, 8), (5003, 72), (20000, 136), (777, 257)])
def test_gram_matches_oracle(prec, n, p):
    rng = np.random.default_rng(n + p)
    U = rounded(rng.standard_normal((n, p)), prec)
    W = rounded(rng.standard_normal((n, p)), prec)
    ld = ld_of(p)
    Cm, Sm, Dm = pkg.gram(padded(U, ld, DT[prec]), padded(W, ld, DT[prec]), p,
                          prec=mode_of(prec))
    # rounding bound of a dot product: c * eps * sqrt(run length) * sum_k |x_k y_k|.
    # FP64: whole chunks in FP64.  FP32 (tensor cores, 4xTF32 or 6xBF16 from three-piece
    # splits): products to ~2^-21, FP32 accumulation over chunks of <= 2048 grid points,
    # chunks summed in FP64.
    if prec == "fp64":
        scale = 2.0 * 2.2e-16 * math.sqrt(n)
    else:
        scale = 4.0 * 6e-8 * math.sqrt(min(n, 2048)) + 2.0 ** -21
    for got, (X, Y) in ((Cm, (W, U)), (Sm, (W, W)), (Dm, (U, U))):
        g = got.cpu().numpy()
        ref = o.inner(X, Y)
        bound = scale * (np.abs(X).T @ np.abs(Y)) + 1e-300
        assert np.all(np.abs(g[:p, :p] - ref) <= bound)
        assert np.all(g[p:, :] == 0.0) and np.all(g[:, p:] == 0.0)


def test_gram_subset_and_symmetry():
    rng = np.random.default_rng(5)
    U = rng.standard_normal((3000, 70))
    Cm, Sm, Dm = pkg.gram(padded(U, 72, torch.float64), padded(U, 72, torch.float64), 70,
                          want=("D",))
    assert Cm is None and Sm is None
    D = Dm.cpu().numpy()
    assert np.array_equal(D, D.T)


def _core_inputs(seed, p):
    shape, lo, hi = (6, 5, 4), (-1.0,) * 3, (1.0, 1.2, 0.9)
    rng = np.random.default_rng(seed)
    V = rng.uniform(-2, 3, 120)
    H = o.hamiltonian(shape, lo, hi, V)
    sigma = o.default_sigma(shape, lo, hi, V)
    U = o.householder_orthonormalize(rng.standard_normal((120, p)))
    W = o.SourceSolver(H, sigma).solve(U)
    return U, W, o.default_tau(shape, lo, hi, V, sigma)


def _core_on_gpu(W, U, tau):
    p = U.shape[1]
    ld = ld_of(p)
    C = np.zeros((ld, ld))
    S = np.zeros((ld, ld))
    C[:p, :p], S[:p, :p] = o.inner(W, U), o.inner(W, W)
    KU, KW, KU_t, KW_t = pkg.core(torch.from_numpy(C).to(DEV), torch.from_numpy(S).to(DEV), p, tau)
    ku, kw = KU.cpu().numpy(), KW.cpu().numpy()
    assert np.all(ku[p:, :] == 0) and np.all(kw[:, p:] == 0)
    return ku[:p, :p], kw[:p, :p]


@pytest.mark.parametrize("p", [1, 5, 17, 67])
@pytest.mark.parametrize("tau_scale", [0.1, 1.0, 30.0])
def test_core_matches_oracle(p, tau_scale):
    """Exact W = GU: the device core equals the paper's Steps 2-3 (oracle)."""
    U, W, tau = _core_inputs(p, p)
    tau *= tau_scale
    ku, kw = _core_on_gpu(W, U, tau)
    KU_ref, KW_ref = o.step_coefficients(W, U, tau)
    assert np.abs(ku - KU_ref).max() <= 1e-12 * max(1.0, np.abs(KU_ref).max())
    assert np.abs(kw - KW_ref).max() <= 1e-12 * max(1.0, np.abs(KW_ref).max())


@pytest.mark.parametrize("p", [3, 40, 129])
def test_core_inexact_W_matches_midpoint_solution(p):
    """Arbitrary W (an inexact Step 1): the device core is the exact solution of (4.1)."""
    rng = np.random.default_rng(p)
    U = o.householder_orthonormalize(rng.standard_normal((400, p)))
    W = 0.2 * rng.standard_normal((400, p))
    tau = 3.0
    ku, kw = _core_on_gpu(W, U, tau)
    A, B = o.midpoint_coefficients(W, U, tau)
    np.testing.assert_allclose(kw, tau * B, atol=1e-12)
    np.testing.assert_allclose(ku, np.eye(p) - tau * A, atol=1e-11)
    assert o.orth_error(U @ ku + W @ kw) < 1e-12


def test_core_reports_breakdown():
    # C = 2 I, S = 0, tau = 1: M = I + (1/4)(0 - 4 I) = 0 exactly (not a Gram of a real W)
    p, ld = 3, 8
    C = np.zeros((ld, ld))
    S = np.zeros((ld, ld))
    C[:p, :p] = 2.0 * np.eye(p)
    with pytest.raises(pkg.OpError) as e:
        pkg.core(torch.from_numpy(C).to(DEV), torch.from_numpy(S).to(DEV), p, 1.0)
    assert e.value.status == pkg.binding.OP_ERR_NOTSPD
    C[0, 0] = np.nan
    with pytest.raises(pkg.OpError):
        pkg.core(torch.from_numpy(C).to(DEV), torch.from_numpy(S).to(DEV), p, 1.0)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "mix_bf16x3"])
# ld a multiple of 32 (p = 90, 128, 256) takes the TMA-fed tensor-core kernel for FP32:
# a ragged last column tile (90 -> ld 96), more tiles than SMs (20000 x 128) and two
# column tiles (256)
@pytest.mark.parametrize("n,p", [(1, 1), (999, 8), (4097, 40), (3001, 130), (5000, 90),
                                 (20000, 128), (3001, 256)])
def test_update_matches_oracle(prec, n, p):
    rng = np.random.default_rng(n * p)
    U = rounded(rng.standard_normal((n, p)), prec)
    W = rounded(rng.standard_normal((n, p)), prec)
    KU = rounded(rng.standard_normal((p, p)), prec)
    KW = rounded(rng.standard_normal((p, p)), prec)
    ld = ld_of(p)
    out = pkg.update(padded(U, ld, DT[prec]), padded(W, ld, DT[prec]), _square(KU, ld, DT[prec]),
                     _square(KW, ld, DT[prec]), p, prec=mode_of(prec))
    ref = U @ KU + W @ KW
    got = out.double().cpu().numpy()
    tol = (1e-14 if prec == "fp64" else 1e-6) * 2 * p * 4
    assert np.abs(got[:, :p] - ref).max() <= tol
    assert np.all(got[:, p:] == 0)


def _square(K, ld, dtype):
    p = K.shape[0]
    out = torch.zeros(ld, ld, dtype=dtype, device=DEV)
    out[:p, :p] = torch.from_numpy(np.ascontiguousarray(K)).to(DEV, dtype)
    return out


@pytest.mark.parametrize("precond", ["none", "jacobi"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_cg_solve_matches_oracle(prec, precond):
    shape, lo, hi, p = (20, 22, 18), (-8.0,) * 3, (8.0,) * 3, 12
    n = int(np.prod(shape))
    V = rounded(random_potential(shape, lo, hi, 3), prec)
    sigma = o.default_sigma(shape, lo, hi, V)
    U = rounded(o.householder_orthonormalize(syn.gaussian_block(4, n, p)), prec)
    H = o.hamiltonian(shape, lo, hi, V)
    W_ref = o.SourceSolver(H, sigma).solve(U)
    ld = ld_of(p)
    Ut, Wt = padded(U, ld, DT[prec]), torch.zeros(n, ld, dtype=DT[prec], device=DEV)
    rtol = 1e-12 if prec == "fp64" else 1e-6
    it = pkg.cg_solve(shape, lo, hi, torch.from_numpy(V).to(DEV, DT[prec]), sigma, Ut, Wt, p, rtol,
                      precond=precond)
    assert 0 < it < 5000
    W = Wt.double().cpu().numpy()
    # ||W - G U|| <= ||G|| ||residual|| <= (1/lambda_min(H + sigma)) rtol ||u||
    err = np.linalg.norm(W[:, :p] - W_ref, axis=0)
    lam_min = o.spectrum_lower_bound(shape, lo, hi, V) + sigma
    assert np.all(err <= 30 * rtol / lam_min)
    assert np.all(W[:, p:] == 0)


# 3-D grids with >= 32 columns run the TMA plane-marching CG kernels: ragged
# x/y tiles, a ragged 32-column chunk, the thinnest z extent they accept.
TMA_GEOMS = [((13, 9, 11), 40), ((16, 16, 16), 64), ((9, 8, 3), 33), ((20, 22, 18), 96)]


@pytest.mark.parametrize("geom", TMA_GEOMS, ids=lambda g: "x".join(map(str, g[0])) + f"_p{g[1]}")
def test_cg_plane_marching_iterates_match_oracle(geom):
    """W after k CG iterations (warm start) equals the oracle's block CG after k iterations."""
    shape, p = geom
    lo, hi = (-4.0,) * 3, (4.0,) * 3
    n = int(np.prod(shape))
    V = rounded(random_potential(shape, lo, hi, 5), "fp32")
    sigma = o.default_sigma(shape, lo, hi, V)
    U = rounded(o.householder_orthonormalize(syn.gaussian_block(6, n, p)), "fp32")
    W0 = rounded(0.05 * syn.gaussian_block(7, n, p), "fp32")
    A = (o.hamiltonian(shape, lo, hi, V) + sigma * sp_identity(n)).tocsr()
    ld = ld_of(p)
    Vt = torch.from_numpy(V).to(DEV, torch.float32)
    Ut = padded(U, ld, torch.float32)
    for k in (1, 2, 5):
        Wt = padded(W0, ld, torch.float32)
        it = pkg.cg_solve(shape, lo, hi, Vt, sigma, Ut, Wt, p, 1e-30, max_iter=k)
        assert it == k
        W = Wt.double().cpu().numpy()
        W_ref, _ = o.block_cg(A, U, W0, rtol=0.0, max_iter=k)
        err = np.abs(W[:, :p] - W_ref).max() / np.abs(W_ref).max()
        assert err < 2e-5, (k, err)
        assert np.all(W[:, p:] == 0)
    # and to convergence
    Wt = padded(W0, ld, torch.float32)
    it = pkg.cg_solve(shape, lo, hi, Vt, sigma, Ut, Wt, p, 1e-6)
    W_exact = o.SourceSolver(o.hamiltonian(shape, lo, hi, V), sigma).solve(U)
    lam_min = o.spectrum_lower_bound(shape, lo, hi, V) + sigma
    err = np.linalg.norm(Wt.double().cpu().numpy()[:, :p] - W_exact, axis=0)
    assert 0 < it < 5000 and np.all(err <= 30 * 1e-6 / lam_min)


@pytest.mark.parametrize("prec,geom", [("fp32", TMA_GEOMS[0]), ("fp32", TMA_GEOMS[3]),
                                       ("fp32", ((17, 15), 24)), ("fp64", ((13, 9, 11), 40)),
                                       ("fp64", ((17, 15), 12))],
                         ids=lambda g: g if isinstance(g, str) else
                         "x".join(map(str, g[0])) + f"_p{g[1]}")
def test_jacobi_cg_iterates_match_oracle(prec, geom):
    """W after k Jacobi-preconditioned CG iterations equals the oracle's block_pcg_jacobi
    after k iterations (3-D FP32: TMA direction kernel; 2-D FP32: row kernels; FP64:
    the three-kernel iteration)."""
    shape, p = geom
    lo, hi = (-4.0,) * len(shape), (4.0,) * len(shape)
    n = int(np.prod(shape))
    V = rounded(random_potential(shape, lo, hi, 5), prec)
    sigma = o.default_sigma(shape, lo, hi, V)
    U = rounded(o.householder_orthonormalize(syn.gaussian_block(6, n, p)), prec)
    W0 = rounded(0.05 * syn.gaussian_block(7, n, p), prec)
    A = (o.hamiltonian(shape, lo, hi, V) + sigma * sp_identity(n)).tocsr()
    ld = ld_of(p)
    Vt = torch.from_numpy(V).to(DEV, DT[prec])
    Ut = padded(U, ld, DT[prec])
    tol = 2e-5 if prec == "fp32" else 1e-12
    for k in (1, 2, 5):
        Wt = padded(W0, ld, DT[prec])
        it = pkg.cg_solve(shape, lo, hi, Vt, sigma, Ut, Wt, p, 1e-30, max_iter=k,
                          precond="jacobi")
        assert it == k
        W = Wt.double().cpu().numpy()
        W_ref, _ = o.block_pcg_jacobi(A, U, W0, rtol=0.0, max_iter=k)
        err = np.abs(W[:, :p] - W_ref).max() / np.abs(W_ref).max()
        assert err < tol, (k, err)
        assert np.all(W[:, p:] == 0)
    # to convergence: the stopping test is on the unpreconditioned (recursively updated)
    # residual; in FP32 the true residual of the result also carries the rounding of
    # the updates, so it is checked like the plain CG's: through the solution error
    # ||W - G U|| <= ||G|| ||residual|| <= rtol ||u|| / lambda_min(H + sigma)
    rtol = 1e-6 if prec == "fp32" else 1e-12
    Wt = padded(W0, ld, DT[prec])
    it = pkg.cg_solve(shape, lo, hi, Vt, sigma, Ut, Wt, p, rtol, precond="jacobi")
    W = Wt.double().cpu().numpy()[:, :p]
    _, it_ref = o.block_pcg_jacobi(A, U, W0, rtol=rtol)
    assert abs(it - it_ref) <= (3 if prec == "fp32" else 1), (it, it_ref)
    W_exact = o.SourceSolver(o.hamiltonian(shape, lo, hi, V), sigma).solve(U)
    lam_min = o.spectrum_lower_bound(shape, lo, hi, V) + sigma
    err = np.linalg.norm(W - W_exact, axis=0)
    assert np.all(err <= 30 * rtol / lam_min), err.max()
    if prec == "fp64":
        res = np.linalg.norm(U - A @ W, axis=0) / np.linalg.norm(U, axis=0)
        assert np.all(res <= 1.5 * rtol), res.max()


def sp_identity(n):
    import scipy.sparse as sp
    return sp.identity(n, format="csr")


# ----------------------------------------------------------------------------
# Whole-step and whole-solve parity through the context API
# ----------------------------------------------------------------------------
def _oracle_steps(P, U0, nsteps):
    H = o.hamiltonian(P.shape, P.lo, P.hi, P.V)
    sigma = o.default_sigma(P.shape, P.lo, P.hi, P.V)
    tau = o.default_tau(P.shape, P.lo, P.hi, P.V, sigma)
    G = o.SourceSolver(H, sigma)
    U = o.householder_orthonormalize(U0)
    Es = [o.energy(H, U)]
    for _ in range(nsteps):
        U = o.scheme_step(U, G.solve(U), tau)
        Es.append(o.energy(H, U))
    return U, Es, sigma, tau


def test_init_orthonormalises_like_householder():
    P = syn.config_2d_laplace()
    U0 = syn.gaussian_block(0, P.n, P.p)
    with pkg.Solver(P.shape, P.lo, P.hi, P.V, U0, P.p) as s:
        U = s.get_U()
    assert np.abs(U - o.householder_orthonormalize(U0)).max() < 1e-13


@pytest.mark.parametrize("P", [syn.config_2d_laplace(), syn.wells_3d(12, 10, 4, 7)],
                         ids=["laplace2d", "wells3d_12"])
def test_steps_match_oracle_fp64(P):
    U0 = syn.gaussian_block(1, P.n, P.p)
    U_ref, Es, sigma, tau = _oracle_steps(P, U0, 6)
    with pkg.Solver(P.shape, P.lo, P.hi, P.V, U0, P.p, cg_rtol=1e-14) as s:
        st0 = s.stats()
        assert st0["sigma"] == pytest.approx(sigma, rel=1e-14, abs=1e-14)
        assert st0["tau"] == pytest.approx(tau, rel=1e-14)
        energies = [st0["energy"]]
        for _ in range(6):
            energies.append(s.step(1)["energy"])
        U = s.get_U()
    assert np.abs(U - U_ref).max() < 1e-10
    np.testing.assert_allclose(energies, Es, rtol=1e-12)


def test_laplace_solve_fp64_closed_form():
    """2D Laplace (32 x 32, p = 8) to r <= 1e-8: eigenvalues to 1e-10 of the closed form."""
    P = syn.config_2d_laplace()
    U0 = syn.gaussian_block(0, P.n, P.p)
    h = 1.0 / 33
    lam = np.sort([(2 / h ** 2) * (math.sin(i * math.pi / 66) ** 2 + math.sin(j * math.pi / 66) ** 2)
                   for i in range(1, 33) for j in range(1, 33)])[: P.p]
    ref = o.run(P.shape, P.lo, P.hi, P.V, U0, stop="residual", tol=1e-8, max_steps=2000)
    with pkg.Solver(P.shape, P.lo, P.hi, P.V, U0, P.p, check_every=1) as s:
        Es = [s.stats()["energy"]]
        st = s.solve(1e-8, 2000, pkg.OP_STOP_RESIDUAL)
        assert st["converged"]
        ritz = s.eigenvalues(pkg.OP_EIG_RITZ)
        paper = s.eigenvalues(pkg.OP_EIG_PAPER)
        U = s.get_U()
    np.testing.assert_allclose(ritz, lam, rtol=1e-10)
    np.testing.assert_allclose(paper, lam, rtol=1e-10)
    assert np.linalg.norm(U.T @ U - np.eye(P.p)) < 1e-12
    assert abs(st["steps"] - ref.steps) <= 2
    assert st["energy"] == pytest.approx(0.5 * lam.sum(), rel=1e-11)


def test_energy_monotone_and_orthogonality_every_step_fp64():
    P = syn.wells_3d(16, 12, 5, 3)
    U0 = syn.gaussian_block(2, P.n, P.p)
    with pkg.Solver(P.shape, P.lo, P.hi, P.V, U0, P.p) as s:
        E = [s.stats()["energy"]]
        orth = []
        for _ in range(40):
            st = s.step(1)
            E.append(st["energy"])
            orth.append(st["orth"])
    E = np.array(E)
    assert np.all(np.diff(E) <= 1e-11 * np.abs(E[1:]))
    assert max(orth) < 1e-12


def test_wells_3d_solve_fp64_vs_dense_eigensolve():
    # p = 5 sits at a spectral gap of 0.34: about 70 steps per decade of residual
    # (the contraction 1 - tau (mu_p - mu_{p+1}) of the linearised step)
    P = syn.wells_3d(14, 5, 4, 11)
    U0 = syn.gaussian_block(5, P.n, P.p)
    lam = np.linalg.eigvalsh(o.hamiltonian(P.shape, P.lo, P.hi, P.V).toarray())
    assert lam[P.p] - lam[P.p - 1] > 0.3
    with pkg.Solver(P.shape, P.lo, P.hi, P.V, U0, P.p) as s:
        st = s.solve(1e-10, 20000, pkg.OP_STOP_RESIDUAL)
        ritz = s.eigenvalues()
    np.testing.assert_allclose(ritz, lam[: P.p], rtol=1e-10)
    assert st["orth"] < 1e-12


def test_laplace_solve_fp32():
    P = syn.config_2d_laplace()
    U0 = syn.gaussian_block(0, P.n, P.p)
    h = 1.0 / 33
    lam = np.sort([(2 / h ** 2) * (math.sin(i * math.pi / 66) ** 2 + math.sin(j * math.pi / 66) ** 2)
                   for i in range(1, 33) for j in range(1, 33)])[: P.p]
    with pkg.Solver(P.shape, P.lo, P.hi, P.V, U0, P.p, prec="fp32") as s:
        st = s.solve(2e-6, 3000, pkg.OP_STOP_RESIDUAL)
        ritz = s.eigenvalues()
        U = s.get_U()
    np.testing.assert_allclose(ritz, lam, rtol=1e-5)
    assert np.linalg.norm(U.T @ U - np.eye(P.p)) < 1e-5


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_edge_cases_p1_and_p_equals_n(prec):
    # p = 1 on a 2D grid; p = n on a tiny grid (the whole spectrum)
    shape, lo, hi = (5, 4), (0.0, 0.0), (1.0, 1.0)
    V = np.random.default_rng(0).uniform(0, 1, 20)
    lam = np.linalg.eigvalsh(o.hamiltonian(shape, lo, hi, V).toarray())
    tol = 1e-10 if prec == "fp64" else 1e-5
    for p in (1, 20):
        U0 = syn.gaussian_block(9, 20, p)
        with pkg.Solver(shape, lo, hi, V, U0, p, prec=prec) as s:
            s.solve(1e-9 if prec == "fp64" else 1e-6, 5000, pkg.OP_STOP_RESIDUAL,
                    raise_on_max=False)
            ritz = s.eigenvalues()
        np.testing.assert_allclose(ritz, lam[:p], rtol=tol)


def test_degenerate_grid_line():
    # a 1 x N grid (2D with nx = 1) is a 1D chain: closed-form spectrum
    N, p = 40, 4
    shape, lo, hi = (1, N), (0.0, 0.0), (1.0, 1.0)
    with pkg.Solver(shape, lo, hi, np.zeros(N), syn.gaussian_block(3, N, p), p) as s:
        s.solve(1e-10, 20000, pkg.OP_STOP_RESIDUAL)
        ritz = s.eigenvalues()
    hx, hy = 0.5, 1.0 / (N + 1)
    lam = (2 / hx ** 2) * math.sin(math.pi / 4) ** 2 + \
        (2 / hy ** 2) * np.sin(np.arange(1, p + 1) * math.pi / (2 * (N + 1))) ** 2
    np.testing.assert_allclose(ritz, lam, rtol=1e-10)


def test_init_rejects_nonfinite_V_and_dependent_U0():
    P = syn.config_2d_laplace()
    V = P.V.copy()
    V[5] = np.nan
    with pytest.raises(pkg.OpError) as e:
        pkg.Solver(P.shape, P.lo, P.hi, V, syn.gaussian_block(0, P.n, P.p), P.p)
    assert e.value.status == pkg.binding.OP_ERR_ARG
    U0 = syn.gaussian_block(0, P.n, P.p)
    U0[:, 3] = U0[:, 2]  # rank deficient: Cholesky-QR must report it
    with pytest.raises(pkg.OpError) as e:
        pkg.Solver(P.shape, P.lo, P.hi, P.V, U0, P.p)
    assert e.value.status == pkg.binding.OP_ERR_NOTSPD


# ----------------------------------------------------------------------------
# Full-size workload (64^3, p = 128) in the launch configuration bench.py uses
# ----------------------------------------------------------------------------
@pytest.fixture(scope="module")
def c2():
    P = syn.config_3d_wells(0)
    return P, syn.gaussian_block(0, P.n, P.p)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_full_size_3d_wells_steps(c2, prec):
    """64^3 x 128: sampled stencil rows, sampled Gram entries and the invariants."""
    P, U0 = c2
    n, p, ld = P.n, P.p, 128
    Vt = torch.from_numpy(P.V).to(DEV, DT[prec])
    # stencil on sampled rows
    X = torch.randn(n, ld, dtype=torch.float64, device=DEV, generator=torch.Generator(DEV).manual_seed(0))
    X = X.to(DT[prec])
    Y = pkg.apply_H(P.shape, P.lo, P.hi, Vt, 0.5, X)
    H = o.hamiltonian(P.shape, P.lo, P.hi, rounded(P.V, prec))
    rows = np.random.default_rng(1).choice(n, 200, replace=False)
    Xh = X.double().cpu().numpy()
    ref = H[rows] @ Xh + 0.5 * Xh[rows]
    scale = o.gershgorin_norm(P.shape, P.lo, P.hi, P.V, 0.5) * np.abs(Xh).max()
    assert np.abs(Y.double().cpu().numpy()[rows] - ref).max() <= (1e-14 if prec == "fp64" else 4e-7) * scale
    # Gram on sampled entries
    Cm, Sm, Dm = pkg.gram(X, Y, p)
    Yh = Y.double().cpu().numpy()
    ij = np.random.default_rng(2).integers(0, p, (40, 2))
    for i, j in ij:
        assert Cm[i, j].item() == pytest.approx(Yh[:, i] @ Xh[:, j], rel=1e-9 if prec == "fp64" else 1e-5,
                                                abs=1e-6 * n)
    # a few steps of the whole path: orthogonality and energy decrease
    with pkg.Solver(P.shape, P.lo, P.hi, P.V, U0, P.p, prec=prec) as s:
        E0 = s.stats()["energy"]
        E = [E0]
        for _ in range(3):
            st = s.step(1)
            E.append(st["energy"])
        U = s.get_U()
    E = np.array(E)
    assert np.all(np.diff(E) < 0)
    assert np.linalg.norm(U.T @ U - np.eye(p)) < (1e-12 if prec == "fp64" else 1e-4)
    assert math.isfinite(st["g_residual"])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_seeded_init_draws_the_synthetic_gaussian_block(prec):
    """op_init_seeded draws U0 on the device from the same SplitMix64 / Box-Muller stream as
    synthetic.gaussian_block(seed): both contexts hold the same orthonormal U (the device's
    log and cos may differ from the host's by an ulp)."""
    P = syn.wells_3d(12, 9, 3, 2)
    with pkg.Solver(P.shape, P.lo, P.hi, P.V, None, P.p, prec=prec, seed=77) as a, \
            pkg.Solver(P.shape, P.lo, P.hi, P.V, syn.gaussian_block(77, P.n, P.p), P.p,
                       prec=prec) as b:
        Ua, Ub = a.get_U(), b.get_U()
    assert np.abs(Ua - Ub).max() <= (1e-12 if prec == "fp64" else 1e-6)
    assert np.linalg.norm(Ua.T @ Ua - np.eye(P.p)) < (1e-13 if prec == "fp64" else 1e-5)
