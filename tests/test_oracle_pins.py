"""Pins of the FP64 oracle to facts fixed outside the oracle itself.

Each test checks the oracle against a closed form, a brute-force computation
built independently here, an invariant proved in the paper, or a number the
paper prints.  A plausible mistake in the oracle (a dropped term, a wrong sign
or index, a transposed operand, an axis-order slip) fails at least one test.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import oracle as o
import synthetic as syn

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------
# Independent constructions used by the pins
# ----------------------------------------------------------------------------
def dense_stencil(shape, lo, hi, V):
    """H built point by point from the FD stencil (no Kronecker products)."""
    dim = len(shape)
    h = [(hi[d] - lo[d]) / (shape[d] + 1) for d in range(dim)]
    n = int(np.prod(shape))
    Hd = np.zeros((n, n))
    strides = [1, shape[0], shape[0] * (shape[1] if dim > 1 else 1)]
    for idx in range(n):
        rem = idx
        coord = []
        for d in range(dim):
            coord.append(rem % shape[d])
            rem //= shape[d]
        Hd[idx, idx] = V[idx] + sum(1.0 / (h[d] ** 2) for d in range(dim))
        for d in range(dim):
            for s in (-1, 1):
                c = coord[d] + s
                if 0 <= c < shape[d]:
                    Hd[idx, idx + s * strides[d]] -= 0.5 / (h[d] ** 2)
    return Hd


def fd_laplace_eigs(shape, lengths):
    """Closed-form eigenvalues of -1/2 Delta_h with Dirichlet ends:
    sum_d (2/h_d^2) sin^2(k_d pi / (2 (n_d + 1))), k_d = 1..n_d."""
    per_axis = []
    for m, L in zip(shape, lengths):
        h = L / (m + 1)
        k = np.arange(1, m + 1)
        per_axis.append((2.0 / h ** 2) * np.sin(k * math.pi / (2.0 * (m + 1))) ** 2)
    tot = per_axis[0]
    for a in per_axis[1:]:
        tot = np.add.outer(tot, a).ravel()
    return np.sort(tot)


def cayley_step(U, W, tau):
    """Midpoint scheme (4.1) solved by brute force: with L = U W^T - W U^T
    (the matrix of L_U for W = GU), (I + tau/2 L) U^{n+1} = (I - tau/2 L) U^n."""
    n = U.shape[0]
    L = U @ W.T - W @ U.T
    I = np.eye(n)
    return np.linalg.solve(I + 0.5 * tau * L, (I - 0.5 * tau * L) @ U)


def random_problem(seed, shape=(5, 4, 3), p=4):
    rng = np.random.default_rng(seed)
    lo, hi = (-1.0,) * len(shape), (1.3, 0.9, 1.1)[: len(shape)]
    V = rng.uniform(-2.0, 3.0, int(np.prod(shape)))
    H = o.hamiltonian(shape, lo, hi, V)
    sigma = o.default_sigma(shape, lo, hi, V)
    U = o.householder_orthonormalize(rng.standard_normal((H.shape[0], p)))
    return shape, lo, hi, V, H, sigma, U


# ----------------------------------------------------------------------------
# Generators (the inputs both sides share)
# ----------------------------------------------------------------------------
def test_splitmix64_published_vector():
    # SplitMix64 seeded with 0: the first output is 0xE220A8397B1DCDAF.
    assert int(syn.splitmix64(np.uint64(0), 0, 1)[0]) == 0xE220A8397B1DCDAF


def test_gaussian_columns_equal_the_block_columns():
    B = syn.gaussian_block(11, 40, 9)
    np.testing.assert_array_equal(syn.gaussian_columns(11, 40, 9, [0, 3, 8]), B[:, [0, 3, 8]])


def test_gaussian_moments():
    g = syn.gaussian(syn.stream_key(7, syn.STREAM_U0), 0, 400000)
    assert abs(g.mean()) < 5e-3 and abs(g.std() - 1.0) < 5e-3
    assert abs(np.mean(g ** 4) - 3.0) < 0.05


# ----------------------------------------------------------------------------
# The Hamiltonian
# ----------------------------------------------------------------------------
def test_H_matches_pointwise_stencil_anisotropic_3d():
    shape, lo, hi, V, H, _, _ = random_problem(0)
    np.testing.assert_allclose(H.toarray(), dense_stencil(shape, lo, hi, V), rtol=0, atol=1e-12)


def test_H_matches_pointwise_stencil_2d():
    shape, lo, hi = (6, 4), (0.0, -1.0), (1.0, 2.0)
    V = np.random.default_rng(3).normal(size=24)
    np.testing.assert_allclose(o.hamiltonian(shape, lo, hi, V).toarray(),
                               dense_stencil(shape, lo, hi, V), rtol=0, atol=1e-12)


def test_laplacian_closed_form_2d_unit_square():
    P = syn.config_2d_laplace()
    lam = np.linalg.eigvalsh(o.hamiltonian(P.shape, P.lo, P.hi, P.V).toarray())
    np.testing.assert_allclose(lam, fd_laplace_eigs(P.shape, (1.0, 1.0)), rtol=1e-12, atol=1e-10)
    assert lam[0] == pytest.approx(o.spectrum_lower_bound(P.shape, P.lo, P.hi, P.V), rel=1e-12)


def test_laplacian_closed_form_3d_anisotropic():
    shape, lo, hi = (5, 4, 3), (0.0, 0.0, 0.0), (1.0, 2.0, 0.5)
    lam = np.linalg.eigvalsh(o.hamiltonian(shape, lo, hi, np.zeros(60)).toarray())
    np.testing.assert_allclose(lam, fd_laplace_eigs(shape, (1.0, 2.0, 0.5)), rtol=1e-12)


def test_separable_potential_axis_order():
    # V = f(x) + g(y) + k(z): the spectrum is the sum of three 1D spectra.
    # Putting V on the wrong axis (with n_x, n_y, n_z all different) breaks this.
    shape, lo, hi = (6, 5, 4), (-1.0, -2.0, 0.0), (1.0, 1.0, 3.0)
    xs = syn.grid_coords(shape, lo, hi)
    f, g, k = np.sin(3 * xs[0]) + xs[0] ** 2, np.exp(xs[1]), 2.0 * xs[2]
    V = (f[None, None, :] + g[None, :, None] + k[:, None, None]).ravel()
    lam = np.linalg.eigvalsh(o.hamiltonian(shape, lo, hi, V).toarray())
    one_d = []
    for d, pot in enumerate((f, g, k)):
        m, h = shape[d], (hi[d] - lo[d]) / (shape[d] + 1)
        T = np.diag(np.full(m, 1.0 / h ** 2) + pot) - np.diag(np.full(m - 1, 0.5 / h ** 2), 1) \
            - np.diag(np.full(m - 1, 0.5 / h ** 2), -1)
        one_d.append(np.linalg.eigvalsh(T))
    ref = np.sort(np.add.outer(np.add.outer(one_d[2], one_d[1]), one_d[0]).ravel())
    np.testing.assert_allclose(lam, ref, rtol=1e-12, atol=1e-11)


def test_synthetic_potential_ordering_matches_coordinates():
    # The generator's V(ix + nx (iy + ny iz)) must be the potential at (x_ix, y_iy, z_iz).
    shape, lo, hi = (5, 4, 3), (-1.0, -2.0, -3.0), (1.0, 2.0, 3.0)
    wells = [syn.Well((0.3, -0.5, 1.0), 2.0, 0.7)]
    V = syn.potential(shape, lo, hi, 0.5, wells)
    xs = syn.grid_coords(shape, lo, hi)
    ix, iy, iz = 3, 1, 2
    x = np.array([xs[0][ix], xs[1][iy], xs[2][iz]])
    ref = 0.5 * x @ x - 2.0 * math.exp(-np.sum((x - np.array(wells[0].center)) ** 2) / (2 * 0.49))
    assert V[ix + 5 * (iy + 4 * iz)] == pytest.approx(ref, rel=1e-14)


# ----------------------------------------------------------------------------
# Step 1 and the sub-steps 2-4
# ----------------------------------------------------------------------------
def test_source_solve_direct_and_cg_agree():
    shape, lo, hi, V, H, sigma, U = random_problem(1, (6, 5, 4), 5)
    Gd = np.linalg.solve(H.toarray() + sigma * np.eye(H.shape[0]), U)
    Wd = o.SourceSolver(H, sigma).solve(U)
    Wc = o.SourceSolver(H, sigma, direct_max=0, cg_rtol=1e-14).solve(U)
    np.testing.assert_allclose(Wd, Gd, rtol=0, atol=1e-12)
    np.testing.assert_allclose(Wc, Gd, rtol=0, atol=1e-11)


def test_jacobi_pcg_solves_a_diagonal_system_in_one_iteration():
    # M^-1 A = I: the first step length is 1 and x_1 = b / d exactly
    import scipy.sparse as sp
    d = np.linspace(0.5, 40.0, 30)
    B = np.random.default_rng(2).standard_normal((30, 4))
    X, it = o.block_pcg_jacobi(sp.diags(d).tocsr(), B, rtol=1e-14)
    assert it == 1
    np.testing.assert_allclose(X, B / d[:, None], rtol=1e-15, atol=0)


def test_jacobi_pcg_equals_cg_for_a_constant_diagonal():
    # a constant diagonal scales the residual only: the iterates are those of CG
    shape, lo, hi = (5, 4, 3), (-1.0,) * 3, (1.0,) * 3
    n = int(np.prod(shape))
    A = o.hamiltonian(shape, lo, hi, np.full(n, 0.7)).tocsr()
    B = np.random.default_rng(3).standard_normal((n, 3))
    X0 = 0.1 * np.random.default_rng(4).standard_normal((n, 3))
    for k in (1, 2, 4, 7):
        Xp, ip = o.block_pcg_jacobi(A, B, X0, rtol=0.0, max_iter=k)
        Xc, ic = o.block_cg(A, B, X0, rtol=0.0, max_iter=k)
        assert ip == ic == k
        np.testing.assert_allclose(Xp, Xc, rtol=0, atol=1e-12 * np.abs(Xc).max())


def test_jacobi_pcg_iterate_minimises_the_energy_error_over_the_krylov_space():
    # x_k = argmin ||x - x*||_A over x_0 + span{z0, (M^-1 A) z0, ..}, brute force
    import scipy.sparse as sp
    shape, lo, hi, V, H, sigma, U = random_problem(7, (4, 3, 3), 2)
    n = H.shape[0]
    As = (H + sigma * sp.identity(n)).tocsr()
    A = As.toarray()
    d = np.diag(A)
    b = U[:, 1]
    x0 = 0.2 * np.random.default_rng(8).standard_normal(n)
    xs = np.linalg.solve(A, b)
    z0 = (b - A @ x0) / d
    for k in (1, 2, 3, 5):
        K = np.empty((n, k))
        K[:, 0] = z0
        for j in range(1, k):
            K[:, j] = (A @ K[:, j - 1]) / d
        Q, _ = np.linalg.qr(K)
        c = np.linalg.solve(Q.T @ A @ Q, Q.T @ (b - A @ x0))
        x_best = x0 + Q @ c
        Xk, it = o.block_pcg_jacobi(As, b[:, None], x0[:, None], rtol=0.0, max_iter=k)
        assert it == k
        np.testing.assert_allclose(Xk[:, 0], x_best, rtol=0, atol=1e-9 * np.abs(xs).max())


def test_jacobi_pcg_stops_on_the_unpreconditioned_residual():
    # the stop test is ||b - A x_k|| <= rtol ||b|| per column, at the first such k
    import scipy.sparse as sp
    shape, lo, hi, V, H, sigma, U = random_problem(41, (6, 5, 4), 3)
    A = (H + sigma * sp.identity(H.shape[0])).tocsr()
    rtol = 1e-6
    _, k = o.block_pcg_jacobi(A, U, rtol=rtol)
    for j in range(k + 1):
        X, _ = o.block_pcg_jacobi(A, U, rtol=0.0, max_iter=j)
        res = np.linalg.norm(U - A @ X, axis=0) / np.linalg.norm(U, axis=0)
        if j < k:
            assert np.any(res > rtol * (1 + 1e-9))
        else:
            assert np.all(res <= rtol * (1 + 1e-9))


def test_jacobi_pcg_converges_to_the_direct_solution():
    import scipy.sparse as sp
    shape, lo, hi, V, H, sigma, U = random_problem(1, (6, 5, 4), 5)
    As = (H + sigma * sp.identity(H.shape[0])).tocsr()
    Gd = np.linalg.solve(As.toarray(), U)
    X, it = o.block_pcg_jacobi(As, U, rtol=1e-14)
    assert 0 < it < 500
    np.testing.assert_allclose(X, Gd, rtol=0, atol=1e-11)
    R = U - As @ X
    assert np.all(np.linalg.norm(R, axis=0) <= 1e-14 * np.linalg.norm(U, axis=0))


@pytest.mark.parametrize("p", [1, 3, 6])
@pytest.mark.parametrize("tau_scale", [0.01, 1.0, 1.5, 40.0])
def test_steps_2_to_4_equal_cayley_transform(p, tau_scale):
    """Steps 2-4 of §4.1 reproduce the midpoint scheme (4.1) exactly."""
    shape, lo, hi, V, H, sigma, _ = random_problem(10 + p, (5, 4, 3), p)
    U = o.householder_orthonormalize(np.random.default_rng(p).standard_normal((60, p)))
    W = np.linalg.solve(H.toarray() + sigma * np.eye(60), U)
    tau = tau_scale * o.default_tau(shape, lo, hi, V, sigma)
    np.testing.assert_allclose(o.scheme_step(U, W, tau), cayley_step(U, W, tau), rtol=0, atol=1e-12)


@pytest.mark.parametrize("p", [1, 4, 7])
def test_midpoint_coefficients_any_W_equal_cayley(p):
    """For an arbitrary W (an inexact Step 1), the generalised Steps 2-3 solve (4.1)
    exactly: the result is the Cayley transform and keeps orthogonality."""
    rng = np.random.default_rng(40 + p)
    U = o.householder_orthonormalize(rng.standard_normal((50, p)))
    W = rng.standard_normal((50, p)) * 0.3
    for tau in (0.05, 1.0, 25.0):
        A, B = o.midpoint_coefficients(W, U, tau)
        Un = o.update(U, W, A, B, tau)
        np.testing.assert_allclose(Un, cayley_step(U, W, tau), atol=1e-12)
        assert o.orth_error(Un) < 1e-13


def test_midpoint_coefficients_reduce_to_steps_2_3_for_exact_W():
    shape, lo, hi, V, H, sigma, U = random_problem(6, (5, 4, 3), 5)
    W = np.linalg.solve(H.toarray() + sigma * np.eye(60), U)
    tau = o.default_tau(shape, lo, hi, V, sigma)
    A1, B1, _ = o.core_matrices(W, U, tau)
    A2, B2 = o.midpoint_coefficients(W, U, tau)
    np.testing.assert_allclose(A2, A1, atol=1e-12)
    np.testing.assert_allclose(B2, B1, atol=1e-12)


def test_paper_steps_lose_orthogonality_for_inexact_W():
    """The printed Steps 2-3 assume <GU, U> symmetric; with a perturbed W they do
    not keep <U, U> = I (why the device core solves (4.1) without that assumption)."""
    rng = np.random.default_rng(3)
    U = o.householder_orthonormalize(rng.standard_normal((50, 4)))
    W = rng.standard_normal((50, 4)) * 0.3
    A, B, _ = o.core_matrices(W, U, 2.0)
    assert o.orth_error(o.update(U, W, A, B, 2.0)) > 1e-6


def test_update_forms_agree():
    shape, lo, hi, V, H, sigma, U = random_problem(2, (5, 4, 3), 4)
    W = o.SourceSolver(H, sigma).solve(U)
    tau = o.default_tau(shape, lo, hi, V, sigma)
    A, B, _ = o.core_matrices(W, U, tau)
    KU, KW = o.step_coefficients(W, U, tau)
    C = o.inner(W, U)
    U1 = o.update(U, W, A, B, tau)
    U2 = U @ KU + W @ KW
    U3 = -U + (2.0 * U + tau * (W - U @ C)) @ B
    np.testing.assert_allclose(U2, U1, atol=1e-13)
    np.testing.assert_allclose(U3, U1, atol=1e-13)


def test_lemma_3_1_M_minus_I_is_psd():
    for seed in range(5):
        shape, lo, hi, V, H, sigma, U = random_problem(20 + seed, (5, 4, 3), 6)
        W = o.SourceSolver(H, sigma).solve(U)
        for tau in (0.1, 1.0, 30.0):
            _, _, M = o.core_matrices(W, U, tau)
            ev = np.linalg.eigvalsh(0.5 * (M + M.T) - np.eye(6))
            assert ev.min() > -1e-13


def test_lemma_3_2_skew_symmetry_of_L_U():
    shape, lo, hi, V, H, sigma, U = random_problem(3, (5, 4, 3), 4)
    rng = np.random.default_rng(4)
    Va, Vb = rng.standard_normal((60, 4)), rng.standard_normal((60, 4))
    G = o.SourceSolver(H, sigma)
    GU = G.solve(U)

    def L(X):
        return U @ o.inner(GU, X) - GU @ o.inner(U, X)

    S = o.inner(Va, L(Vb)) + o.inner(L(Va), Vb)
    assert np.abs(S).max() < 1e-12


def test_fixed_point_is_stationary():
    """Exact eigenvectors are a steady state (remark after (3.1))."""
    shape, lo, hi, V, H, sigma, _ = random_problem(5, (5, 4, 3), 5)
    lam, X = np.linalg.eigh(H.toarray())
    U = X[:, :5]
    W = o.SourceSolver(H, sigma).solve(U)
    tau = o.default_tau(shape, lo, hi, V, sigma)
    np.testing.assert_allclose(o.scheme_step(U, W, tau), U, atol=1e-13)


def test_cholesky_qr_matches_householder():
    U0 = syn.gaussian_block(3, 2000, 16)
    np.testing.assert_allclose(o.cholesky_qr(U0), o.householder_orthonormalize(U0), atol=1e-13)


# ----------------------------------------------------------------------------
# Whole runs: invariants, closed forms and brute force
# ----------------------------------------------------------------------------
@pytest.fixture(scope="module")
def laplace_run():
    P = syn.config_2d_laplace()
    U0 = syn.gaussian_block(0, P.n, P.p)
    r = o.run(P.shape, P.lo, P.hi, P.V, U0, stop="residual", tol=1e-8, max_steps=2000)
    return P, r


def test_laplace_2d_converges_to_closed_form(laplace_run):
    P, r = laplace_run
    assert r.converged
    lam = fd_laplace_eigs(P.shape, (1.0, 1.0))[: P.p]
    H = o.hamiltonian(P.shape, P.lo, P.hi, P.V)
    np.testing.assert_allclose(o.ritz_values(H, r.U), lam, rtol=1e-10)
    W = o.SourceSolver(H, r.sigma).solve(r.U)
    np.testing.assert_allclose(o.paper_eigenvalues(W, r.U, r.sigma), lam, rtol=1e-10)
    assert r.energy[-1] == pytest.approx(0.5 * lam.sum(), rel=1e-11)


def test_theorem_4_1_orthogonality_every_step(laplace_run):
    P, r = laplace_run
    assert max(r.orth) <= 1e-13 * math.sqrt(P.p)


def test_theorem_4_2_energy_decreases_every_step(laplace_run):
    _, r = laplace_run
    E = np.array(r.energy)
    assert np.all(np.diff(E) <= 1e-12 * np.abs(E[1:]))


def test_asymptotic_energy_rate(laplace_run):
    """Late energy-error ratio = (max_{j<=p<k} |1 - tau (mu_j - mu_k)|)^2, mu = 1/(lambda + sigma).

    Linearising Steps 1-4 at an exact eigenbasis U*: for a perturbation
    E = eps x_k e_j^T (k unoccupied), C = diag(mu) + O(eps^2), B = I + O(eps^2),
    A = diag(mu) + O(eps^2), so E is multiplied by 1 - tau (mu_j - mu_k) per
    step; the energy error is quadratic in E (Theorem 4.9: twice the rate)."""
    P, r = laplace_run
    lam = fd_laplace_eigs(P.shape, (1.0, 1.0))
    mu = 1.0 / (lam + r.sigma)
    p = P.p
    factor = np.max(np.abs(1.0 - r.tau * (mu[:p, None] - mu[None, p:])))
    E = np.array(r.energy) - 0.5 * lam[:p].sum()
    ratios = E[151:201] / E[150:200]
    assert np.median(ratios) == pytest.approx(factor ** 2, rel=2e-3)


def test_brute_force_3d_random_potential():
    shape, lo, hi = (4, 4, 4), (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0)
    rng = np.random.default_rng(11)
    V = rng.uniform(-3.0, 3.0, 64)
    p = 5
    lam = np.linalg.eigvalsh(dense_stencil(shape, lo, hi, V))
    assert lam[p] - lam[p - 1] > 1e-3
    r = o.run(shape, lo, hi, V, syn.gaussian_block(5, 64, p), stop="err_E", tol=1e-15,
              max_steps=20000)
    H = o.hamiltonian(shape, lo, hi, V)
    np.testing.assert_allclose(o.ritz_values(H, r.U), lam[:p], rtol=1e-12)
    assert r.energy[-1] == pytest.approx(0.5 * lam[:p].sum(), rel=1e-12)


def test_energy_lower_bound_and_equality_at_convergence(laplace_run):
    P, r = laplace_run
    H = o.hamiltonian(P.shape, P.lo, P.hi, P.V)
    G = o.SourceSolver(H, r.sigma)
    U = o.householder_orthonormalize(syn.gaussian_block(0, P.n, P.p))
    assert o.energy_lower_bound(G.solve(U), U, r.sigma) <= o.energy(H, U)
    Wc = G.solve(r.U)
    assert o.energy_lower_bound(Wc, r.U, r.sigma) == pytest.approx(o.energy(H, r.U), rel=1e-10)


def test_steps_far_beyond_explicit_cfl_limit():
    """Energy decays for tau ~ 1.9 (lambda_1 + sigma), ~4e4 x the explicit-Euler limit 2/lambda_max."""
    P = syn.config_2d_laplace()
    H = o.hamiltonian(P.shape, P.lo, P.hi, P.V)
    lam_max = fd_laplace_eigs(P.shape, (1.0, 1.0))[-1]
    tau = 1.9 * o.spectrum_lower_bound(P.shape, P.lo, P.hi, P.V)
    assert tau > 1e4 * (2.0 / lam_max)
    r = o.run(P.shape, P.lo, P.hi, P.V, syn.gaussian_block(1, P.n, P.p), tau=tau,
              stop="steps", max_steps=150, track_residual=False)
    E = np.array(r.energy)
    assert np.all(np.diff(E) <= 1e-12 * np.abs(E[1:]))
    assert max(r.orth) < 1e-13 * math.sqrt(P.p)


# ----------------------------------------------------------------------------
# The paper's printed numbers: Table 1 (test problem I)
# ----------------------------------------------------------------------------
@pytest.mark.slow
def test_table1_step_counts_fd_analog():
    """FD analog of test problem I (§5.1): step counts within 25 % of Table 1.

    The paper's counts come from quadratic FEM with N_g = 39601; this uses the
    FD grid with the same number of unknowns (199^2).  The stopping rule and the
    uniform tau are the paper's.  Eigenvalue errors against the discrete
    reference stay within Table 1's range, and the exact levels n1 + n2 + 1 are
    reproduced to the discretisation error."""
    with open(os.path.join(GOLDEN, "table1_test_problem_I.json")) as f:
        g = json.load(f)
    P = syn.harmonic_2d(199, g["N"], g["box"])
    assert P.n == g["N_g"]
    H = o.hamiltonian(P.shape, P.lo, P.hi, P.V)
    lam = np.sort(spla.eigsh(H.tocsc(), k=g["N"] + 1, sigma=0, which="LM")[0])
    levels = np.array([1, 2, 2, 3, 3, 3, 4, 4, 4, 4, 5, 5, 5, 5, 5], float)
    np.testing.assert_allclose(lam[: g["N"]], levels, rtol=2e-3)
    E_ref = 0.5 * lam[: g["N"]].sum()
    for tau in (1.0, 1.5):
        paper_steps = g["steps"][g["tau"].index(tau)]
        r = o.run(P.shape, P.lo, P.hi, P.V, syn.gaussian_block(0, P.n, P.p), tau=tau,
                  sigma=0.0, stop="E_ref", E_ref=E_ref, tol=g["stop_rel_energy_error"],
                  max_steps=3 * paper_steps, track_residual=False)
        assert r.converged
        assert abs(r.steps - paper_steps) <= 0.25 * paper_steps, (tau, r.steps, paper_steps)
        err = np.abs(o.ritz_values(H, r.U) / lam[: g["N"]] - 1.0)
        assert err.max() <= g["max_err_i_all"]

# ----------------------------------------------------------------------------
# The L2 gradient flow of §1 (the contrast variant)
# ----------------------------------------------------------------------------
def test_l2_flow_step_is_first_order_consistent_with_the_gradient():
    # (U+ - U) / tau -> -(H U - U U^T H U) with an O(tau) error
    shape, lo, hi, V, H, sigma, _ = random_problem(21, (5, 4, 3), 3)
    U = o.householder_orthonormalize(np.random.default_rng(22).standard_normal((60, 3)))
    F = -(H @ U - U @ (U.T @ (H @ U)))
    errs = []
    for tau in (1e-3, 1e-4):
        errs.append(np.abs((o.l2_flow_step(H, sigma, U, tau) - U) / tau - F).max())
    assert errs[1] < 0.2 * errs[0]
    assert errs[1] < 1e-3 * np.abs(F).max()


def test_l2_flow_step_does_not_depend_on_the_shift_and_keeps_orthogonality():
    shape, lo, hi, V, H, sigma, _ = random_problem(23, (5, 4, 3), 4)
    U = o.householder_orthonormalize(np.random.default_rng(24).standard_normal((60, 4)))
    hn = o.gershgorin_norm(shape, lo, hi, V, sigma)
    for tau in (0.5 / hn, 100.0 / hn):
        a = o.l2_flow_step(H, 0.0, U, tau)
        b = o.l2_flow_step(H, 3.7, U, tau)
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-12)
        assert o.orth_error(a) < 1e-12


def test_cayley_coefficients_equal_the_dense_cayley_transform():
    # brute force for a U far from orthonormal: (I - tau/2 L)^-1 (I + tau/2 L) U with
    # L = W U^T - U W^T
    rng = np.random.default_rng(31)
    n, p, tau = 40, 3, 0.37
    U = rng.standard_normal((n, p))
    W = rng.standard_normal((n, p))
    L = W @ U.T - U @ W.T
    Ud = np.linalg.solve(np.eye(n) - 0.5 * tau * L, (np.eye(n) + 0.5 * tau * L) @ U)
    KU, KW = o.cayley_coefficients(W, U, tau)
    np.testing.assert_allclose(U @ KU + W @ KW, Ud, rtol=0, atol=1e-12 * np.abs(Ud).max())
    # <U, U> is kept exactly, whatever it is
    Up = U @ KU + W @ KW
    np.testing.assert_allclose(Up.T @ Up, U.T @ U, rtol=0, atol=1e-11 * np.abs(U.T @ U).max())


def test_cayley_coefficients_reduce_to_steps_2_to_4_for_orthonormal_U():
    shape, lo, hi, V, H, sigma, U = random_problem(32, (5, 4, 3), 4)
    W = np.linalg.solve(H.toarray() + sigma * np.eye(60), U) + 1e-3 * np.random.default_rng(
        33).standard_normal((60, 4))
    tau = o.default_tau(shape, lo, hi, V, sigma)
    KU, KW = o.cayley_coefficients(W, U, tau)
    A, B = o.midpoint_coefficients(W, U, tau)
    np.testing.assert_allclose(U @ KU + W @ KW, o.update(U, W, A, B, tau), rtol=0, atol=1e-12)


def test_l2_flow_is_cfl_limited_and_the_g_flow_is_not():
    # the CFL restriction the paper's model removes (§1, Table 3), on the 2-D Laplacian
    # with p = 2: with tau = 1 / ||H|| the L2 flow decreases the energy every step and
    # needs ~4x the steps per halving of h; with 16x that step it does not converge; the
    # G flow converges at its default step on every mesh in about the same number of steps
    import scipy.sparse.linalg as spla

    def run(N, flow, c=1.0, cap=6000):
        shape, lo, hi = (N, N), (0.0, 0.0), (math.pi, math.pi)
        n = N * N
        V = np.zeros(n)
        H = o.hamiltonian(shape, lo, hi, V)
        sigma = o.default_sigma(shape, lo, hi, V)
        E_star = 0.5 * np.sum(np.sort(spla.eigsh(H, k=2, which="SA")[0]))
        U = o.householder_orthonormalize(syn.gaussian_block(5, n, 2))
        if flow == "l2":
            tau = c / o.gershgorin_norm(shape, lo, hi, V, sigma)
        else:
            tau = o.default_tau(shape, lo, hi, V, sigma)
            G = o.SourceSolver(H, sigma)
        E_prev, monotone = o.energy(H, U), True
        for k in range(1, cap + 1):
            U = o.l2_flow_step(H, sigma, U, tau) if flow == "l2" else \
                o.scheme_step(U, G.solve(U), tau)
            E = o.energy(H, U)
            monotone = monotone and E <= E_prev * (1 + 1e-13)
            E_prev = E
            if E - E_star <= 1e-6 * E_star:
                return k, monotone
        return None, monotone
    l2 = [run(N, "l2") for N in (7, 15)]
    assert all(m for _, m in l2), l2
    assert l2[0][0] and l2[1][0] and 3.0 <= l2[1][0] / l2[0][0] <= 5.0, l2
    big = run(15, "l2", c=16.0, cap=3000)
    assert big[0] is None and not big[1], big
    g = [run(N, "g")[0] for N in (7, 15)]
    assert None not in g and g[1] <= 1.5 * g[0] + 2, g


# ----------------------------------------------------------------------------
# The residual of Algorithm 1's stop rule and its normalisation
# ----------------------------------------------------------------------------
def _max_abs_row_sum(A):
    return float(np.max(np.sum(np.abs(A), axis=1)))


def test_gershgorin_norm_is_the_max_row_sum_of_the_pointwise_stencil():
    # For V + sigma >= 0 with its maximum at a point whose 2 dim neighbours are all
    # inside the grid, the largest absolute row sum of H + sigma (built point by point)
    # is exactly 2 sum_d 1/h_d^2 + max(V + sigma).
    shape, lo, hi = (5, 6, 4), (-1.0, 0.0, 0.5), (1.3, 2.0, 1.1)
    n = int(np.prod(shape))
    V = np.random.default_rng(21).uniform(0.0, 2.0, n)
    V[2 + 5 * (3 + 6 * 2)] = 7.5            # interior point (2, 3, 2)
    sigma = 0.25
    Hd = dense_stencil(shape, lo, hi, V) + sigma * np.eye(n)
    assert o.gershgorin_norm(shape, lo, hi, V, sigma) == pytest.approx(_max_abs_row_sum(Hd),
                                                                       rel=1e-14)


def test_gershgorin_norm_bounds_the_spectral_norm_2d_and_3d():
    # In general it is an upper bound of ||H + sigma||_inf >= ||H + sigma||_2, also for
    # a potential of both signs whose extreme sits on the boundary layer.
    for shape, lo, hi in (((7, 5), (0.0, -1.0), (1.0, 2.0)),
                          ((4, 5, 3), (-1.0, -1.0, -1.0), (1.0, 0.5, 2.0))):
        n = int(np.prod(shape))
        V = np.random.default_rng(5).uniform(-3.0, 3.0, n)
        V[0] = -9.0                          # a corner point
        sigma = 0.5
        Hd = dense_stencil(shape, lo, hi, V) + sigma * np.eye(n)
        g = o.gershgorin_norm(shape, lo, hi, V, sigma)
        assert g >= _max_abs_row_sum(Hd) - 1e-12
        assert g >= np.max(np.abs(np.linalg.eigvalsh(Hd))) - 1e-12
        # and it is not loose by more than the boundary effect of the corner point
        h = [(b - a) / (m + 1) for a, b, m in zip(lo, hi, shape)]
        assert g - _max_abs_row_sum(Hd) <= sum(0.5 / hd ** 2 for hd in h) + 1e-12


def _eigen_setup(seed=9):
    shape, lo, hi = (5, 4, 3), (-1.0, -1.0, -1.0), (1.2, 0.9, 1.1)
    V = np.random.default_rng(seed).uniform(-1.0, 2.0, 60)
    Hd = dense_stencil(shape, lo, hi, V)
    lam, X = np.linalg.eigh(Hd)
    return shape, lo, hi, V, Hd, lam, X


def test_residuals_vanish_on_an_exact_rotated_eigenbasis():
    shape, lo, hi, V, Hd, lam, X = _eigen_setup()
    p = 6
    Q, _ = np.linalg.qr(np.random.default_rng(1).standard_normal((p, p)))
    U = X[:, :p] @ Q
    r, r_theta, ri = o.residuals(o.hamiltonian(shape, lo, hi, V), U, 10.0)
    assert r < 1e-14 and r_theta < 1e-14 and np.max(ri) < 1e-12


def test_residuals_closed_form_for_two_rotated_directions():
    # U = [c1 x_1 + s1 x_k, c2 x_2 + s2 x_m, x_3, .., x_p] Q with k, m > p distinct:
    # Theta = diag(c1^2 l1 + s1^2 lk, c2^2 l2 + s2^2 lm, l3, ..) rotated by Q, and
    # H U - U Theta has Frobenius norm sqrt((c1 s1 (lk - l1))^2 + (c2 s2 (lm - l2))^2)
    # whatever the rotation Q.  r divides it by hnorm sqrt(p); r_theta by ||Theta||_F;
    # the Ritz residuals r_i are |c1 s1 (lk - l1)|, |c2 s2 (lm - l2)| and zeros.
    shape, lo, hi, V, Hd, lam, X = _eigen_setup()
    p, k, m = 5, 11, 17
    t1, t2 = 0.3, 1.1
    c1, s1, c2, s2 = math.cos(t1), math.sin(t1), math.cos(t2), math.sin(t2)
    U = X[:, :p].copy()
    U[:, 0] = c1 * X[:, 0] + s1 * X[:, k]
    U[:, 1] = c2 * X[:, 1] + s2 * X[:, m]
    Q, _ = np.linalg.qr(np.random.default_rng(2).standard_normal((p, p)))
    U = U @ Q
    e1, e2 = c1 * s1 * (lam[k] - lam[0]), c2 * s2 * (lam[m] - lam[1])
    nR = math.hypot(e1, e2)
    theta = np.array([c1 * c1 * lam[0] + s1 * s1 * lam[k], c2 * c2 * lam[1] + s2 * s2 * lam[m],
                      *lam[2:p]])
    hnorm = 37.0
    r, r_theta, ri = o.residuals(o.hamiltonian(shape, lo, hi, V), U, hnorm)
    assert r == pytest.approx(nR / (hnorm * math.sqrt(p)), rel=1e-12)
    assert r_theta == pytest.approx(nR / float(np.linalg.norm(theta)), rel=1e-12)
    np.testing.assert_allclose(np.sort(ri), np.sort([0.0, 0.0, 0.0, abs(e1), abs(e2)]),
                               rtol=1e-10, atol=1e-12)


def test_residual_of_a_run_uses_the_gershgorin_normalisation():
    # The run's recorded residual of U^0 is ||H U - U Theta||_F / (hnorm sqrt(p)) with
    # hnorm = 2 sum_d 1/h_d^2 + max |V + sigma|, computed here from the dense stencil.
    shape, lo, hi, V, Hd, lam, X = _eigen_setup(4)
    p = 4
    U0 = np.random.default_rng(3).standard_normal((60, p))
    res = o.run(shape, lo, hi, V, U0, max_steps=0, stop="steps")
    U = o.householder_orthonormalize(U0)
    HU = Hd @ U
    nR = float(np.linalg.norm(HU - U @ (U.T @ HU)))
    h = [(b - a) / (m + 1) for a, b, m in zip(lo, hi, shape)]
    hn = 2.0 * sum(1.0 / hd ** 2 for hd in h) + float(np.max(np.abs(V + res.sigma)))
    assert res.resid[0] == pytest.approx(nR / (hn * math.sqrt(p)), rel=1e-12)
