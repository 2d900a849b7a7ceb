"""Planted mistakes in the oracle must be caught by its pins.

Each case swaps one oracle function for a copy with a plausible mistake (on
the CPU, inside this process only) and checks that the corresponding pin from
test_oracle_pins fails.
"""
import numpy as np
import pytest

import oracle as o
import oracle.scheme as sch
import synthetic as syn
from tests.test_oracle_pins import cayley_step, dense_stencil, random_problem


def _core_no_C2(W, U, tau):
    p = U.shape[1]
    I = np.eye(p)
    C, S = W.T @ U, W.T @ W
    M = I + (tau * tau / 4.0) * S                       # dropped -tau^2/4 C^2
    B = np.linalg.solve(M, I)
    return (2.0 / tau) * (I - B + (tau / 2.0) * (C @ B)), B, M


def _core_sign(W, U, tau):
    p = U.shape[1]
    I = np.eye(p)
    C, S = W.T @ U, W.T @ W
    M = I + (tau * tau / 4.0) * (S - C @ C)
    B = np.linalg.solve(M, I)
    return (2.0 / tau) * (I - B - (tau / 2.0) * (C @ B)), B, M   # wrong sign


def _core_half_tau(W, U, tau):
    p = U.shape[1]
    I = np.eye(p)
    C, S = W.T @ U, W.T @ W
    M = I + (tau * tau / 2.0) * (S - C @ C)             # tau^2/2 instead of tau^2/4
    B = np.linalg.solve(M, I)
    return (2.0 / tau) * (I - B + (tau / 2.0) * (C @ B)), B, M


@pytest.mark.parametrize("mutant", [_core_no_C2, _core_sign, _core_half_tau])
def test_core_mutants_break_cayley_pin(monkeypatch, mutant):
    shape, lo, hi, V, H, sigma, _ = random_problem(13, (5, 4, 3), 3)
    U = o.householder_orthonormalize(np.random.default_rng(3).standard_normal((60, 3)))
    W = np.linalg.solve(H.toarray() + sigma * np.eye(60), U)
    tau = o.default_tau(shape, lo, hi, V, sigma)
    monkeypatch.setattr(sch, "core_matrices", mutant)
    diff = np.abs(sch.scheme_step(U, W, tau) - cayley_step(U, W, tau)).max()
    assert diff > 1e-6


def test_stencil_factor_mutant_breaks_pointwise_pin(monkeypatch):
    import scipy.sparse as sp

    def wrong(m, h):
        e = np.ones(m)
        return sp.diags([-e[:-1], 2.0 * e, -e[:-1]], [-1, 0, 1], format="csr") / (h * h)

    monkeypatch.setattr(sch, "_second_difference", wrong)
    shape, lo, hi, V, H, _, _ = random_problem(0)
    assert np.abs(H.toarray() - dense_stencil(shape, lo, hi, V)).max() > 1.0


def test_axis_order_mutant_breaks_pointwise_pin():
    # V laid out with z fastest instead of x fastest
    shape, lo, hi = (5, 4, 3), (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0)
    V = np.random.default_rng(1).uniform(-1, 1, 60)
    Vt = V.reshape(3, 4, 5).transpose(2, 1, 0).ravel()
    Hm = o.hamiltonian(shape, lo, hi, Vt).toarray()
    assert np.abs(Hm - dense_stencil(shape, lo, hi, V)).max() > 1e-3


def test_update_sign_mutant_breaks_orthogonality():
    P = syn.config_2d_laplace()
    H = o.hamiltonian(P.shape, P.lo, P.hi, P.V)
    U = o.householder_orthonormalize(syn.gaussian_block(0, P.n, P.p))
    W = o.SourceSolver(H, 0.0).solve(U)
    tau = o.default_tau(P.shape, P.lo, P.hi, P.V, 0.0)
    A, B, _ = o.core_matrices(W, U, tau)
    Ubad = U + tau * (U @ A) + tau * (W @ B)           # wrong sign on the U A term
    assert o.orth_error(Ubad) > 1e-3
    assert o.orth_error(o.update(U, W, A, B, tau)) < 1e-13


def _pcg_mutant(kind):
    """Copy of oracle.block_pcg_jacobi with one plausible mistake."""
    def pcg(A, Bm, X0=None, rtol=1e-13, max_iter=20000):
        d = np.asarray(A.diagonal(), dtype=np.float64)
        X = np.zeros_like(Bm) if X0 is None else np.array(X0, dtype=np.float64)
        R = Bm - A @ X
        Z = R / d[:, None]
        P = (R if kind == "direction_from_r" else Z).copy()
        rho = np.einsum("ij,ij->j", R, R if kind == "beta_from_rr" else Z)
        target = (rtol * np.linalg.norm(Bm, axis=0)) ** 2
        it = 0
        while it < max_iter and np.any(np.einsum("ij,ij->j", R, R) > target):
            Q = A @ P
            alpha = rho / np.einsum("ij,ij->j", P, Q)
            X += P * alpha
            R -= Q * alpha
            Z = R / d[:, None]
            rho_new = np.einsum("ij,ij->j", R, R if kind == "beta_from_rr" else Z)
            P = (R if kind == "direction_from_r" else Z) + P * (rho_new / rho)
            rho = rho_new
            it += 1
        return X, it
    return pcg


@pytest.mark.parametrize("kind", ["direction_from_r", "beta_from_rr"])
def test_pcg_mutants_break_krylov_optimality_pin(monkeypatch, kind):
    from tests.test_oracle_pins import \
        test_jacobi_pcg_iterate_minimises_the_energy_error_over_the_krylov_space as pin
    monkeypatch.setattr(o, "block_pcg_jacobi", _pcg_mutant(kind))
    with pytest.raises(AssertionError):
        pin()


def test_pcg_mutant_copy_is_faithful_without_mistake(monkeypatch):
    # the mutant template itself, with no mistake planted, passes the pin
    from tests.test_oracle_pins import \
        test_jacobi_pcg_iterate_minimises_the_energy_error_over_the_krylov_space as pin
    monkeypatch.setattr(o, "block_pcg_jacobi", _pcg_mutant("none"))
    pin()


def _residuals_no_sqrt_p(H, U, hnorm):
    HU = H @ U
    R = HU - U @ (U.T @ HU)
    nr = float(np.linalg.norm(R))
    lam, Y = np.linalg.eigh(U.T @ HU)
    ri = np.linalg.norm(H @ (U @ Y) - (U @ Y) * lam, axis=0)
    return nr / hnorm, nr / float(np.linalg.norm(U.T @ HU)), ri     # dropped sqrt(p)


def _residuals_theta_norm(H, U, hnorm):
    HU = H @ U
    Th = U.T @ HU
    nr = float(np.linalg.norm(HU - U @ Th))
    lam, Y = np.linalg.eigh(Th)
    ri = np.linalg.norm(H @ (U @ Y) - (U @ Y) * lam, axis=0)
    return nr / float(np.linalg.norm(Th)), nr / float(np.linalg.norm(Th)), ri  # wrong normaliser


def _residuals_diagonal_theta(H, U, hnorm):
    HU = H @ U
    Th = U.T @ HU
    R = HU - U * np.diag(Th)                               # Theta replaced by its diagonal
    nr = float(np.linalg.norm(R))
    lam, Y = np.linalg.eigh(Th)
    ri = np.linalg.norm(H @ (U @ Y) - (U @ Y) * lam, axis=0)
    return nr / (hnorm * np.sqrt(U.shape[1])), nr / float(np.linalg.norm(Th)), ri


@pytest.mark.parametrize("mutant", [_residuals_no_sqrt_p, _residuals_theta_norm,
                                    _residuals_diagonal_theta])
def test_residual_mutants_break_the_closed_form_pin(monkeypatch, mutant):
    from tests.test_oracle_pins import test_residuals_closed_form_for_two_rotated_directions as pin
    monkeypatch.setattr(o, "residuals", mutant)
    with pytest.raises(AssertionError):
        pin()


def test_gershgorin_diagonal_only_mutant_breaks_the_row_sum_pin(monkeypatch):
    from tests.test_oracle_pins import \
        test_gershgorin_norm_is_the_max_row_sum_of_the_pointwise_stencil as pin

    def diag_only(shape, lo, hi, V, sigma):
        h = o.grid_spacing(shape, lo, hi)
        return sum(1.0 / (hd * hd) for hd in h) + float(np.max(np.abs(np.asarray(V) + sigma)))

    monkeypatch.setattr(o, "gershgorin_norm", diag_only)
    with pytest.raises(AssertionError):
        pin()
