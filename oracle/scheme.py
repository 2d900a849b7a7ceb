"""Plain FP64 implementation of the orthogonality-preserving scheme.

TEST INFRASTRUCTURE ONLY (see the package docstring): a slow, literal CPU
restatement of the paper's method that the CUDA path is checked against.  It
shares no code with the CUDA library.

Paper: Chu, Dai, Wang, Zhou, "An orthogonality-preserving approach for
eigenvalue problems", arXiv 2511.06788.  Every function cites the passage it
follows.  Notation follows the paper: ``<U, V>`` is the inner matrix
(§2.1, ``<U,V>_ij = (u_i, v_j)``), ``G = (H + sigma)^-1`` the solution operator
(§3.1), ``W = G U``.

Discretisation (the paper uses finite elements in §5; this oracle uses finite
differences): ``H = -1/2 Delta_h + diag(V)`` with the standard 3-point second
difference per axis and homogeneous Dirichlet values outside the interior
grid.  The discrete inner product is the Euclidean one on R^n (the h^d weight
of the L2 product cancels in the scheme because G is linear and
``<U, U> = I`` is imposed in the same product).

Parity status of each function: every function below is pinned by
``tests/test_oracle_pins.py`` (closed-form eigenvalues, brute-force dense
eigensolves, the Cayley-transform form of the midpoint step, the paper's
invariants and its Table 1 step counts); none is "parity unpinned".
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

__all__ = [
    "grid_spacing", "hamiltonian", "spectrum_lower_bound", "default_sigma", "default_tau",
    "gershgorin_norm", "householder_orthonormalize", "cholesky_qr", "inner", "SourceSolver",
    "block_cg", "block_pcg_jacobi", "core_matrices", "core_from_inner", "update", "scheme_step", "energy", "residuals",
    "paper_eigenvalues", "ritz_values", "orth_error", "energy_lower_bound", "run",
    "RunResult", "step_coefficients", "midpoint_coefficients", "l2_flow_step",
    "cayley_coefficients",
]


# ----------------------------------------------------------------------------
# The discrete Hamiltonian
# ----------------------------------------------------------------------------
def grid_spacing(shape, lo, hi):
    """h_d = (hi_d - lo_d) / (n_d + 1): n_d interior points, zero boundary values."""
    return tuple((b - a) / (m + 1) for a, b, m in zip(lo, hi, shape))


def _second_difference(m: int, h: float) -> sp.csr_matrix:
    """1D operator -1/2 d^2/dx^2 with Dirichlet ends: (1/(2h^2)) tridiag(-1, 2, -1)."""
    e = np.ones(m)
    return sp.diags([-e[:-1], 2.0 * e, -e[:-1]], [-1, 0, 1], format="csr") / (2.0 * h * h)


def hamiltonian(shape, lo, hi, V) -> sp.csr_matrix:
    """H = -1/2 Delta_h + diag(V) as a Kronecker sum (grid index ix + nx*(iy + ny*iz)).

    The continuous operator is the one of the paper's test problems (§5.1,
    §5.2: ``-1/2 Delta + V``); the Kronecker sum with x as the fastest index
    is the 5-point (2D) / 7-point (3D) finite-difference stencil.
    """
    h = grid_spacing(shape, lo, hi)
    dim = len(shape)
    n = int(np.prod(shape))
    H = sp.csr_matrix((n, n))
    for d in range(dim):
        # axis d sits at position (dim - 1 - d) of the Kronecker product (x fastest)
        factors = [sp.identity(shape[k], format="csr") for k in reversed(range(dim))]
        factors[dim - 1 - d] = _second_difference(shape[d], h[d])
        T = factors[0]
        for f in factors[1:]:
            T = sp.kron(T, f, format="csr")
        H = H + T
    return (H + sp.diags(np.asarray(V, dtype=np.float64), 0)).tocsr()


def spectrum_lower_bound(shape, lo, hi, V) -> float:
    """L = lambda_min(-1/2 Delta_h) + min V, a lower bound of spec(H).

    lambda_min of the 1D factor is (2/h^2) sin^2(pi h / (2 l)), l = (n+1) h.
    """
    h = grid_spacing(shape, lo, hi)
    lap = sum((2.0 / (hd * hd)) * math.sin(math.pi / (2.0 * (m + 1))) ** 2
              for hd, m in zip(h, shape))
    return lap + float(np.min(V))


def default_sigma(shape, lo, hi, V) -> float:
    """Shift reading: sigma = max(0, 1 - L) so that H + sigma >= 1 is SPD.

    The paper assumes the bilinear form is an inner product (§2.2), i.e. H SPD,
    and is silent on a shift; G = (H + sigma)^-1 is then used in Step 1.
    """
    return max(0.0, 1.0 - spectrum_lower_bound(shape, lo, hi, V))


def default_tau(shape, lo, hi, V, sigma) -> float:
    """Time-step reading: tau = 1.5 (L + sigma), a fixed uniform step as in §5."""
    return 1.5 * (spectrum_lower_bound(shape, lo, hi, V) + sigma)


def gershgorin_norm(shape, lo, hi, V, sigma) -> float:
    """Gershgorin bound of ||H + sigma||: 2 sum_d 1/h_d^2 + max |V + sigma|."""
    h = grid_spacing(shape, lo, hi)
    return 2.0 * sum(1.0 / (hd * hd) for hd in h) + float(np.max(np.abs(np.asarray(V) + sigma)))


# ----------------------------------------------------------------------------
# Initial data (§5: "random data with mutually orthogonal columns")
# ----------------------------------------------------------------------------
def householder_orthonormalize(U0: np.ndarray) -> np.ndarray:
    """Q of the Householder QR of U0 (LAPACK geqrf), columns signed so diag(R) > 0."""
    Q, R = np.linalg.qr(np.asarray(U0, dtype=np.float64), mode="reduced")
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return Q * s


def cholesky_qr(U0: np.ndarray) -> np.ndarray:
    """Cholesky-QR: R = chol(U0^T U0) (upper), Q = U0 R^-1."""
    U0 = np.asarray(U0, dtype=np.float64)
    R = np.linalg.cholesky(U0.T @ U0).T
    return sla.solve_triangular(R, U0.T, trans="T", lower=False).T


def inner(U: np.ndarray, V: np.ndarray) -> np.ndarray:
    """Inner matrix <U, V>_ij = (u_i, v_j) (§2.1)."""
    return U.T @ V


# ----------------------------------------------------------------------------
# Step 1: the N source problems (H + sigma) W = U
# ----------------------------------------------------------------------------
def block_cg(A, Bm: np.ndarray, X0: np.ndarray | None = None, rtol: float = 1e-13,
             max_iter: int = 20000):
    """Independent conjugate-gradient solves A x_j = b_j, one per column.

    Textbook CG (Hestenes-Stiefel) run on all columns at once; each column has
    its own alpha_j, beta_j and stops when ||r_j|| <= rtol ||b_j||.
    Returns (X, iterations).
    """
    X = np.zeros_like(Bm) if X0 is None else np.array(X0, dtype=np.float64)
    R = Bm - A @ X
    P = R.copy()
    rr = np.einsum("ij,ij->j", R, R)
    bnorm = np.sqrt(np.einsum("ij,ij->j", Bm, Bm))
    target = (rtol * bnorm) ** 2
    it = 0
    while it < max_iter:
        active = rr > target
        if not np.any(active):
            break
        Q = A @ P
        pq = np.einsum("ij,ij->j", P, Q)
        alpha = np.where(active & (pq > 0), rr / np.where(pq > 0, pq, 1.0), 0.0)
        X += P * alpha
        R -= Q * alpha
        rr_new = np.einsum("ij,ij->j", R, R)
        beta = np.where(active & (rr > 0), rr_new / np.where(rr > 0, rr, 1.0), 0.0)
        P = R + P * beta
        rr = rr_new
        it += 1
    return X, it


def block_pcg_jacobi(A, Bm: np.ndarray, X0: np.ndarray | None = None, rtol: float = 1e-13,
                     max_iter: int = 20000):
    """As block_cg, preconditioned with the diagonal of A (Jacobi).

    Step 1 of §4.1 only asks for W = (H + sigma)^-1 U; the paper does not say how
    the source problems are solved.  This is textbook preconditioned CG with
    M = diag(A): z = M^-1 r, rho = r . z, alpha = rho / (p . A p),
    beta = rho_new / rho, p = z + beta p.  Each column stops on the same test as
    block_cg, ||r_j|| <= rtol ||b_j|| (the unpreconditioned residual).
    Returns (X, iterations).
    """
    d = np.asarray(A.diagonal(), dtype=np.float64)
    X = np.zeros_like(Bm) if X0 is None else np.array(X0, dtype=np.float64)
    R = Bm - A @ X
    Z = R / d[:, None]
    P = Z.copy()
    rho = np.einsum("ij,ij->j", R, Z)
    rr = np.einsum("ij,ij->j", R, R)
    bnorm = np.sqrt(np.einsum("ij,ij->j", Bm, Bm))
    target = (rtol * bnorm) ** 2
    it = 0
    while it < max_iter:
        active = rr > target
        if not np.any(active):
            break
        Q = A @ P
        pq = np.einsum("ij,ij->j", P, Q)
        alpha = np.where(active & (pq > 0), rho / np.where(pq > 0, pq, 1.0), 0.0)
        X += P * alpha
        R -= Q * alpha
        Z = R / d[:, None]
        rho_new = np.einsum("ij,ij->j", R, Z)
        beta = np.where(active & (rho > 0), rho_new / np.where(rho > 0, rho, 1.0), 0.0)
        P = Z + P * beta
        rho = rho_new
        rr = np.einsum("ij,ij->j", R, R)
        it += 1
    return X, it


class SourceSolver:
    """Step 1 of §4.1: W = G U with G = (H + sigma)^-1, solved to (near) exactness.

    Sparse LU (SuperLU) when n <= direct_max, else CG to relative residual
    ``cg_rtol`` per column, warm-started from the previous W.
    """

    def __init__(self, H: sp.csr_matrix, sigma: float, direct_max: int = 70000,
                 cg_rtol: float = 1e-13):
        n = H.shape[0]
        self.A = (H + sigma * sp.identity(n, format="csr")).tocsr()
        self.lu = (spla.splu(self.A.tocsc(), permc_spec="MMD_AT_PLUS_A")
                   if n <= direct_max else None)
        self.cg_rtol = cg_rtol
        self.last_iters = 0

    def solve(self, U: np.ndarray, W0: np.ndarray | None = None) -> np.ndarray:
        if self.lu is not None:
            self.last_iters = 0
            return self.lu.solve(np.asarray(U, dtype=np.float64))
        W, self.last_iters = block_cg(self.A, U, W0, self.cg_rtol)
        return W


# ----------------------------------------------------------------------------
# Steps 2-4 of §4.1
# ----------------------------------------------------------------------------
def core_matrices(W: np.ndarray, U: np.ndarray, tau: float):
    """Steps 2 and 3 of §4.1 (Theorem 4.1 gives the well-posedness).

    Step 2: I = (I + tau^2/4 <GU,GU> - tau^2/4 <GU,U><GU,U>) B.
    Step 3: (tau/2) A = I - B + (tau/2) <GU,U> B.
    Returns (A, B, M) with M the Step-2 matrix (M - I is PSD by Lemma 3.1).
    """
    return core_from_inner(inner(W, U), inner(W, W), tau)


def core_from_inner(C: np.ndarray, S: np.ndarray, tau: float):
    """Steps 2 and 3 of §4.1 from the inner matrices C = <GU, U> and S = <GU, GU>.

    The same arithmetic as core_matrices, for callers that hold C and S but not the
    blocks (a row-sharded run sums them over its slabs).  Returns (A, B, M).
    """
    I = np.eye(C.shape[0])
    M = I + (tau * tau / 4.0) * S - (tau * tau / 4.0) * (C @ C)
    B = np.linalg.solve(M, I)
    A = (2.0 / tau) * (I - B + (tau / 2.0) * (C @ B))
    return A, B, M


def midpoint_coefficients(W: np.ndarray, U: np.ndarray, tau: float):
    """Exact solution of the midpoint scheme (4.1) when W is any n x p block.

    (4.1) with L V = U <W, V> - W <U, V> (the operator L_U of (3.2) with GU
    replaced by W) is solved by U^{n+1} = U - tau U A + tau W B with
    A = <W, U^{n+1/2}>, B = <U, U^{n+1/2}> as in §4.1.  Repeating the
    derivation of Steps 2-3 under <U, U> = I but without using the symmetry
    of C = <W, U> (it holds only for the exact W = GU) gives
        (I + tau/2 (C - C^T) + tau^2/4 (S - C C^T)) B = I,
        tau/2 A = I - B + tau/2 C^T B,
    which is Steps 2-3 when C = C^T.  Since L is skew-symmetric for every W
    (Lemma 3.2 uses only the algebra), the step is an exact Cayley transform and
    keeps <U, U> for any W, e.g. an inexact Step-1 solve.  Returns (A, B).
    """
    p = U.shape[1]
    I = np.eye(p)
    C = inner(W, U)
    S = inner(W, W)
    M = I + (tau / 2.0) * (C - C.T) + (tau * tau / 4.0) * (S - C @ C.T)
    B = np.linalg.solve(M, I)
    A = (2.0 / tau) * (I - B + (tau / 2.0) * (C.T @ B))
    return A, B


def update(U: np.ndarray, W: np.ndarray, A: np.ndarray, B: np.ndarray, tau: float) -> np.ndarray:
    """Step 4 of §4.1 / (4.1*): U^{n+1} = U^n - tau U^n A^n + tau G U^n B^n."""
    return U - tau * (U @ A) + tau * (W @ B)


def step_coefficients(W: np.ndarray, U: np.ndarray, tau: float):
    """Step 4 written as U^{n+1} = U K_U + W K_W: K_U = I - tau A, K_W = tau B."""
    A, B, _ = core_matrices(W, U, tau)
    p = U.shape[1]
    return np.eye(p) - tau * A, tau * B


def scheme_step(U: np.ndarray, W: np.ndarray, tau: float) -> np.ndarray:
    """One time step (4.1) given W = G U^n (Steps 2-4)."""
    A, B, _ = core_matrices(W, U, tau)
    return update(U, W, A, B, tau)


def cayley_coefficients(W: np.ndarray, U: np.ndarray, tau: float):
    """The midpoint step (4.1) for any U, without assuming <U, U> = I.

    With Y = [U W] and J = [[0, -I], [I, 0]], the operator of (4.1),
    L V = W <U, V> - U <W, V>, is Y J Y^T V, and the midpoint step is the Cayley
    transform U+ = (I - tau/2 L)^-1 (I + tau/2 L) U.  The Woodbury identity turns it
    into one 2p x 2p solve with the joint Gram Y^T Y = [[D, C^T], [C, S]]
    (D = <U,U>, C = <W,U>, S = <W,W>):
        (I - tau/2 Y^T Y J) Z = Y^T U = [D; C],   U+ = U (I - tau Z_2) + W (tau Z_1),
    Z_1, Z_2 the top and bottom p rows of Z.  For <U, U> = I this is Steps 2-4; for
    any U it keeps <U, U> exactly (an orthogonal transform), where the p x p Steps
    2-3 assume <U, U> = I.  Returns (K_U, K_W).
    """
    p = U.shape[1]
    I = np.eye(p)
    D = inner(U, U)
    C = inner(W, U)
    S = inner(W, W)
    M2 = np.block([[I - (tau / 2.0) * C.T, (tau / 2.0) * D],
                   [-(tau / 2.0) * S, I + (tau / 2.0) * C]])
    Z = np.linalg.solve(M2, np.vstack([D, C]))
    return I - tau * Z[p:], tau * Z[:p]


def l2_flow_step(H, sigma: float, U: np.ndarray, tau: float) -> np.ndarray:
    """One midpoint step of the L2 gradient flow the paper contrasts its model with (§1).

    The earlier orthogonality-preserving schemes evolve the orbitals by the L2 gradient
    flow dU/dt = -(H U - U <H U, U>).  For <U, U> = I this is the model of §2.2 with
    G U replaced by -H U: dU/dt = W <U, U> - U <W, U> with W = -H U.  The midpoint step
    is taken as the exact Cayley transform (cayley_coefficients) with
    W = -(H + sigma) U; the shift cancels in U+.  Its time step is limited by the mesh
    (a CFL condition).  (With the p x p Steps 2-3, which assume <U, U> = I, this flow
    amplifies the rounding drift of <U, U> until it diverges.)
    """
    Hs = H + sigma * sp.identity(H.shape[0], format="csr")
    W = -(Hs @ U)
    KU, KW = cayley_coefficients(W, U, tau)
    return U @ KU + W @ KW


# ----------------------------------------------------------------------------
# Monitored quantities
# ----------------------------------------------------------------------------
def energy(H, U: np.ndarray) -> float:
    """E(U) = 1/2 (U, U)_a = 1/2 tr(U^T H U) (§2.2), unshifted H."""
    return 0.5 * float(np.einsum("ij,ij->", U, H @ U))


def orth_error(U: np.ndarray) -> float:
    """||I - <U, U>||_F, the orthogonality error plotted in Fig. 1(b)."""
    return float(np.linalg.norm(np.eye(U.shape[1]) - inner(U, U)))


def residuals(H, U: np.ndarray, hnorm: float):
    """Residuals of the (rotation-invariant) Rayleigh-Ritz pair (U, Theta).

    Theta = U^T H U, R = H U - U Theta.  Returns
      r      = ||R||_F / (hnorm sqrt(p))        (backward-error normalisation)
      r_theta= ||R||_F / ||Theta||_F
      r_i    = ||H u_i - lambda_i u_i|| for the Ritz vectors (cf. §5.2, Table 2)
    """
    HU = H @ U
    Th = inner(U, HU)
    R = HU - U @ Th
    nr = float(np.linalg.norm(R))
    p = U.shape[1]
    lam, Y = np.linalg.eigh(0.5 * (Th + Th.T))
    Ur = U @ Y
    ri = np.linalg.norm(H @ Ur - Ur * lam, axis=0)
    return nr / (hnorm * math.sqrt(p)), nr / float(np.linalg.norm(Th)), ri


def paper_eigenvalues(W: np.ndarray, U: np.ndarray, sigma: float) -> np.ndarray:
    """§5 error measures: lambda_i = eig(<GU, U>^-1), shifted back by -sigma."""
    C = inner(W, U)
    mu = np.linalg.eigvals(np.linalg.inv(C))
    return np.sort(mu.real) - sigma


def ritz_values(H, U: np.ndarray) -> np.ndarray:
    """Eigenvalues of Theta = U^T H U (ascending)."""
    Th = inner(U, H @ U)
    return np.linalg.eigvalsh(0.5 * (Th + Th.T))


def energy_lower_bound(W: np.ndarray, U: np.ndarray, sigma: float) -> float:
    """1/2 tr(<GU,U>^-1) - p sigma / 2 <= E(U) for orthonormal U (Loewner order:
    (U^T G U)^-1 <= U^T (H + sigma) U); equality at an invariant subspace."""
    C = inner(W, U)
    return 0.5 * float(np.trace(np.linalg.inv(0.5 * (C + C.T)))) - 0.5 * U.shape[1] * sigma


# ----------------------------------------------------------------------------
# Algorithm 1
# ----------------------------------------------------------------------------
@dataclass
class RunResult:
    U: np.ndarray
    W: np.ndarray
    steps: int
    converged: bool
    energy: list = field(default_factory=list)      # E(U^n), n = 0..steps
    err_E: list = field(default_factory=list)       # |E^{n+1}-E^n| / |E^n|
    orth: list = field(default_factory=list)        # ||I - <U^n,U^n>||_F
    resid: list = field(default_factory=list)       # backward-error residual r
    cg_iters: list = field(default_factory=list)
    sigma: float = 0.0
    tau: float = 0.0


def run(shape, lo, hi, V, U0: np.ndarray, *, tau: float | None = None,
        sigma: float | None = None, tol: float = 1e-10, max_steps: int = 10000,
        stop: str = "err_E", E_ref: float | None = None, track_residual: bool = True,
        orthonormalize: bool = True, direct_max: int = 70000, cg_rtol: float = 1e-13,
        callback=None) -> RunResult:
    """Algorithm 1 of §4.1 with a uniform time step (the setting of §5).

    ``stop``:
      * ``"err_E"``    Algorithm 1: |E(U^{n+1}) - E(U^n)| / |E(U^n)| <= tol
                       (err_E^0 = |E(U^0)|);
      * ``"E_ref"``    §5: (E(U^n) - E_ref) / |E_ref| < tol;
      * ``"residual"`` backward-error residual r <= tol (see ``residuals``);
      * ``"steps"``    exactly ``max_steps`` steps.
    """
    H = hamiltonian(shape, lo, hi, V)
    if sigma is None:
        sigma = default_sigma(shape, lo, hi, V)
    if tau is None:
        tau = default_tau(shape, lo, hi, V, sigma)
    hnorm = gershgorin_norm(shape, lo, hi, V, sigma)
    U = householder_orthonormalize(U0) if orthonormalize else np.array(U0, dtype=np.float64)
    solver = SourceSolver(H, sigma, direct_max=direct_max, cg_rtol=cg_rtol)

    res = RunResult(U=U, W=None, steps=0, converged=False, sigma=sigma, tau=tau)
    E = energy(H, U)
    res.energy.append(E)
    res.orth.append(orth_error(U))
    if track_residual or stop == "residual":
        res.resid.append(residuals(H, U, hnorm)[0])
    err = abs(E)
    W = None
    n = 0
    while n < max_steps:
        if stop == "err_E" and err <= tol:
            res.converged = True
            break
        if stop == "E_ref" and (E - E_ref) / abs(E_ref) < tol:
            res.converged = True
            break
        if stop == "residual" and res.resid[-1] <= tol:
            res.converged = True
            break
        W = solver.solve(U, W)                       # Step 1
        res.cg_iters.append(solver.last_iters)
        U = scheme_step(U, W, tau)                   # Steps 2-4
        E_new = energy(H, U)
        err = abs(E_new - E) / abs(E)
        E = E_new
        n += 1
        res.energy.append(E)
        res.err_E.append(err)
        res.orth.append(orth_error(U))
        if track_residual or stop == "residual":
            res.resid.append(residuals(H, U, hnorm)[0])
        if callback is not None:
            callback(n, U, W)
    else:
        if stop == "steps":
            res.converged = True
    res.U, res.W, res.steps = U, W, n
    return res
