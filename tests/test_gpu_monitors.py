"""Parity of the monitored quantities of Algorithm 1 (§4.1) and the error measures of §5
with the FP64 oracle, on the same U, through the C ABI.

Quantities: the residual r = ||H U - U Theta||_F / (||H + sigma||_G sqrt(p)) of the stop
rule (op_residual), the G-residual tr<W,W> - ||<W,U>||_F^2 and the orthogonality error
||<U,U> - I||_F of the U entering a step (op_stats), the paper's eigenvalues
eig(<GU,U>^-1) - sigma and the Ritz values eig(U^T H U) (op_eigenvalues).

Tolerances (derived from the arithmetic).  FP64: the library and the oracle differ in
summation order and, for quantities that use Step 1, in the Step-1 solve (CG to 1e-13
against a sparse direct solve).  FP32: the blocks are stored in FP32 and every block
kernel rounds to FP32; an entry of H U, <U,V> or U Theta carries a relative error of a few
2^-24 of the sum of the magnitudes it adds, so r carries an absolute error of at most a
few 1e-7 times ||H U||_F / (||H+sigma||_G sqrt(p)) <= 1, the G-residual one of about
1e-6 tr<W,W> (the Step-1 solve stops at 1e-6), and the paper's eigenvalue lambda_i one of
about 1e-6 (lambda_i + sigma)^2 / (lambda_1 + sigma).
"""
import math

import numpy as np
import pytest

import oracle as o
import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2511_06788_gb300 as pkg  # noqa: E402

PROBLEMS = {
    "laplace2d_32x32_p8": lambda: syn.config_2d_laplace(),
    "wells3d_24^3_p40": lambda: syn.wells_3d(24, 40, 8, 5),
}


def _V_used(P, prec):
    # FP32 contexts keep V in FP32 on the device
    return P.V if prec == "fp64" else P.V.astype(np.float32).astype(np.float64)


@pytest.fixture(scope="module", params=list(PROBLEMS))
def problem(request):
    P = PROBLEMS[request.param]()
    return P, syn.gaussian_block(17, P.n, P.p)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_residual_matches_oracle_on_the_same_U(problem, prec):
    P, U0 = problem
    H = o.hamiltonian(P.shape, P.lo, P.hi, _V_used(P, prec))
    with pkg.Solver(P.shape, P.lo, P.hi, P.V, U0, P.p, prec=prec) as s:
        sigma = s.stats()["sigma"]
        hnorm = o.gershgorin_norm(P.shape, P.lo, P.hi, P.V, sigma)
        seen = []
        for k in (0, 5, 40):
            if k:
                s.step(k)
            U = s.get_U()
            r_gpu = s.residual()
            r_orc = o.residuals(H, U, hnorm)[0]
            scale = float(np.linalg.norm(H @ U)) / (hnorm * math.sqrt(P.p))
            tol = (1e-12 * r_orc + 1e-14 * scale) if prec == "fp64" else 2e-6 * scale
            assert abs(r_gpu - r_orc) <= tol, (k, r_gpu, r_orc)
            assert s.stats()["residual"] == r_gpu
            seen.append(r_orc)
    assert seen[-1] < seen[0]  # the run makes progress, so the stages differ


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_g_residual_and_orthogonality_of_a_non_orthonormal_U(problem, prec):
    """Load a U with <U,U> != I (through a checkpoint) and take one step with a tight
    Step-1 solve: the step's statistics are those of that U and its W = G U."""
    P, U0 = problem
    n, p, ld = P.n, P.p, (P.p + 7) // 8 * 8
    rtol = 1e-13 if prec == "fp64" else 1e-6
    with pkg.Solver(P.shape, P.lo, P.hi, P.V, U0, P.p, prec=prec, cg_rtol=rtol,
                    cg_max_iter=20000) as s:
        s.step(2)
        sigma = s.stats()["sigma"]
        buf = s.checkpoint()
        elem = 8 if prec == "fp64" else 4
        # the header, then U (then W, and for FP64 contexts the block before the last
        # update); the header is shorter than a block
        hdr = buf.size % (n * ld * elem)
        dt = np.float64 if prec == "fp64" else np.float32
        Ublk = buf[hdr:hdr + n * ld * elem].view(dt).reshape(n, ld)
        rng = np.random.default_rng(4)
        # a perturbation of size ~1e-3 that breaks <U,U> = I
        Up = Ublk[:, :p].astype(np.float64) @ (np.eye(p) + 1e-3 * rng.standard_normal((p, p)))
        Ublk[:, :p] = Up.astype(dt)
        s.restore(buf)
        st = s.step(1)
    U = Ublk[:, :p].astype(np.float64)  # exactly the values the context held
    H = o.hamiltonian(P.shape, P.lo, P.hi, _V_used(P, prec))
    W = o.SourceSolver(H, sigma).solve(U)
    C, S, D = W.T @ U, W.T @ W, U.T @ U
    g_res = float(np.trace(S) - np.sum(C * C))
    orth = float(np.linalg.norm(D - np.eye(p)))
    assert orth > 1e-4
    if prec == "fp64":
        assert st["orth"] == pytest.approx(orth, rel=1e-10)
        assert abs(st["g_residual"] - g_res) <= 1e-10 * float(np.trace(S))
    else:
        assert abs(st["orth"] - orth) <= 1e-6 * p
        assert abs(st["g_residual"] - g_res) <= 1e-5 * float(np.trace(S))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_paper_and_ritz_eigenvalues_match_oracle(problem, prec):
    P, U0 = problem
    H = o.hamiltonian(P.shape, P.lo, P.hi, _V_used(P, prec))
    with pkg.Solver(P.shape, P.lo, P.hi, P.V, U0, P.p, prec=prec) as s:
        s.step(30)
        sigma = s.stats()["sigma"]
        hnorm = o.gershgorin_norm(P.shape, P.lo, P.hi, P.V, sigma)
        U = s.get_U()
        ritz = s.eigenvalues(pkg.binding.OP_EIG_RITZ)
        paper = s.eigenvalues(pkg.binding.OP_EIG_PAPER)
    ritz_o = o.ritz_values(H, U)
    W = o.SourceSolver(H, sigma).solve(U)
    paper_o = o.paper_eigenvalues(W, U, sigma)
    if prec == "fp64":
        np.testing.assert_allclose(ritz, ritz_o, rtol=1e-12, atol=1e-13 * hnorm)
        np.testing.assert_allclose(paper, paper_o, rtol=1e-10)
    else:
        np.testing.assert_allclose(ritz, ritz_o, rtol=0, atol=2e-6 * hnorm)
        l1 = paper_o[0] + sigma
        tol = 4e-6 * (paper_o + sigma) ** 2 / l1
        assert np.all(np.abs(paper - paper_o) <= tol), np.max(np.abs(paper - paper_o) / tol)
