"""Adaptive shift and time step (op_problem.adapt_every) against fixed ones.

The fixed points of the scheme do not depend on sigma or tau, so an adaptive
solve must reach the same eigenvalues as the reference.  Here the reference is
ARPACK shift-invert on the oracle's H.  With the shift re-tuned towards
lambda_p - 2 lambda_1, it should need fewer steps.
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
from scipy.sparse.linalg import eigsh  # noqa: E402


@pytest.fixture(scope="module")
def problem():
    P = syn.wells_3d(24, 20, 6, 4)
    H = o.hamiltonian(P.shape, P.lo, P.hi, P.V)
    lam = np.sort(eigsh(H.tocsc(), k=P.p + 1, sigma=float(P.V.min()) - 1.0, which="LM",
                        return_eigenvectors=False))
    return P, lam


@pytest.mark.parametrize("prec,tol,eig_tol", [("fp32", 1e-6, 1e-5), ("fp64", 1e-9, 1e-9)])
def test_adaptive_shift_same_eigenvalues_fewer_steps(problem, prec, tol, eig_tol):
    P, lam = problem
    U0 = syn.gaussian_block(9, P.n, P.p)
    res = {}
    for adapt in (0, 50):
        with pkg.Solver(P.shape, P.lo, P.hi, P.V, U0, P.p, prec=prec, adapt_every=adapt) as s:
            sigma0 = s.stats()["sigma"]
            st = s.solve(tol, 20000)
            ev = s.eigenvalues()
            U = s.get_U()
        err = np.max(np.abs(ev - lam[:P.p]) / np.abs(lam[:P.p]).clip(1e-3))
        res[adapt] = (st["steps"], st["sigma"], st["cg_iters"], err)
        print(prec, adapt, "steps", st["steps"], "sigma", sigma0, "->", st["sigma"],
              "cg", st["cg_iters"], "eig err", err)
        assert err <= eig_tol
        assert np.linalg.norm(U.T @ U - np.eye(P.p)) <= (1e-5 if prec == "fp32" else 1e-12)
    assert res[50][1] > res[0][1]           # the shift moved
    assert res[50][0] < res[0][0]           # and the solve took fewer steps
