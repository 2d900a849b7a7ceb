"""Precision modes against a dense FP64 eigensolve (the oracle's H, eigvalsh).

Stated tolerances (max relative eigenvalue error, ||U^T U - I||_F) at the
residual each mode reaches:
  OP_FP64      1e-10, 1e-12   (residual 1e-10)
  OP_FP32      1e-5,  1e-5    (residual 1e-6; tensor-core Gram/update with TF32
                               hi/lo splits, FP64 core)
  OP_MIX_TF32  2e-3,  5e-3    (one TF32 MMA per product: operands rounded to 2^-11
                               relative; the residual stalls near 1e-5, so this
                               mode does not meet the 1e-5 target)
  OP_MIX_BF16X3 1e-5, 1e-5    (residual 1e-6; BF16 pieces x = b0 + b1 + b2 to 2^-24,
                               six MMAs per product, FP64 core)
  OP_MIX_BF16  2e-2,  5e-2    (one BF16 MMA per product: operands rounded to 2^-9
                               relative; stalls like TF32-only, earlier)
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

MODES = {
    "fp64": (1e-10, 20000, 1e-10, 1e-12),
    "fp32": (1e-6, 20000, 1e-5, 1e-5),
    "mix_tf32": (1e-6, 1500, 2e-3, 5e-3),
    "mix_bf16x3": (1e-6, 20000, 1e-5, 1e-5),
    "mix_bf16": (1e-6, 1500, 2e-2, 5e-2),
}


@pytest.fixture(scope="module")
def problem():
    P = syn.wells_3d(24, 20, 6, 4)
    lam = np.linalg.eigvalsh(o.hamiltonian(P.shape, P.lo, P.hi, P.V).toarray())
    return P, lam


@pytest.mark.parametrize("prec", list(MODES))
def test_precision_mode_accuracy(problem, prec):
    P, lam = problem
    tol, max_steps, eig_tol, orth_tol = MODES[prec]
    with pkg.Solver(P.shape, P.lo, P.hi, P.V, syn.gaussian_block(0, P.n, P.p), P.p,
                    prec=prec) as s:
        st = s.solve(tol, max_steps, pkg.OP_STOP_RESIDUAL, raise_on_max=False)
        ritz = s.eigenvalues()
        U = s.get_U()
    err = float(np.abs(ritz / lam[: P.p] - 1.0).max())
    orth = float(np.linalg.norm(U.T @ U - np.eye(P.p)))
    print(f"{prec}: steps {st['steps']} residual {st['residual']:.2e} eig {err:.2e} orth {orth:.2e}")
    if prec not in ("mix_tf32", "mix_bf16"):
        assert st["converged"]
    assert err <= eig_tol and orth <= orth_tol
