"""The 128^3 x 1024 configuration restricted to a 32^3 grid: the same kind of
potential (harmonic trap plus 32 wells on [-8, 8]^3) with p = 1024.

One time step of every precision mode is compared with the FP64 oracle's step
from the same U0 (exact Step 1).  This exercises the paths that only wide blocks
take:
- the LU core solve for p > 128;
- 8 x 8 tiles of the tensor-core Gram and update;
- 32 column chunks of the TMA CG kernel.

Step-1 tolerances are fixed (cg_rtol) so that the step is comparable.
Expected agreement:
- FP64: CG error 1e-12 plus rounding;
- FP32: CG rtol 1e-6 times tau ||B|| (about 1.5e-6) plus FP32 rounding;
- TF32: a 2^-11 relative operand rounding in the Gram and update;
- BF16 x 3: as FP32 (three-piece operands to 2^-24).
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

#           cg_rtol  max|dU| / max|U|  ||U^T U - I||_F  |dE| / |E|
# (measured on GB300: fp64 7.5e-13 / 2.7e-13 / 1.4e-15; fp32 1.0e-6 / 1.2e-6 / 3.5e-8;
#  mix_tf32 6.7e-5 / 6.8e-4 / 8.6e-6)
MODES = {"fp64": (1e-12, 1e-11, 1e-11, 1e-13),
         "fp32": (1e-6, 1e-5, 1e-5, 1e-6),
         "mix_tf32": (1e-6, 5e-4, 5e-3, 1e-4),
         "mix_bf16x3": (1e-6, 1e-5, 1e-5, 1e-6)}


@pytest.fixture(scope="module")
def restricted():
    P = syn.wells_3d(32, 1024, 32, seed=3)
    U0 = syn.gaussian_block(3, P.n, P.p)
    H = o.hamiltonian(P.shape, P.lo, P.hi, P.V)
    sigma = o.default_sigma(P.shape, P.lo, P.hi, P.V)
    tau = o.default_tau(P.shape, P.lo, P.hi, P.V, sigma)
    U = o.householder_orthonormalize(U0)
    U1 = o.scheme_step(U, o.SourceSolver(H, sigma).solve(U), tau)
    return P, U0, U1, o.energy(H, U1)


@pytest.mark.parametrize("prec", list(MODES))
def test_one_step_p1024_matches_oracle(restricted, prec):
    P, U0, U1, E1 = restricted
    rtol, du_tol, orth_tol, e_tol = MODES[prec]
    with pkg.Solver(P.shape, P.lo, P.hi, P.V, U0, P.p, prec=prec, cg_rtol=rtol) as s:
        st = s.step(1)
        U = s.get_U()
    du = np.abs(U - U1).max() / np.abs(U1).max()
    orth = np.linalg.norm(U.T @ U - np.eye(P.p))
    print(f"{prec}: max|dU|/max|U| {du:.2e}  orth {orth:.2e}  dE/E {abs(st['energy'] - E1) / abs(E1):.2e}")
    assert du <= du_tol
    assert orth <= orth_tol
    assert st["energy"] == pytest.approx(E1, rel=e_tol)
