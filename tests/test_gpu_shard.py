"""Row-sharded steps (op_step_sharded) through the C ABI.

The grid is split into slabs of whole planes along its slowest axis; each slab holds
only its planes plus one halo plane per neighbour, exchanges halo planes before every
stencil apply and contributes partial sums to the CG's dot products, to the three inner
matrices of Steps 2-3 (§4.1) and to the energy.  A run split this way must agree with
the unsplit run of the same context settings up to the order of those sums, and with
the FP64 oracle's steps.

Tolerances.  Both runs solve Step 1 by FP64 CG to a relative residual of 1e-13 per
column; the split changes only the order of the dot products, so the CG iterates agree
to a few 1e-15 relative per iteration and the stopped W to about 1e-13, and U after a
step (a map with coefficients of order one) to about 1e-12.  The oracle solves Step 1
with a sparse direct solver; its W differs from the CG's by at most the 1e-13 tolerance
times the condition number of H + sigma (< 1e3 here), so U agrees to a few 1e-10.
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


def _problem(shape, p, seed, box=6.0):
    lo, hi = (-box,) * len(shape), (box,) * len(shape)
    wells = syn.draw_wells(seed, 4, lo, hi)
    V = syn.potential(shape, lo, hi, 0.5, wells)
    return syn.Problem(tuple(shape), lo, hi, V, p, f"shard_{shape}_p{p}")


def _solver(P, U0, precond, gemm):
    return pkg.Solver(P.shape, P.lo, P.hi, P.V, U0, P.p, prec="fp64", cg_rtol=1e-13,
                      precond=precond, fp64_gemm=gemm, step1="cg")


CASES = [
    # shape, p, slabs, precond, fp64 products
    ((14, 13, 23), 12, 3, "jacobi", "tc"),      # 23 planes: slabs of 8, 8, 7
    ((14, 13, 23), 12, 5, "none", "fma"),       # 5, 5, 5, 4, 4
    ((12, 11, 9), 20, 9, "jacobi", "fma"),      # one plane per slab
    ((12, 11, 9), 20, 1, "jacobi", "tc"),       # one slab: no exchanges
    ((40, 37), 8, 4, "jacobi", "tc"),           # 2-D: slabs along y
]


@pytest.mark.parametrize("shape,p,nslab,precond,gemm", CASES,
                         ids=[f"{'x'.join(map(str, c[0]))}_p{c[1]}_s{c[2]}_{c[3]}_{c[4]}"
                              for c in CASES])
def test_sharded_steps_match_unsplit_steps_and_oracle(shape, p, nslab, precond, gemm):
    P = _problem(shape, p, seed=len(shape) * 100 + p)
    U0 = syn.gaussian_block(31, P.n, P.p)
    nsteps = 3
    with _solver(P, U0, precond, gemm) as a, _solver(P, U0, precond, gemm) as b:
        ref_stats = [a.step(1) for _ in range(nsteps)]
        got = []
        comm_total = {"halo_copies": 0, "halo_bytes": 0, "reductions": 0}
        for _ in range(nsteps):
            st, comm = b.step_sharded(nslab, 1)
            got.append(st)
            for k in comm_total:
                comm_total[k] += comm[k]
            assert comm["slabs"] == nslab
            # the schedule: one halo round for W, one per CG iteration, one for U+; two
            # sums per CG iteration, one at the CG start, the Gram sum, the energy sum
            it = st["last_cg_iters"]
            ld = (p + 7) // 8 * 8
            plane = int(np.prod(shape[:-1]))
            assert comm["halo_copies"] == 2 * (nslab - 1) * (it + 2)
            assert comm["halo_bytes"] == comm["halo_copies"] * plane * ld * 8
            assert comm["reductions"] == 2 * it + 3
            assert comm["reduction_bytes"] == 8 * ld * (3 + 3 * it + 1) + 8 * 3 * ld * ld
        Ua, Ub = a.get_U(), b.get_U()
        # the context continues after sharded steps
        b.step(1)
        a.step(1)
        Ua2, Ub2 = a.get_U(), b.get_U()
    for ra, rb in zip(ref_stats, got):
        assert abs(ra["energy"] - rb["energy"]) <= 1e-12 * abs(ra["energy"])
        assert abs(ra["last_cg_iters"] - rb["last_cg_iters"]) <= 1
        assert abs(ra["orth"] - rb["orth"]) <= 1e-13
    assert np.abs(Ua - Ub).max() <= 1e-11
    assert np.abs(Ua2 - Ub2).max() <= 1e-11
    # the oracle's steps from the same U0 (Householder QR; the library's Cholesky-QR gives
    # the same orthonormal block up to rounding, both with positive R diagonals)
    H = o.hamiltonian(P.shape, P.lo, P.hi, P.V)
    sigma, tau = got[0]["sigma"], got[0]["tau"]
    U = o.householder_orthonormalize(U0)
    G = o.SourceSolver(H, sigma)
    for k in range(nsteps):
        U = o.scheme_step(U, G.solve(U), tau)
        assert abs(o.energy(H, U) - got[k]["energy"]) <= 1e-10 * abs(got[k]["energy"])
    assert np.abs(U - Ub).max() <= 5e-10
    assert o.orth_error(Ub) <= 1e-12


def test_sharded_step_rejects_what_it_does_not_cover():
    P = _problem((10, 9, 8), 4, seed=3)
    U0 = syn.gaussian_block(1, P.n, P.p)
    with _solver(P, U0, "jacobi", "fma") as s:
        for bad in (0, 9):
            with pytest.raises(pkg.OpError) as e:
                s.step_sharded(bad, 1)
            assert e.value.status == pkg.binding.OP_ERR_ARG
        assert s.stats()["steps"] == 0
    with pkg.Solver(P.shape, P.lo, P.hi, P.V, U0, P.p, prec="fp32") as s:
        with pytest.raises(pkg.OpError) as e:
            s.step_sharded(2, 1)
        assert e.value.status == pkg.binding.OP_ERR_ARG
