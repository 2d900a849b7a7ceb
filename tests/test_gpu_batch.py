"""Batches of uneven problems advanced by graph-captured batched kernels.

Checks (FP32 contexts): a batch reproduces the per-problem path step by step;
a batched solve reaches the dense-eigensolve eigenvalues of every problem; the
err_E rule freezes problems on the device; the autotuner writes and reuses its
cache; the launch counter counts graph replays.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as o
import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2511_06788_gb300 as pkg  # noqa: E402

# (N, p, wells, seed) with spectral gaps giving 17-123 steps per decade of residual
SHAPES = [(10, 8, 3, 0), (14, 13, 5, 26), (13, 16, 6, 26), (8, 12, 2, 15)]


def make(shapes, prec="fp32", **kw):
    probs = [syn.wells_3d(N, p, w, s) for N, p, w, s in shapes]
    solvers = [pkg.Solver(P.shape, P.lo, P.hi, P.V, syn.gaussian_block(i, P.n, P.p), P.p,
                          prec=prec, **kw) for i, P in enumerate(probs)]
    return probs, solvers


def test_batch_steps_match_single_problem_steps():
    probs, single = make(SHAPES)
    _, batched = make(SHAPES)
    for s in single:
        s.step(5)
    with pkg.Batch(batched, cg_iters=200) as b:
        b.step(5)
        for s1, s2, P in zip(single, batched, probs):
            st1, st2 = s1.stats(), s2.stats()
            assert st2["steps"] == 5
            assert st2["energy"] == pytest.approx(st1["energy"], rel=2e-5)
            U1, U2 = s1.get_U(), s2.get_U()
            # same iteration up to FP32 rounding of differently partitioned reductions
            assert np.abs(U1 - U2).max() < 2e-3 * np.abs(U1).max()
            assert np.linalg.norm(U2.T @ U2 - np.eye(P.p)) < 1e-5
    for s in single + batched:
        s.close()


def test_batch_solve_reaches_dense_eigenvalues():
    probs, solvers = make(SHAPES)
    with pkg.Batch(solvers, cg_iters=16) as b:
        nconv = b.solve(1e-6, 4000, pkg.OP_STOP_RESIDUAL, check_every=20)
        assert nconv == len(probs)
        for i, (s, P) in enumerate(zip(solvers, probs)):
            lam = np.linalg.eigvalsh(o.hamiltonian(P.shape, P.lo, P.hi, P.V).toarray())[: P.p]
            np.testing.assert_allclose(s.eigenvalues(), lam, rtol=1e-5)
            U = s.get_U()
            assert np.linalg.norm(U.T @ U - np.eye(P.p)) < 1e-5
            assert b.stats(i)["frozen"] == 1
    for s in solvers:
        s.close()


def test_batch_err_E_rule_freezes_on_device():
    probs, solvers = make(SHAPES[:2])
    with pkg.Batch(solvers, cg_iters=16) as b:
        b.solve(1e-9, 3000, pkg.OP_STOP_ERR_E, check_every=50)
        for i in range(len(probs)):
            st = b.stats(i)
            assert st["frozen"] == 1 and st["err_E"] <= 1e-9
        steps = [b.stats(i)["steps"] for i in range(len(probs))]
        b.step(3)  # frozen problems do not move
        assert [b.stats(i)["steps"] for i in range(len(probs))] == steps
    for s in solvers:
        s.close()


def test_autotuner_writes_and_reuses_cache(tmp_path):
    probs, solvers = make(SHAPES)
    cache = str(tmp_path / "tiles.jsonl")
    with pkg.Batch(solvers, cg_iters=8) as b:
        ms = b.autotune(cache, steps_per_trial=1)
        assert ms > 0 and os.path.exists(cache)
        entry = json.loads(open(cache).read().strip().splitlines()[-1])
        assert (entry["rows_per_item"], entry["gram_rows"]) == b.tiles()
        b.set_tiles(128, 1024)
        b.autotune(cache, steps_per_trial=1)  # cached: no new trials, same tiles
        assert b.tiles() == (entry["rows_per_item"], entry["gram_rows"])
        assert len(open(cache).read().strip().splitlines()) == 1
    for s in solvers:
        s.close()


def test_batch_counts_graph_replays_as_launches():
    probs, solvers = make(SHAPES[:2])
    with pkg.Batch(solvers, cg_iters=4) as b:
        L = pkg.lib()
        n0 = L.op_kernel_launches()
        b.step(2)
        per_step = (L.op_kernel_launches() - n0) / 2
        # set_tol + cg_init + fin + 4 x 4 CG + gram 2 + core 7 + update 2 + energy 2 + end
        assert per_step == 1 + 2 + 16 + 2 + 7 + 2 + 2 + 1
    for s in solvers:
        s.close()


def test_batch_rejects_fp64_contexts():
    _, solvers = make(SHAPES[:1], prec="fp64")
    with pytest.raises(pkg.OpError):
        pkg.Batch(solvers)
    solvers[0].close()


def test_batch_solve_with_adaptive_shift():
    """Per-problem shift re-tuning inside the batch: same eigenvalues, shifts moved,
    and no more steps than with fixed shifts."""
    probs, fixed = make(SHAPES)
    _, adapt = make(SHAPES, adapt_every=50)
    steps = {}
    for name, solvers in (("fixed", fixed), ("adapt", adapt)):
        with pkg.Batch(solvers, cg_iters=16) as b:
            assert b.solve(1e-6, 4000, pkg.OP_STOP_RESIDUAL, check_every=10) == len(probs)
            steps[name] = [b.stats(i)["steps"] for i in range(len(probs))]
            sig = [b.stats(i)["sigma"] for i in range(len(probs))]
        for s, P in zip(solvers, probs):
            lam = np.linalg.eigvalsh(o.hamiltonian(P.shape, P.lo, P.hi, P.V).toarray())[: P.p]
            np.testing.assert_allclose(s.eigenvalues(), lam, rtol=1e-5)
        if name == "adapt":
            assert any(a > f for a, f in zip(sig, [st.stats()["sigma"] for st in fixed]))
    print("steps fixed", steps["fixed"], "adaptive", steps["adapt"])
    assert sum(steps["adapt"]) <= sum(steps["fixed"])
    for s in fixed + adapt:
        s.close()


# Five problems of the 64-problem workload (synthetic.batch_problems(0)): a 48^3 grid,
# p = 96, and three more between 26^3 and 46^3 with p from 22 to 69.
C4_PICK = (43, 46, 0, 1, 37)


def test_batch_step_matches_oracle_at_the_batch_workload_sizes():
    """One batched step against the oracle's step with an exact Step 1 (§4.1, Steps 1-4),
    problem by problem, from the same U (the FP32 values each context holds).  The batch
    solves Step 1 to the FP32 floor (cg_rtol 1e-6, enough iterations to converge); the
    expected agreement is that of one FP32 step at p = 1024: CG rtol 1e-6 times tau ||B||
    plus FP32 rounding, max|dU| / max|U| <= 1e-5, ||U^T U - I||_F <= 1e-5 and
    |dE| / |E| <= 1e-6."""
    allp = syn.batch_problems(0, 64)
    probs = [allp[i] for i in C4_PICK]
    assert max(P.shape[0] for P in probs) == 48 and max(P.p for P in probs) == 96
    solvers = [pkg.Solver(P.shape, P.lo, P.hi, P.V, syn.gaussian_block(100 + i, P.n, P.p), P.p,
                          prec="fp32", cg_rtol=1e-6) for i, P in zip(C4_PICK, probs)]
    U0 = [s.get_U() for s in solvers]
    with pkg.Batch(solvers, cg_iters=200) as b:
        b.step(1)
        out = [(s.get_U(), b.stats(i)) for i, s in enumerate(solvers)]
    for (U, st), Ua, P in zip(out, U0, probs):
        assert st["steps"] == 1 and st["last_cg_iters"] < 200  # converged before the cap
        H = o.hamiltonian(P.shape, P.lo, P.hi, P.V.astype(np.float32).astype(np.float64))
        W = o.SourceSolver(H, st["sigma"], cg_rtol=1e-11).solve(Ua)
        U1 = o.scheme_step(Ua, W, st["tau"])
        E1 = o.energy(H, U1)
        du = np.abs(U - U1).max() / np.abs(U1).max()
        orth = np.linalg.norm(U.T @ U - np.eye(P.p))
        print(f"{P.name}: max|dU|/max|U| {du:.2e} orth {orth:.2e} "
              f"dE/E {abs(st['energy'] - E1) / abs(E1):.2e} cg {st['last_cg_iters']}")
        assert du <= 1e-5
        assert orth <= 1e-5
        assert st["energy"] == pytest.approx(E1, rel=1e-6)
    for s in solvers:
        s.close()
