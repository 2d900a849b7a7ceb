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
