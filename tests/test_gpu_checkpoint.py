"""Checkpoint / resume: a context restored from a checkpoint continues exactly as
the uninterrupted run (the scheme is a one-step map of U, with Step 1 warm-started
from the previous W), and restore rejects buffers of another size or format."""
import numpy as np
import pytest

import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2511_06788_gb300 as pkg  # noqa: E402


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_restored_run_is_bit_identical(prec):
    P = syn.wells_3d(14, 13, 5, 26)
    U0 = syn.gaussian_block(2, P.n, P.p)
    with pkg.Solver(P.shape, P.lo, P.hi, P.V, U0, P.p, prec=prec) as a:
        ea = [a.step(1)["energy"] for _ in range(6)]
        Ua = a.get_U()
        sa = a.stats()
    with pkg.Solver(P.shape, P.lo, P.hi, P.V, U0, P.p, prec=prec) as b:
        b.step(3)
        ck = b.checkpoint()
    # a fresh context of the same problem, started elsewhere, resumes from the checkpoint
    with pkg.Solver(P.shape, P.lo, P.hi, P.V, syn.gaussian_block(7, P.n, P.p), P.p,
                    prec=prec) as c:
        c.restore(ck)
        assert c.stats()["steps"] == 3
        eb = [c.step(1)["energy"] for _ in range(3)]
        Ub = c.get_U()
        sb = c.stats()
    assert np.array_equal(Ua, Ub)
    assert eb == ea[3:]
    assert sb["steps"] == sa["steps"] == 6 and sb["cg_iters"] == sa["cg_iters"]


def test_restore_rejects_other_sizes_and_formats():
    P = syn.wells_3d(10, 8, 3, 0)
    Q = syn.wells_3d(10, 16, 3, 0)
    with pkg.Solver(P.shape, P.lo, P.hi, P.V, syn.gaussian_block(0, P.n, P.p), P.p,
                    prec="fp32") as a, \
         pkg.Solver(Q.shape, Q.lo, Q.hi, Q.V, syn.gaussian_block(0, Q.n, Q.p), Q.p,
                    prec="fp32") as b, \
         pkg.Solver(P.shape, P.lo, P.hi, P.V, syn.gaussian_block(0, P.n, P.p), P.p,
                    prec="fp64") as d:
        ck = a.checkpoint()
        with pytest.raises(pkg.OpError):
            b.restore(ck)           # other p
        with pytest.raises(pkg.OpError):
            d.restore(ck)           # other precision
        bad = ck.copy()
        bad[0] ^= 0xFF
        with pytest.raises(pkg.OpError):
            a.restore(bad)          # not a checkpoint
        with pytest.raises(pkg.OpError):
            a.restore(ck[: ck.size // 2])  # truncated
        a.restore(ck)


def test_run_logged_writes_the_per_step_series(tmp_path):
    import json
    P = syn.wells_3d(10, 8, 3, 0)
    log = tmp_path / "run.jsonl"
    with pkg.Solver(P.shape, P.lo, P.hi, P.V, syn.gaussian_block(0, P.n, P.p), P.p,
                    prec="fp32") as s:
        s.run_logged(6, str(log), residual_every=3)
    rows = [json.loads(x) for x in log.read_text().splitlines()]
    assert [r["step"] for r in rows] == [1, 2, 3, 4, 5, 6]
    assert all(b["energy"] <= a["energy"] for a, b in zip(rows, rows[1:]))
    assert "residual" in rows[2] and "residual" in rows[5] and "residual" not in rows[0]
