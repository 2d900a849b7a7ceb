"""Failure detection on the device, tested without a fault: every wait inside the
library's kernels is bounded.  The self-test entry point makes one wait of each kind
run out on an mbarrier that nothing ever completes (a flag no one sets); both must
give up, report it, and leave the GPU context usable."""
import time

import numpy as np
import pytest

import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2511_06788_gb300 as pkg  # noqa: E402


def test_bounded_waits_give_up_report_and_leave_the_context_usable():
    t0 = time.perf_counter()
    clock_wait, iter_wait = pkg.selftest_bounded_waits()
    wall = time.perf_counter() - t0
    print(f"clock-bounded wait {clock_wait:.3f} s, iteration-bounded wait {iter_wait:.3f} s, "
          f"call {wall:.3f} s")
    assert 0.19 <= clock_wait <= 2.0          # the 0.2 s limit of the probe
    assert 0.5 <= iter_wait <= 30.0           # 2^24 polls with a 64 ns sleep each
    # the context is intact: a solve afterwards works and is correct
    P = syn.laplace_2d(16, 4)
    with pkg.Solver(P.shape, P.lo, P.hi, P.V, syn.gaussian_block(0, P.n, P.p), P.p) as s:
        st = s.solve(1e-8, 5000)
        assert st["converged"]
        U = s.get_U()
    assert np.linalg.norm(U.T @ U - np.eye(P.p)) < 1e-12
