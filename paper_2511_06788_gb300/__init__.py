"""GB300 (sm_103a) implementation of the orthogonality-preserving eigensolver
of arXiv 2511.06788: a C-ABI CUDA library (``libopevo.so``, API in
``include/opevo.h``, the learned warm start in ``include/opnet.h``) and this thin
ctypes binding.

``import paper_2511_06788_gb300`` works without the compiled library; the first
call into it raises ImportError when ``libopevo.so`` has not been built.
"""
from .binding import (OP_EIG_PAPER, OP_EIG_RITZ, OP_FP32, OP_FP64, OP_STOP_ERR_E,  # noqa: F401
                      OP_STOP_RESIDUAL, OP_STOP_STEPS, OpError, Solver, Batch, Net, apply_H, cg_solve,
                      check, core, gram, last_error, lib, make_problem, selftest_bounded_waits,
                      update)
