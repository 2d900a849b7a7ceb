"""FP64 CPU oracle for the orthogonality-preserving eigensolver (arXiv 2511.06788).

TEST INFRASTRUCTURE ONLY.  This package is imported by ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py``; the CUDA library and its Python binding never import,
link or execute anything here, and nothing here imports the library.
"""
from .scheme import *  # noqa: F401,F403
