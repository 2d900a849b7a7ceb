import os
import sys

# Small dense products in the oracle are dominated by BLAS thread start-up;
# one thread keeps the CPU suite fast and deterministic.
os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
os.environ.setdefault("OMP_NUM_THREADS", "1")
os.environ.setdefault("MKL_NUM_THREADS", "1")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a GB300 and the compiled CUDA library")
    config.addinivalue_line("markers", "slow: takes more than ~20 s on the CPU")
