import os
import sys

# The checker's small dense and vector operations run single-threaded: multithreaded BLAS
# partitions reductions by thread timing, which made the checker's own results (and so the
# sensitive stopping steps it is compared on) differ between runs, and oversubscribed the host
# cores next to the GPU process.  Set before NumPy loads its BLAS.
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import pytest  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the built bl library")


@pytest.fixture(scope="session")
def rng():
    import numpy as np
    return np.random.default_rng(1234)
