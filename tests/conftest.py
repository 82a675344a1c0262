import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def oracle_all():
    """Oracle results of whole generated workloads on every host core, cached by workload
    name, size, seed and parameters, so that several full-size parity tests of one batch
    share one oracle run (only for batches made by the synth generators)."""
    import oracle
    cache = {}

    def get(batch):
        key = (batch.name, batch.n_pairs, batch.X, batch.delta, batch.zdrop, repr(sorted(batch.meta.items())))
        if key not in cache:
            cache[key] = oracle.run_batch(batch, threads=max(1, os.cpu_count() or 1))
        return cache[key]

    return get
