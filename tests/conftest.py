import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running case")


@pytest.fixture(scope="session")
def model():
    import workload

    return workload.microcircuit_model()


def pytest_collection_finish(session):
    """When GPU tests that compare against long oracle runs are selected, start those runs
    in background threads now, before any GPU work, so that they overlap the session."""
    gpu_modules = {item.module.__name__.split(".")[-1] for item in session.items
                   if item.get_closest_marker("gpu") is not None}
    if not gpu_modules:
        return
    try:
        import torch

        if not torch.cuda.is_available():
            return
    except ImportError:
        return
    tests_dir = os.path.dirname(os.path.abspath(__file__))
    if tests_dir not in sys.path:
        sys.path.insert(0, tests_dir)
    import oracle_runs

    oracle_runs.start_for_modules(gpu_modules)
