import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")
    config.addinivalue_line("markers", "oracle_job(name): compares with an oracle run that "
                            "starts in a background worker when the session starts")


def pytest_collection_finish(session):
    """Start the oracle runs the selected tests wait for, so that they compute
    while the other tests run (only where a GPU can run those tests)."""
    names = []
    for item in session.items:
        for m in item.iter_markers("oracle_job"):
            names.extend(m.args)
    if not names:
        return
    try:
        import torch
        if not torch.cuda.is_available():
            return
    except ImportError:
        return
    import _oracle_jobs
    _oracle_jobs.start(sorted(set(names)))


def pytest_sessionfinish(session, exitstatus):
    mod = sys.modules.get("_oracle_jobs")
    if mod is not None:
        mod.shutdown()


@pytest.fixture(scope="session")
def gpu_lib():
    """The native library, loaded once; skips when no GPU is visible."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2504_21784_gb300 as sm
    sm.load()
    return sm
