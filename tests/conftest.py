import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(autouse=True)
def _checked_build_word(request):
    """Under DDSG_VARIANT=checked every GPU test must leave the library's
    table-index check word clean (no bounds test failed in any kernel)."""
    yield
    if os.environ.get("DDSG_VARIANT") != "checked" or request.node.get_closest_marker("gpu") is None:
        return
    import torch
    if not torch.cuda.is_available():
        return
    import paper_2202_06555_gb300 as G
    torch.cuda.synchronize()
    assert G.load().ddsg_checked_build() == 1
    failed = G.take_check_word()
    assert not failed, f"checked build: table index tests failed at {failed}"
