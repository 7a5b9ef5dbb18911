import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: large parity case (minutes of oracle time)")


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle
    return oracle.lib()


@pytest.fixture(autouse=True)
def several_outcomes_share():
    """After each test that compared GPU pixels with the oracle's correct outcomes: the share
    of checked pixels with several correct outcomes, over all the frames the test checked,
    stays under gvtest.MULTI_CAP."""
    yield
    gt = sys.modules.get("gvtest")
    if gt is not None:
        gt.check_multi_share()
