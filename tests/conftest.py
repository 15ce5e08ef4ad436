import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long CPU test")


@pytest.fixture(scope="session")
def cfg1():
    from paper_1709_04794_gb300 import synth
    return synth.make_problem("single_fp64_2k")


@pytest.fixture(scope="session")
def tiny():
    """A tiny problem for dense checks (N=120, D=60)."""
    from paper_1709_04794_gb300 import synth
    return synth.custom_problem(120, 60, 8, seed=11, values="counts", n_labelled=40, k=4,
                                shifts=(1e-2, 1e1, 4))
