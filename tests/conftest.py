import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU check")


@pytest.fixture(scope="session")
def oracle():
    import oracle as O
    O.build()
    return O


@pytest.fixture(scope="session")
def inputs():
    from paper_2404_18034_gb300 import inputs as I
    return I


@pytest.fixture(scope="session")
def params(inputs):
    return inputs.load_params()


@pytest.fixture(scope="session")
def params7(inputs):
    return inputs.load_params(nu=7)


def rand_state(rng, m=1.7):
    x = np.concatenate([[m], rng.normal(size=3) * 3, rng.normal(size=3), rng.normal(size=4) * 0.5,
                        rng.normal(size=3) * 0.7, [0.01]])
    return x


def rand_control(rng, nu, s=4.0):
    return np.concatenate([rng.normal(size=3) * 3, rng.normal(size=nu - 4) * 0.3, [s]])
