import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libvmat")


@pytest.fixture(scope="session")
def tiny_case():
    import synth
    return synth.make_case("tiny", seed=0)


@pytest.fixture(scope="session")
def ragged_case():
    import synth
    return synth.make_case("ragged", seed=1)


@pytest.fixture(scope="session")
def cfg1_case():
    import synth
    return synth.make_case("cfg1", seed=0)


def dense_from_coo(V, J, vox, blt, val):
    """Dense float64 D built entry by entry (brute force for tiny grids)."""
    D = np.zeros((V, J), np.float64)
    for i, j, v in zip(vox.tolist(), blt.tolist(), val.tolist()):
        D[i, j] += v
    return D
