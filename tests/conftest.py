import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def oracle_problem(scene):
    """Oracle view (float64) of a scene, built from exactly the arrays the GPU gets."""
    from oracle.vfpi import make_problem
    return make_problem(scene.row_ptr, scene.col_idx, scene.vals, scene.b, scene.node_i,
                        scene.node_j, scene.R, scene.mu, scene.phi)


@pytest.fixture
def rng():
    return np.random.default_rng(1234)
