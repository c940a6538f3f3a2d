"""Shared test fixtures.  Tests marked `gpu` need a CUDA device and the
built library; everything else runs on the CPU."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


# GPU test modules of the newest components run after the rest of the suite, so
# that under -x a failure there cannot hide the results of the established tests;
# modules named test_zz_* run after those, last of all.
RUN_LAST = ("test_gpu_electrostatic.py", "test_gpu_octree.py")


def _order(item):
    name = os.path.basename(str(item.fspath))
    if name.startswith("test_zz_"):
        return 2
    return 1 if name in RUN_LAST else 0


def pytest_collection_modifyitems(config, items):
    items.sort(key=_order)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the built libefe library")
    config.addinivalue_line("markers", "slow: oracle runs that take tens of seconds")


@pytest.fixture(scope="session")
def h2_system():
    import efe_workloads as W
    from oracle import operators
    return operators.System(W.h2())


@pytest.fixture(scope="session")
def h2_ground(h2_system):
    """Self-consistent ground state of the H2 workload from the oracle."""
    import numpy as np
    from oracle import tdks
    psi, eps = tdks.ground_state(h2_system, 1, np.array([2.0]), mix=0.5, tol=1e-11)
    return psi, eps
