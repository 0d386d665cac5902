import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def box10k():
    from scenegen import make_scene
    return make_scene("box10k")


@pytest.fixture(scope="session")
def small_floor():
    """A 60k-leaf multi-room floor: several tiles of work per view but fast on CPU."""
    from scenegen import make_floor_scene
    return make_floor_scene(60_000, seed=11, size=(8.0, 6.0, 3.0), n_clusters=4,
                            cluster_size=2000)
