import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
# the tests time launch variants on small meshes: keep their choices out of the user's
# persistent autotune file (the persistence test points a subprocess at a file of its own)
os.environ["MF_AUTOTUNE_CACHE"] = "off"
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libmf.so")


@pytest.fixture(scope="session")
def oracle():
    import oracle as orc

    orc.build()
    return orc
