import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running oracle case")
    config.addinivalue_line("markers", "resident: runs batches of small volumes whole in one "
                                       "launch (the library's default)")


@pytest.fixture(autouse=True)
def _batch_form(request):
    """GPU tests run the stencil kernels on every volume size, so that small
    and odd shapes keep testing them; tests marked `resident` take the
    library's default instead, where batches of volumes that fit a CTA's
    shared memory run whole in one launch."""
    if request.node.get_closest_marker("gpu") is None:
        yield
        return
    from paper_2002_01981_gb300 import build, native
    if not os.path.exists(build.LIB_PATH):
        yield
        return
    native.load().ifcm_resident_enable(1 if request.node.get_closest_marker("resident") else 0)
    yield
    native.load().ifcm_resident_enable(1)


def read_golden(name):
    """key = value lines of a golden fixture (comments start with '#')."""
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            if "=" in line:
                k, v = line.split("=", 1)
                out[k.strip()] = v.split()
            else:
                out.setdefault("_rows", []).append(line.split())
    return out
