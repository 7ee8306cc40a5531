import importlib.util
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)


def _load_file(name, path):
    spec = importlib.util.spec_from_file_location(name, path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


# Build the in-tree libraries before test modules import them (nvcc
# cross-compiles for sm_103a without a GPU; g++ builds the oracle).
_load_file("_qld_build", os.path.join(ROOT, "paper_1511_03390_b300", "build.py")).build()
_load_file("_orc_build", os.path.join(ROOT, "oracle", "build.py")).build()
import qldscene  # noqa: E402

qldscene.build()


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a)")
    config.addinivalue_line("markers", "large: full-size workload (tens of GB of device memory)")
