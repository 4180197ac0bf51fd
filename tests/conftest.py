import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built CUDA library")


def find_libcurand():
    """Path of NVIDIA's cuRAND shared library, or None.  Used only as an
    independent third-party implementation to pin the oracle against."""
    import ctypes.util
    cands = []
    cuda_home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    for d in (os.path.join(cuda_home, "lib64"), os.path.join(cuda_home, "lib"),
              os.path.join(cuda_home, "targets", "sbsa-linux", "lib"),
              os.path.join(cuda_home, "targets", "x86_64-linux", "lib")):
        for name in ("libcurand.so", "libcurand.so.10"):
            cands.append(os.path.join(d, name))
    found = ctypes.util.find_library("curand")
    if found:
        cands.append(found)
    for c in cands:
        if os.path.exists(c) or not os.path.isabs(c):
            try:
                ctypes.CDLL(c)
                return c
            except OSError:
                continue
    return None


@pytest.fixture(scope="session")
def curand_path():
    p = find_libcurand()
    if p is None:
        pytest.skip("libcurand not found")
    return p


def pytest_collection_modifyitems(config, items):
    """GPU tests skip (not fail) on a machine without CUDA; on the GPU machine they run."""
    try:
        import torch
        has_cuda = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        has_cuda = False
    if has_cuda:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)
