import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")


def read_golden(name):
    rows = []
    with open(os.path.join(ROOT, "tests", "golden", name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append([float(v) for v in line.split()])
    return rows


@pytest.fixture(scope="session")
def rb():
    """The built library on cuda:0 (GPU tests fail, not skip, without a GPU or the library)."""
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2508_06710_gb300 import build

    build.build()
    import paper_2508_06710_gb300 as pkg

    pkg.lib()
    torch.cuda.set_device(0)
    return pkg


def to_dev(a, dtype=None):
    import numpy as np
    import torch

    a = np.ascontiguousarray(a)
    t = torch.as_tensor(a)
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def componentwise_ok(Y, Yref, bound, tol):
    """max over entries of |Y - Yref| / bound <= tol, with bound = (|A||X|) (scaled by |c|)."""
    import numpy as np

    err = np.abs(np.asarray(Y, dtype=np.float64) - Yref)
    lim = tol * bound + 1e-300
    bad = err > lim
    return (not bad.any()), float((err / np.maximum(bound, 1e-300)).max())
