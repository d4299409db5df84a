import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden(name):
    import json

    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


@pytest.fixture(scope="session")
def built_lib():
    from paper_2210_16435_gb300 import buildlib as _b

    return _b.build()


def to_dev(a, dtype, device="cuda"):
    import numpy as np
    import torch

    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=device)


def graph_tensors(g, value_dtype=None, device="cuda"):
    import torch

    value_dtype = value_dtype or torch.float64
    return (to_dev(g.row_ptr, torch.int32, device), to_dev(g.col_idx, torch.int32, device),
            to_dev(g.values, value_dtype, device), to_dev(g.groups, torch.int32, device))
