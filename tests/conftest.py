import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)


def read_golden(name):
    """Parse a tests/golden/*.txt file: '# ...' comments, then sections made of
    a one-word header line followed by rows of integers."""
    path = os.path.join(ROOT, "tests", "golden", name)
    sections, cur = {}, None
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            toks = line.split()
            if len(toks) == 1 and not toks[0].lstrip("-").isdigit() and not toks[0].startswith("0x"):
                cur = toks[0]
                sections[cur] = []
            else:
                sections.setdefault(cur, []).append([int(t, 0) for t in toks])
    return sections
