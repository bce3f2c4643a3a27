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


def oracle_decode_parallel(H, sets, synd, llr, iters, alpha, rule=0, precision="f32", chunks=None, **kw):
    """oracle.mbbp_decode over a large batch, split into shot ranges decoded
    by host threads (the oracle's C code runs without the GIL) and
    concatenated in shot order; identical to one call on the whole batch."""
    import concurrent.futures as cf

    import numpy as np

    import oracle
    synd = np.ascontiguousarray(synd)
    batch = synd.shape[0]
    per_shot_llr = np.ndim(llr) == 2
    k = chunks or min(64, max(1, (os.cpu_count() or 1) * 2))
    edges = np.linspace(0, batch, k + 1).astype(int)
    parts = [(a, b) for a, b in zip(edges[:-1], edges[1:]) if b > a]

    def run(ab):
        a, b = ab
        return oracle.mbbp_decode(H, sets, synd[a:b], llr[a:b] if per_shot_llr else llr, iters, alpha, rule,
                                  precision=precision, **kw)

    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        outs = list(ex.map(run, parts))
    return {key: np.concatenate([o[key] for o in outs]) for key in outs[0]}
