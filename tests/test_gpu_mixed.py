"""Persistent mixed-batch decoder (mbbp_decode_mixed): one launch over the
shots of several codes gives exactly what one mbbp_decode per code gives,
also after autotuning and when replayed from a captured CUDA graph."""
import numpy as np
import pytest

import oracle
from paper_2605_14170_gb300.inputs import channel_llr, named_code

pytestmark = pytest.mark.gpu

FIG2 = np.array([[1, 1, 1, 0, 0, 0], [0, 1, 1, 0, 0, 1], [1, 0, 0, 1, 1, 0], [0, 0, 0, 1, 1, 1]], np.uint8)


def _codes():
    """[[72]] R=8, [[144]] R=16, [[288]] R=32 (the mixed workload), plus the
    Fig. 2 matrix (irregular rows) with its two subtrees."""
    from paper_2605_14170_gb300 import mbbp
    out = []
    for name, R, batch in (("bb72", 8, 700), ("bb144", 16, 500), ("bb288", 32, 300)):
        H = named_code(name).HZ
        out.append((H, mbbp.mbbp_build_bases(H, R, 5), batch, 0.05))
    out.append((FIG2, mbbp.mbbp_build_bases_from_sets(FIG2, [[0, 2], [3, 1]]), 16, 0.1))
    return out


def _inputs(codes, seed):
    import torch
    synd, llrs = [], []
    for H, B, batch, p in codes:
        ex, _ = oracle.sample(seed, 0, batch, H.shape[1], p, "depolarizing")
        synd.append(torch.from_numpy(oracle.syndrome(H, ex)).cuda())
        llrs.append(torch.from_numpy(channel_llr(H.shape[1], 2 * p / 3).astype(np.float32)).cuda())
    return synd, llrs


def _per_code(codes, synd, llrs, iters):
    from paper_2605_14170_gb300 import mbbp
    return [mbbp.decode(B, s, l, iters, 0.625) for (H, B, _, _), s, l in zip(codes, synd, llrs)]


def _same(ios, refs):
    import torch
    for x, r in zip(ios, refs):
        for key in ("e_hat", "conv", "iters", "success", "selected"):
            assert torch.equal(x[key], r[key]), key


def test_mixed_equals_per_code_decode():
    import torch
    from paper_2605_14170_gb300 import mbbp
    codes = _codes()
    P = mbbp.mbbp_plan_create([B for _, B, _, _ in codes])
    info = mbbp.mbbp_plan_info(P)
    assert info["kind"] == [0, 0, 1, 1]  # small path for the regular small codes
    assert info["order"][0] == 2  # the heaviest code ([[288]], R = 32) first
    synd, llrs = _inputs(codes, 11)
    ios, ws = mbbp.mixed_buffers(P, synd, llrs)
    mbbp.mbbp_decode_mixed(P, ios, 100, 0.625, mbbp.RULE_NMS, ws)
    torch.cuda.synchronize()
    _same(ios, _per_code(codes, synd, llrs, 100))
    # the [[288]] code has no other parity test: compare a sample with the oracle
    H, B, _, _ = codes[2]
    s = synd[2][:40].cpu().numpy()
    ref = oracle.mbbp_decode(H, B.sets, s, llrs[2].cpu().numpy(), 100, 0.625, precision="f32")
    assert np.array_equal(ios[2]["e_hat"][:40].cpu().numpy(), ref["ehat"])
    assert np.array_equal(ios[2]["iters"][:40].cpu().numpy().view(np.uint16), ref["iters"])


def test_autotune_keeps_results_and_graph_replay():
    import torch
    from paper_2605_14170_gb300 import mbbp
    codes = _codes()[:3]
    P = mbbp.mbbp_plan_create([B for _, B, _, _ in codes])
    synd, llrs = _inputs(codes, 12)
    ios, ws = mbbp.mixed_buffers(P, synd, llrs)
    best = mbbp.mbbp_plan_autotune(P, ios, 100, 0.625, mbbp.RULE_NMS, ws)
    assert best > 0
    info = mbbp.mbbp_plan_info(P)
    assert info["warps"] in (4, 6, 7, 8) and all(c in (1, 2, 4, 8, 16) for c in info["chunk"])
    mbbp.mbbp_decode_mixed(P, ios, 100, 0.625, mbbp.RULE_NMS, ws)
    torch.cuda.synchronize()
    _same(ios, _per_code(codes, synd, llrs, 100))
    # capture one decode into a CUDA graph, then replay it on new syndromes
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        mbbp.mbbp_decode_mixed(P, ios, 100, 0.625, mbbp.RULE_NMS, ws, stream=s)
        s.synchronize()
        with torch.cuda.graph(graph, stream=s):
            mbbp.mbbp_decode_mixed(P, ios, 100, 0.625, mbbp.RULE_NMS, ws, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    synd2, _ = _inputs(codes, 13)
    for x, s2 in zip(ios, synd2):
        x["syndromes"].copy_(s2)
    graph.replay()
    torch.cuda.synchronize()
    _same(ios, _per_code(codes, synd2, llrs, 100))


def test_mixed_with_an_empty_code():
    import torch
    from paper_2605_14170_gb300 import mbbp
    codes = _codes()[:2]
    P = mbbp.mbbp_plan_create([B for _, B, _, _ in codes])
    synd, llrs = _inputs(codes, 14)
    synd[0] = synd[0][:0]
    ios, ws = mbbp.mixed_buffers(P, synd, llrs)
    mbbp.mbbp_decode_mixed(P, ios, 50, 0.625, mbbp.RULE_NMS, ws)
    torch.cuda.synchronize()
    ref = mbbp.decode(codes[1][1], synd[1], llrs[1], 50, 0.625)
    assert torch.equal(ios[1]["e_hat"], ref["e_hat"]) and torch.equal(ios[1]["iters"], ref["iters"])


def test_mixed_launch_groups_per_shape():
    """A plan whose small codes have different register-resident shapes
    ([[72]]; a random column-weight-3 code with 97..128 rows of H^(t)) and a
    generic-path code: one launch per shape plus the generic launch, outputs
    identical to one mbbp_decode per code and, for the four-row-step code, to
    the FP32 oracle."""
    import torch
    from paper_2605_14170_gb300 import mbbp
    rng = np.random.default_rng(21)
    n, m = 160, 80
    sock = rng.permutation(np.repeat(np.arange(n), 3)).reshape(m, 6)
    for _ in range(100000):
        bad = [r for r in range(m) if len(set(sock[r])) < 6]
        if not bad:
            break
        i, r2, j = rng.integers(6), rng.integers(m), rng.integers(6)
        sock[bad[0], i], sock[r2, j] = sock[r2, j], sock[bad[0], i]
    H4 = np.zeros((m, n), np.uint8)
    for r in range(m):
        H4[r, sock[r]] = 1
    sets4 = oracle.collect_subtrees(H4, 6, 9)
    assert 96 < m + max(len(t) for t in sets4) <= 128
    codes = [c for c in _codes() if c[0].shape[1] in (72, 288)]
    codes.append((H4, mbbp.mbbp_build_bases_from_sets(H4, sets4), 400, 0.05))
    P = mbbp.mbbp_plan_create([B for _, B, _, _ in codes])
    assert mbbp.mbbp_plan_info(P)["kind"] == [0, 1, 0]
    synd, llrs = _inputs(codes, 17)
    ios, ws = mbbp.mixed_buffers(P, synd, llrs)
    mbbp.mbbp_decode_mixed(P, ios, 60, 0.625, mbbp.RULE_NMS, ws)
    torch.cuda.synchronize()
    _same(ios, _per_code(codes, synd, llrs, 60))
    s = synd[2].cpu().numpy()
    ref = oracle.mbbp_decode(H4, sets4, s, llrs[2].cpu().numpy(), 60, 0.625, precision="f32")
    assert np.array_equal(ios[2]["e_hat"].cpu().numpy(), ref["ehat"])
    assert np.array_equal(ios[2]["iters"].cpu().numpy().view(np.uint16), ref["iters"])
