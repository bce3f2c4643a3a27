"""Parity of the persistent launches where their warps pull many work items.

Every BP kernel is a persistent grid: its warps pull work items (a chunk of
shots of one representation, or one (shot, representation) pair) from a
counter until none is left, reusing their shared memory and registers from
one item to the next.  Here every launch has at least twice as many work
items as the GPU can hold warps resident (SMs x the most warps an SM
holds, whatever the kernel's occupancy), so most warps run several items,
as in the 1e6-shot benchmark launches.  Every output is compared bit for bit
with the FP32 oracle (flooding BP of Section II-B with FWS of Section
III-B, and the serial schedule), at the sizes of the batched [[144,12,12]]
workload.
"""
import numpy as np
import pytest

import oracle
from conftest import oracle_decode_parallel
from paper_2605_14170_gb300.inputs import channel_llr, named_code

pytestmark = pytest.mark.gpu

SEED = 20260520


@pytest.fixture(scope="module")
def M():
    import torch  # noqa: F401
    from paper_2605_14170_gb300 import mbbp
    return mbbp


def resident_warp_bound():
    """Upper bound on the warps a launch can hold resident at once."""
    import torch
    props = torch.cuda.get_device_properties(0)
    per_sm = getattr(props, "max_threads_per_multi_processor", 2048) // 32
    return props.multi_processor_count * per_sm


def _decode(M, B, s, llr, iters, alpha, **kw):
    import torch
    out = M.decode(B, torch.from_numpy(np.ascontiguousarray(s)).cuda(),
                   torch.from_numpy(np.ascontiguousarray(llr, np.float32)).cuda(), iters, alpha, **kw)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items() if k not in ("cand", "workspace")}
    res["iters"] = res["iters"].view(np.uint16)
    res["cand"] = M.unpack_words(out["cand"], B.n)
    return res


def _assert_exact(got, ref, what):
    for key, rkey in (("conv", "conv"), ("iters", "iters"), ("cand", "cand"), ("selected", "selected"),
                      ("success", "success"), ("e_hat", "ehat")):
        assert np.array_equal(got[key], ref[rkey]), (what, key)


@pytest.mark.parametrize("which", ["HZ", "HX"])
@pytest.mark.parametrize("p", [0.02, 0.08])
def test_small_kernel_many_items_per_warp(M, which, p):
    """The register-resident kernel ([[144,12,12]], R = 16, 100 iterations,
    chunks of 8 shots per item) on 10,000 depolarizing shots: 20,000 items."""
    shots, R = 10000, 16
    c = named_code("bb144")
    H = getattr(c, which)
    ex, ez = oracle.sample(SEED, 0, shots, 144, p, "depolarizing")
    s = oracle.syndrome(H, ex if which == "HZ" else ez)
    B = M.mbbp_build_bases(H, R, SEED)
    items = -(-shots // 8) * R
    bound = resident_warp_bound()
    assert items >= 2 * bound, (items, bound)
    print(f"\n[[144]] {which} p={p}: {items} items, at most {bound} resident warps ({items / bound:.2f} per warp)")
    llr = channel_llr(144, 2 * p / 3).astype(np.float32)
    got = _decode(M, B, s, llr, 100, 0.625)
    ref = oracle_decode_parallel(H, B.sets, s, llr, 100, 0.625)
    _assert_exact(got, ref, f"bb144 {which} p={p}")


def test_generic_kernel_many_items_per_warp(M):
    """The generic flooding kernel ([[288,12,18]], R = 32, one warp per
    (shot, representation)) on 800 shots: 25,600 items."""
    shots, R, p = 800, 32, 0.06
    c = named_code("bb288")
    H = c.HZ
    ex, _ = oracle.sample(SEED + 1, 0, shots, 288, p, "depolarizing")
    s = oracle.syndrome(H, ex)
    B = M.mbbp_build_bases(H, R, SEED)
    items, bound = shots * R, resident_warp_bound()
    assert items >= 2 * bound, (items, bound)
    print(f"\n[[288]] R=32: {items} items, at most {bound} resident warps ({items / bound:.2f} per warp)")
    llr = channel_llr(288, 2 * p / 3).astype(np.float32)
    got = _decode(M, B, s, llr, 100, 0.625)
    ref = oracle_decode_parallel(H, B.sets, s, llr, 100, 0.625)
    _assert_exact(got, ref, "bb288")


def test_serial_kernel_many_refills_per_warp(M):
    """The serial-schedule chunk kernel ([[144,12,12]], R = 16, alpha =
    0.875, least-metric selection) on 5,000 shots: its warps hold at most 4
    shots at a time and refill their slots from per-representation counters,
    so 80,000 (shot, representation) pairs are at least twice what the
    resident warps' slots can hold."""
    shots, R, p = 5000, 16, 0.06
    H = named_code("bb144").HZ
    ex, _ = oracle.sample(SEED + 2, 0, shots, 144, p, "depolarizing")
    s = oracle.syndrome(H, ex)
    B = M.mbbp_build_bases(H, R, SEED)
    pairs, bound = shots * R, resident_warp_bound()
    assert pairs >= 2 * 4 * bound, (pairs, bound)
    llr = channel_llr(144, 2 * p / 3).astype(np.float32)
    got = _decode(M, B, s, llr, 100, 0.875, schedule=M.SCHEDULE_SERIAL, decision=M.DECISION_LMS)
    ref = oracle_decode_parallel(H, B.sets, s, llr, 100, 0.875, schedule=oracle.SCHEDULE_SERIAL,
                                 decision=oracle.DECISION_LMS)
    _assert_exact(got, ref, "serial bb144")


def test_mixed_launches_many_items_per_warp(M):
    """The persistent mixed-batch launches ([[72]] R = 8 and [[144]] R = 16
    on the small-code body, one launch per shape; [[288]] R = 32 on the
    generic body): every launch group gets at least twice the resident-warp
    bound in items, and each code's outputs equal the FP32 oracle's."""
    import torch
    bound = resident_warp_bound()
    specs = [("bb72", 8), ("bb144", 16), ("bb288", 32)]
    Bs = [M.mbbp_build_bases(named_code(name).HZ, R, SEED + 3) for name, R in specs]
    P = M.mbbp_plan_create(Bs)
    info = M.mbbp_plan_info(P)
    assert info["kind"] == [0, 0, 1]
    p = 0.05
    synd, llrs, refs, Hs = [], [], [], []
    for (name, R), B, chunk, kind in zip(specs, Bs, info["chunk"], info["kind"]):
        per_item = chunk if kind == 0 else 1
        shots = -(-2 * bound * per_item // R) + 64  # items = ceil(shots / per_item) * R >= 2 * bound
        H = named_code(name).HZ
        ex, _ = oracle.sample(SEED + 4, 0, shots, H.shape[1], p, "depolarizing")
        s = oracle.syndrome(H, ex)
        llr = channel_llr(H.shape[1], 2 * p / 3).astype(np.float32)
        assert -(-shots // per_item) * R >= 2 * bound
        synd.append(torch.from_numpy(s).cuda())
        llrs.append(torch.from_numpy(llr).cuda())
        refs.append(oracle_decode_parallel(H, B.sets, s, llr, 100, 0.625))
        Hs.append(H)
    ios, ws = M.mixed_buffers(P, synd, llrs)
    M.mbbp_decode_mixed(P, ios, 100, 0.625, M.RULE_NMS, ws)
    torch.cuda.synchronize()
    for (name, _), x, ref in zip(specs, ios, refs):
        got = {k: x[k].cpu().numpy() for k in ("e_hat", "conv", "success", "selected")}
        got["iters"] = x["iters"].cpu().numpy().view(np.uint16)
        for key, rkey in (("conv", "conv"), ("iters", "iters"), ("selected", "selected"),
                          ("success", "success"), ("e_hat", "ehat")):
            assert np.array_equal(got[key], ref[rkey]), (name, key)


def test_generic_kernel_length_882_many_items_per_group(M):
    """The generic flooding kernel on the length-882 GB code with R = 64
    (its largest workload: rows of H^(t) up to 617, where two warps share
    each item's message area) on 320 shots: 20,480 (shot, representation)
    items, at least twice the resident-warp bound, every output equal to the
    FP32 oracle's."""
    shots, R, p = 320, 64, 0.04
    H = named_code("gb882").HZ
    ex, _ = oracle.sample(SEED + 5, 0, shots, 882, p, "depolarizing")
    s = oracle.syndrome(H, ex)
    B = M.mbbp_build_bases(H, R, SEED)
    items, bound = shots * R, resident_warp_bound()
    assert items >= 2 * bound, (items, bound)
    llr = channel_llr(882, 2 * p / 3).astype(np.float32)
    got = _decode(M, B, s, llr, 100, 0.625)
    ref = oracle_decode_parallel(H, B.sets, s, llr, 100, 0.625)
    _assert_exact(got, ref, "gb882")
