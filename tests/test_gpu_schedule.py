"""Serial schedule and least-metric selection on the GPU (mbbp_decode_ex
through the C ABI) against the oracle.

The serial kernel forms every q_{v->c} and check output with the oracle's
operations in the oracle's order, so with normalized min-sum every
candidate, convergence flag, iteration count, selection and final estimate
equals the FP32 oracle's on every shot.  Sum-product differs only through
expm1f/log1pf: posteriors after 1, 2 and 5 iterations within 1e-4, decisions
by agreement.  LMS sums float LLRs in ascending variable order on both
sides, so its choice is exact too.
"""
import numpy as np
import pytest

import oracle
from paper_2605_14170_gb300.inputs import channel_llr, named_code
from test_gpu_decode import assert_exact, workload

pytestmark = pytest.mark.gpu

SEED = 20260519
SERIAL, LMS = oracle.SCHEDULE_SERIAL, oracle.DECISION_LMS


@pytest.fixture(scope="module")
def M():
    import torch  # noqa: F401
    from paper_2605_14170_gb300 import mbbp
    return mbbp


def gpu(M, B, s, llr, iters, alpha, rule=0, schedule=0, decision=0, post=False):
    import torch
    dev = torch.device("cuda:0")
    out = M.decode(B, torch.from_numpy(np.ascontiguousarray(s)).to(dev),
                   torch.from_numpy(np.ascontiguousarray(llr, np.float32)).to(dev),
                   iters, alpha, rule, want_posterior=post, schedule=schedule, decision=decision)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items() if k not in ("cand", "workspace")}
    res["iters"] = res["iters"].view(np.uint16)
    res["cand"] = M.unpack_words(out["cand"], B.n)
    return res


def ref(H, B, s, llr, iters, alpha, rule=0, schedule=0, decision=0, post=False, precision="f32"):
    return oracle.mbbp_decode(H, B.sets, s, llr, iters, alpha, rule, precision=precision, want_post=post,
                              schedule=schedule, decision=decision)


def test_layers_are_greedy_and_variable_disjoint(M):
    c = named_code("bb144")
    H = c.HZ
    B = M.mbbp_build_bases(H, 8, SEED)
    info = M.mbbp_bases_info(B)
    for t in range(B.R):
        Ht = np.vstack([H, H[B.sets[t]]]) if len(B.sets[t]) else H
        layers = M.mbbp_bases_layers(B, t)
        rows = np.concatenate(layers)
        assert sorted(rows.tolist()) == list(range(info["rows"][t]))
        for L, lay in enumerate(layers):
            assert lay.tolist() == sorted(lay.tolist())
            assert Ht[lay].sum(0).max() <= 1  # no shared variable
            for r in lay:  # first fit: r clashes with an earlier row of every earlier layer
                for Lp in range(L):
                    prev = [x for x in layers[Lp] if x < r]
                    assert (Ht[prev] @ Ht[r] > 0).any() if prev else False


@pytest.mark.parametrize("code,which,R,shots", [("bb72", "HZ", 8, 1500), ("bb144", "HX", 16, 200)])
def test_serial_nms_exact(M, code, which, R, shots):
    """alpha = 0.875, 100 iterations (the setting of the numerical results)."""
    c, H, e, s = workload(code, which, shots, 0.06, "depolarizing")
    B = M.mbbp_build_bases(H, R, SEED)
    llr = channel_llr(H.shape[1], 0.04).astype(np.float32)
    got = gpu(M, B, s, llr, 100, 0.875, schedule=SERIAL)
    assert_exact(got, ref(H, B, s, llr, 100, 0.875, schedule=SERIAL))
    # serial differs from flooding on these inputs (the schedules are not confused)
    flo = ref(H, B, s, llr, 100, 0.875)
    assert not np.array_equal(got["iters"], flo["iters"])


def test_serial_edge_cases_exact(M):
    c, H, e, s = workload("bb72", "HX", 200, 0.07, "depolarizing", first=777)
    rng = np.random.default_rng(3)
    llr = rng.uniform(-1.0, 4.0, (200, 72)).astype(np.float32)  # per-shot, some negative
    B = M.mbbp_build_bases(H, 6, 3)
    for iters in (0, 1, 7):
        got = gpu(M, B, s, llr, iters, 0.75, schedule=SERIAL, post=True)
        r = ref(H, B, s, llr, iters, 0.75, schedule=SERIAL, post=True)
        assert_exact(got, r)
        assert np.array_equal(got["posterior"], r["post"])
    # plain BP (no extra rows), the Fig. 2 matrix with every syndrome
    B1 = M.mbbp_build_bases_from_sets(H, [[]])
    assert_exact(gpu(M, B1, s, llr, 30, 0.875, schedule=SERIAL),
                 ref(H, B1, s, llr, 30, 0.875, schedule=SERIAL))
    H2 = np.array([[1, 1, 1, 0, 0, 0], [0, 1, 1, 0, 0, 1], [1, 0, 0, 1, 1, 0], [0, 0, 0, 1, 1, 1]], np.uint8)
    s2 = np.array([[(k >> i) & 1 for i in range(4)] for k in range(16)], np.uint8)
    llr2 = np.array([2.0, 1.0, 1.5, 0.5, 3.0, 2.5], np.float32)
    B2 = M.mbbp_build_bases_from_sets(H2, [[0, 2], [3, 1]])
    assert_exact(gpu(M, B2, s2, llr2, 10, 0.75, schedule=SERIAL), ref(H2, B2, s2, llr2, 10, 0.75, schedule=SERIAL))


def test_serial_irregular_and_wide(M):
    """Per-row degrees in the width-8 kernel, and the length-882 GB code
    (width 6, the generic-size rows of H^(t)) with R = 16."""
    rng = np.random.default_rng(7)
    m, n = 40, 90
    H = np.zeros((m, n), np.uint8)
    col_w = np.zeros(n, int)
    for r in range(m):
        avail = np.nonzero(col_w < 4)[0]
        cols = rng.choice(avail, min(int(rng.integers(3, 9)), len(avail)), replace=False)
        H[r, cols] = 1
        col_w[cols] += 1
    e = (rng.random((150, n)) < 0.04).astype(np.uint8)
    s = oracle.syndrome(H, e)
    B = M.mbbp_build_bases_from_sets(H, oracle.collect_subtrees(H, 5, 11))
    llr = channel_llr(n, 0.04).astype(np.float32)
    assert_exact(gpu(M, B, s, llr, 40, 0.7, schedule=SERIAL), ref(H, B, s, llr, 40, 0.7, schedule=SERIAL))
    c, H, e, s = workload("gb882", "HZ", 8, 0.04, "depolarizing")
    B = M.mbbp_build_bases(H, 16, SEED)
    llr = channel_llr(882, 2 * 0.04 / 3).astype(np.float32)
    assert_exact(gpu(M, B, s, llr, 100, 0.875, schedule=SERIAL), ref(H, B, s, llr, 100, 0.875, schedule=SERIAL))


def test_serial_sum_product(M):
    c, H, e, s = workload("bb144", "HZ", 300, 0.05, "depolarizing", first=9000)
    B = M.mbbp_build_bases(H, 8, 2)
    llr = channel_llr(144, 2 * 0.05 / 3).astype(np.float32)
    # One serial iteration chains as many check updates as there are layers
    # (flooding chains one), so the last-bit differences of expm1f/log1pf
    # grow faster per iteration: 1e-4 after 1 and 2 iterations, 1e-3 after 5.
    for it, tol in ((1, 1e-4), (2, 1e-4), (5, 1e-3)):
        got = gpu(M, B, s, llr, it, 1.0, 1, schedule=SERIAL, post=True)
        r = ref(H, B, s, llr, it, 1.0, 1, schedule=SERIAL, post=True)
        same = got["iters"] == r["iters"]
        assert same.mean() > 0.99
        err = np.abs(got["posterior"][same] - r["post"][same]) / np.maximum(np.abs(r["post"][same]), 1.0)
        assert err.max() <= tol, (it, err.max())
    got = gpu(M, B, s, llr, 60, 1.0, 1, schedule=SERIAL)
    r = ref(H, B, s, llr, 60, 1.0, 1, schedule=SERIAL)
    assert (got["e_hat"] == r["ehat"]).all(1).mean() >= 0.99
    assert (got["conv"] == r["conv"]).mean() >= 0.99


def test_serial_fp64_decisions(M):
    """Against the FP64 oracle: hard decisions on >= 99.9% of shots."""
    c, H, e, s = workload("bb72", "HZ", 2000, 0.05, "bsc", first=3000)
    B = M.mbbp_build_bases(H, 4, SEED)
    llr = channel_llr(72, 0.05)
    got = gpu(M, B, s, llr, 100, 0.875, schedule=SERIAL)
    r = ref(H, B, s, llr, 100, 0.875, schedule=SERIAL, precision="f64")
    assert (got["e_hat"] == r["ehat"]).all(1).mean() >= 0.999


@pytest.mark.parametrize("schedule", [0, SERIAL])
def test_lms_exact(M, schedule):
    """LMS with per-shot LLRs (metrics differ per shot; small-integer LLRs
    make ties frequent, so the lowest-index rule is exercised)."""
    c, H, e, s = workload("bb72", "HZ", 1000, 0.08, "bsc", first=40000)
    B = M.mbbp_build_bases(H, 12, SEED)
    rng = np.random.default_rng(5)
    llr = rng.integers(1, 5, (1000, 72)).astype(np.float32)
    got = gpu(M, B, s, llr, 40, 0.75, schedule=schedule, decision=LMS)
    r = ref(H, B, s, llr, 40, 0.75, schedule=schedule, decision=LMS)
    assert_exact(got, r)
    fws = ref(H, B, s, llr, 40, 0.75, schedule=schedule)
    assert not np.array_equal(r["selected"], fws["selected"])  # the rules differ here
    # shared LLR vector (llr_stride = 0)
    llr1 = channel_llr(72, 0.08).astype(np.float32)
    assert_exact(gpu(M, B, s, llr1, 40, 0.75, schedule=schedule, decision=LMS),
                 ref(H, B, s, llr1, 40, 0.75, schedule=schedule, decision=LMS))


def test_decode_ex_defaults_and_errors(M):
    import torch
    c, H, e, s = workload("bb144", "HZ", 300, 0.05, "depolarizing")
    B = M.mbbp_build_bases(H, 8, 4)
    llr = channel_llr(144, 0.04).astype(np.float32)
    a = gpu(M, B, s, llr, 50, 0.625)
    dev = torch.device("cuda:0")
    st, lt = torch.from_numpy(s).to(dev), torch.from_numpy(llr).to(dev)
    out = {k: torch.empty(sh, dtype=dt, device=dev) for k, sh, dt in (
        ("e_hat", (300, 144), torch.uint8), ("conv", (300, 8), torch.uint8),
        ("success", (300,), torch.uint8), ("selected", (300,), torch.int16), ("iters", (300, 8), torch.int16))}
    ws = torch.empty(M.mbbp_decode_workspace_size(B, 300), dtype=torch.uint8, device=dev)
    M.mbbp_decode_ex(B, st, lt, 50, M.Options(0, 0.625, 0, 0), out["e_hat"], out["conv"], out["success"], ws,
                     iters_run=out["iters"], selected=out["selected"])
    torch.cuda.synchronize()
    assert np.array_equal(out["e_hat"].cpu().numpy(), a["e_hat"])
    assert np.array_equal(out["selected"].cpu().numpy(), a["selected"])
    for bad in (M.Options(0, 0.625, 2, 0), M.Options(0, 0.625, 0, 5), M.Options(3, 0.625, 1, 0),
                M.Options(0, 0.0, 1, 1)):
        with pytest.raises(M.MBBPError):
            M.mbbp_decode_ex(B, st, lt, 50, bad, out["e_hat"], out["conv"], out["success"], ws)


@pytest.mark.parametrize("rule", [0, 1])
def test_width12_code_both_schedules(M, rule):
    """Rows of weight up to 11: the width-12 kernels (generic flooding kernel
    and the one-item-per-warp serial kernel), min-sum exact, sum-product by
    agreement."""
    rng = np.random.default_rng(12)
    m, n = 30, 120
    H = np.zeros((m, n), np.uint8)
    for r in range(m):
        H[r, rng.choice(n, int(rng.integers(5, 12)), replace=False)] = 1
    e = (rng.random((120, n)) < 0.03).astype(np.uint8)
    s = oracle.syndrome(H, e)
    B = M.mbbp_build_bases_from_sets(H, oracle.collect_subtrees(H, 4, 5))
    llr = channel_llr(n, 0.03).astype(np.float32)
    for schedule in (0, SERIAL):
        got = gpu(M, B, s, llr, 30, 0.8, rule, schedule=schedule)
        r = ref(H, B, s, llr, 30, 0.8, rule, schedule=schedule)
        if rule == 0:
            assert_exact(got, r)
        else:
            assert (got["e_hat"] == r["ehat"]).all(1).mean() >= 0.97
