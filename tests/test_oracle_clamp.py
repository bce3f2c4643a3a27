"""The message clamp (q clamped to +-LMAX, a reading: the paper states no
clamp) and how often it acts.  Pinned on a closed form: a variable whose LLR
alone exceeds LMAX sends a clamped message on every iteration, a small one
never; then the clamp rate of the oracle on the [[144]] workload at the
highest noise level is measured (a diagnostic, reported, not a parity
value)."""
import numpy as np
import pytest

import oracle
from paper_2605_14170_gb300.inputs import channel_llr, named_code


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("schedule", [0, 1])
def test_clamp_counts_closed_form(precision, schedule):
    # one check on two variables; mu_0 = 2 LMAX reaches the check alone
    Ht = np.array([[1, 1]], np.uint8)
    mu = np.array([2.0e4, 1.0])
    for iters in (1, 3):
        oracle.clamp_reset()
        oracle.bp(Ht, np.array([0], np.uint8), mu, iters, 0.75, early_stop=False,
                  precision=precision, schedule=schedule)
        assert oracle.clamp_stats() == (2 * iters, iters)
    oracle.clamp_reset()
    oracle.bp(Ht, np.array([1], np.uint8), np.array([3.0, 1.0]), 4, 0.75, early_stop=False,
              precision=precision, schedule=schedule)
    assert oracle.clamp_stats() == (8, 0)


def test_clamp_rate_on_bb144():
    """[[144]] R = 16, depolarizing p = 0.08 (the workload's hardest point),
    flooding alpha = 0.625 and serial alpha = 0.875, FP32, 200 shots."""
    c = named_code("bb144")
    H = c.HZ
    ex, _ = oracle.sample(20260514, 0, 200, 144, 0.08, "depolarizing")
    s = oracle.syndrome(H, ex)
    sets = oracle.collect_subtrees(H, 16, 20260514)
    llr = channel_llr(144, 2 * 0.08 / 3).astype(np.float32)
    rates = {}
    for name, schedule, alpha in (("flooding", 0, 0.625), ("serial", 1, 0.875)):
        oracle.clamp_reset()
        oracle.mbbp_decode(H, sets, s, llr, 100, alpha, precision="f32", schedule=schedule)
        total, clamped = oracle.clamp_stats()
        assert total > 0 and 0 <= clamped <= total
        rates[name] = clamped / total
    print("clamp rate", rates)
