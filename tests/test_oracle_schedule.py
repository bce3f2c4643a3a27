"""Pins of the oracle's serial schedule (Section II-B), least-metric selector
(Section III-A) and random augmentation (Table II).

Serial schedule: checks are processed one at a time, in the layer-major
order of a greedy first-fit split of the rows into variable-disjoint layers,
and every check uses the newest messages.  Pinned by
* a two-check example worked by hand (it differs from flooding in the value
  the second check sends);
* rows that share no variable (one layer): serial equals flooding exactly;
* BP is exact on trees: serial sum-product / min-sum posteriors equal the
  brute-force bitwise-MAP log-ratios / min-cost differences;
* on a chain of checks the serial schedule reaches the exact fixed point in
  fewer iterations than flooding (it passes messages along the chain within
  one iteration);
* Algorithm 1 with the serial schedule: every converged candidate satisfies
  H e = s.

LMS: the converged candidate with the smallest sum_i mu_i e_i, ties to the
first; checked on hand-made lists and against a brute-force argmin.
"""
import numpy as np
import pytest

import oracle
from paper_2605_14170_gb300.inputs import named_code, random_errors
from test_oracle_bp import brute_force, random_tree


# ------------------------------------------------------------------ serial

def test_serial_two_checks_by_hand():
    # rows {0,1} and {1,2} share variable 1, so they form two layers
    H = np.array([[1, 1, 0], [0, 1, 1]], np.uint8)
    s = np.array([0, 1], np.uint8)
    mu = np.array([1.0, -2.0, 3.0])
    # check 0 (s = 0) sends m(0->0) = -2, m(0->1) = +1; check 1 (s = 1) then
    # sees q(1->1) = -2 + 1 = -1 and q(2->1) = 3, sends m(1->1) = -3 and
    # m(1->2) = +1 (flooding would send +2 from q = -2).
    ser = oracle.bp(H, s, mu, 1, 1.0, oracle.RULE_NMS, schedule=oracle.SCHEDULE_SERIAL)
    np.testing.assert_array_equal(ser["post"], [-1.0, -4.0, 4.0])
    assert ser["conv"] and ser["K"] == 1 and ser["ehat"].tolist() == [1, 1, 0]
    flo = oracle.bp(H, s, mu, 1, 1.0, oracle.RULE_NMS)
    np.testing.assert_array_equal(flo["post"], [-1.0, -4.0, 5.0])
    # normalized: alpha scales each check output once
    ser = oracle.bp(H, s, mu, 1, 0.5, oracle.RULE_NMS, schedule=oracle.SCHEDULE_SERIAL, early_stop=False)
    # m(0->0) = -1, m(0->1) = 0.5; q(1->1) = -1.5 -> m(1->2) = +0.75; m(1->1) = -1.5
    np.testing.assert_array_equal(ser["post"], [0.0, -3.0, 3.75])


def test_serial_layer_order_by_hand():
    # rows {0,1}, {1,2}, {2,3}: greedy layers {r0, r2}, {r1}, so the order is
    # r0, r2, r1 (row order r0, r1, r2 would give v1 = -4 and v3 = 4.5)
    H = np.array([[1, 1, 0, 0], [0, 1, 1, 0], [0, 0, 1, 1]], np.uint8)
    s = np.array([0, 1, 0], np.uint8)
    mu = np.array([1.0, -2.0, 3.0, 0.5])
    # r0: m(0->0) = -2, m(0->1) = 1; r2: q = (3, 0.5) -> m(2->2) = 0.5,
    # m(2->3) = 3; r1 (s = 1): q = (-2 + 1, 3 + 0.5) -> m(1->1) = -3.5,
    # m(1->2) = 1
    ser = oracle.bp(H, s, mu, 1, 1.0, oracle.RULE_NMS, early_stop=False, schedule=oracle.SCHEDULE_SERIAL)
    np.testing.assert_array_equal(ser["post"], [-1.0, -4.5, 4.5, 3.5])


@pytest.mark.parametrize("rule", [oracle.RULE_NMS, oracle.RULE_SP])
def test_serial_equals_flooding_on_disjoint_rows(rule):
    rng = np.random.default_rng(5)
    n = 24
    perm = rng.permutation(n)
    H = np.zeros((6, n), np.uint8)
    for r in range(6):
        H[r, perm[4 * r:4 * r + 4]] = 1
    for trial in range(5):
        s = rng.integers(0, 2, 6).astype(np.uint8)
        mu = rng.normal(1.0, 2.0, n)
        for iters in (1, 3, 7):
            a = oracle.bp(H, s, mu, iters, 0.75, rule, early_stop=False)
            b = oracle.bp(H, s, mu, iters, 0.75, rule, early_stop=False, schedule=oracle.SCHEDULE_SERIAL)
            np.testing.assert_array_equal(a["post"], b["post"])


@pytest.mark.parametrize("trial", range(10))
def test_serial_tree_exactness(trial):
    rng = np.random.default_rng(300 + trial)
    H = random_tree(rng)
    m, n = H.shape
    s = rng.integers(0, 2, m).astype(np.uint8)
    mu = rng.uniform(-1.0, 3.0, n)
    lr, mc = brute_force(H, s, mu)
    iters = 2 * n
    sp = oracle.bp(H, s, mu, iters, 1.0, oracle.RULE_SP, early_stop=False, schedule=oracle.SCHEDULE_SERIAL)
    np.testing.assert_allclose(sp["post"], lr, rtol=1e-9, atol=1e-9)
    ms = oracle.bp(H, s, mu, iters, 1.0, oracle.RULE_NMS, early_stop=False, schedule=oracle.SCHEDULE_SERIAL)
    np.testing.assert_allclose(ms["post"], mc, rtol=1e-12, atol=1e-12)


def _iters_to_exact(H, s, mu, schedule, target):
    for it in range(1, 200):
        r = oracle.bp(H, s, mu, it, 1.0, oracle.RULE_SP, early_stop=False, schedule=schedule)
        if np.allclose(r["post"], target, rtol=1e-10, atol=1e-10):
            return it
    return None


def test_serial_converges_faster_on_a_chain():
    # checks {i, i+1}, i = 0..10: a path; layers are the even and odd checks
    n = 12
    H = np.zeros((n - 1, n), np.uint8)
    for i in range(n - 1):
        H[i, i] = H[i, i + 1] = 1
    rng = np.random.default_rng(11)
    s = rng.integers(0, 2, n - 1).astype(np.uint8)
    mu = rng.uniform(0.5, 2.0, n)
    lr, _ = brute_force(H, s, mu)
    kf = _iters_to_exact(H, s, mu, oracle.SCHEDULE_FLOODING, lr)
    ks = _iters_to_exact(H, s, mu, oracle.SCHEDULE_SERIAL, lr)
    assert kf is not None and ks is not None
    assert ks < kf


@pytest.mark.parametrize("rule", [oracle.RULE_NMS, oracle.RULE_SP])
def test_serial_mbbp_candidates_satisfy_syndrome(rule):
    H = named_code("bb72").HZ
    m, n = H.shape
    R = 6
    sets = oracle.collect_subtrees(H, R, 3)
    e = random_errors(60, n, 0.06, 2)
    synd = oracle.syndrome(H, e)
    llr = np.full(n, np.log((1 - 0.04) / 0.04))
    out = oracle.mbbp_decode(H, sets, synd, llr, 40, 0.875, rule, schedule=oracle.SCHEDULE_SERIAL)
    for b in range(60):
        for t in range(R):
            if out["conv"][b, t]:
                assert np.array_equal(oracle.syndrome(H, out["cand"][b, t][None])[0], synd[b])
    assert out["conv"].mean() > 0.5
    # converging at least as often as flooding at the same iteration cap
    flo = oracle.mbbp_decode(H, sets, synd, llr, 40, 0.875, rule)
    assert out["success"].sum() >= flo["success"].sum() - 2


# ---------------------------------------------------------------------- LMS

def test_lms_hand_lists():
    mu = np.array([1.0, 2.0, 3.0, 4.0, 5.0, 6.0], np.float32)
    c = np.array([[1, 1, 0, 0, 0, 0],    # 3
                  [0, 0, 1, 0, 0, 0],    # 3 (tie with the first)
                  [0, 0, 0, 0, 0, 1],    # 6
                  [1, 0, 0, 0, 0, 0]],   # 1, but not converged
                 np.uint8)
    ehat, ok, sel = oracle.lms(c, [1, 1, 1, 0], mu)
    assert ok and sel == 0 and ehat.tolist() == c[0].tolist()
    _, _, sel = oracle.lms(c, [0, 1, 1, 1], mu)
    assert sel == 3
    # negative LLRs: setting a bit with mu < 0 lowers the metric
    mu2 = np.array([1.0, -2.0, 3.0, 4.0, 5.0, 6.0], np.float32)
    _, _, sel = oracle.lms(c, [1, 1, 1, 0], mu2)
    assert sel == 0  # metric -1 < 3 < 6
    # frequency does not matter to LMS (FWS would pick the repeated estimate)
    c3 = np.array([[0, 0, 1, 1, 0, 0], [0, 0, 1, 1, 0, 0], [1, 1, 0, 0, 0, 0]], np.uint8)
    _, _, sel = oracle.lms(c3, [1, 1, 1], mu)
    assert sel == 2
    _, _, fsel = oracle.fws(c3, [1, 1, 1])
    assert fsel == 0
    ehat, ok, sel = oracle.lms(c, [0, 0, 0, 0], mu)
    assert not ok and sel == -1 and ehat.sum() == 0


def test_lms_brute_force_argmin():
    rng = np.random.default_rng(9)
    for _ in range(50):
        R, n = int(rng.integers(1, 10)), int(rng.integers(1, 40))
        c = rng.integers(0, 2, (R, n)).astype(np.uint8)
        conv = rng.integers(0, 2, R).astype(np.uint8)
        mu = rng.integers(-8, 9, n).astype(np.float32) / 4  # exact sums, ties likely
        ehat, ok, sel = oracle.lms(c, conv, mu)
        metric = [sum(float(mu[v]) for v in range(n) if c[a, v]) for a in range(R)]
        cands = [a for a in range(R) if conv[a]]
        if not cands:
            assert sel == -1 and not ok
            continue
        best = min(cands, key=lambda a: (metric[a], a))
        assert sel == best and ehat.tolist() == c[best].tolist()


def test_lms_decode_picks_the_least_metric():
    H = named_code("bb72").HZ
    m, n = H.shape
    sets = oracle.collect_subtrees(H, 8, 1)
    rng = np.random.default_rng(4)
    e = random_errors(80, n, 0.07, 4)
    synd = oracle.syndrome(H, e)
    llr = rng.uniform(1.0, 4.0, (80, n)).astype(np.float32)
    out = oracle.mbbp_decode(H, sets, synd, llr, 30, 0.625, precision="f32", decision=oracle.DECISION_LMS)
    for b in range(80):
        conv = out["conv"][b]
        if not conv.any():
            assert out["selected"][b] == -1 and out["ehat"][b].sum() == 0
            continue
        met = [float(np.float32(llr[b][out["cand"][b, t] == 1].astype(np.float64).sum())) for t in range(8)]
        sel = int(out["selected"][b])
        assert conv[sel]
        for t in range(8):
            if conv[t]:
                assert met[sel] <= met[t] + 1e-4


# ------------------------------------------------------------ random sets

def test_random_sets_sizes_ranges_and_prefixes():
    m = 36
    sizes = [0, 1, 5, 36, 40, 12]
    sets = oracle.random_sets(m, sizes, 123)
    for s, k in zip(sets, sizes):
        assert len(s) == min(k, m)
        assert len(set(s.tolist())) == len(s)
        assert all(0 <= r < m for r in s)
    # set t is a prefix of a permutation fixed by (seed, t)
    longer = oracle.random_sets(m, [36] * 6, 123)
    for s, full in zip(sets, longer):
        assert s.tolist() == full[:len(s)].tolist()
        assert sorted(full.tolist()) == list(range(m))
    # reproducible, and different seeds / indices give different sets
    assert [x.tolist() for x in oracle.random_sets(m, sizes, 123)] == [x.tolist() for x in sets]
    assert longer[0].tolist() != longer[1].tolist()
    assert oracle.random_sets(m, [36], 124)[0].tolist() != longer[0].tolist()


def test_random_sets_first_row_is_uniform():
    m, T = 6, 6000
    first = np.array([s[0] for s in oracle.random_sets(m, [1] * T, 77)])
    counts = np.bincount(first, minlength=m)
    exp = T / m
    chi2 = float(((counts - exp) ** 2 / exp).sum())
    assert chi2 < 20.5  # 5 degrees of freedom, p ~ 0.001
