"""Pins of the oracle's weighted min-sum (WMS) and its adjoint.

* w == alpha, g == 0 reproduces normalized min-sum (flooding, no early stop);
* on a tree with w == 1, g == 0 the posterior is the exact min-cost
  difference (max-product is exact on trees);
* the adjoint equals central finite differences of the forward (FP64) at
  points where no min or sign decision is within 10 h of a tie;
* a planted mistake in the adjoint (damping path dropped) breaks the
  finite-difference agreement.
"""
import numpy as np
import pytest

import oracle
from paper_2605_14170_gb300.inputs import named_code, random_errors
from test_oracle_bp import brute_force, random_tree


def _edges(Ht):
    return int(Ht.sum())


def test_wms_reduces_to_normalized_min_sum():
    c = named_code("bb72")
    H = c.HZ
    sets = oracle.collect_subtrees(H, 2, 1)
    e = random_errors(8, 72, 0.06, 3)
    s = oracle.syndrome(H, e)
    mu = np.full(72, np.log(0.94 / 0.06))
    for b in range(8):
        Ht = np.concatenate([H, H[sets[b % 2]]])
        st = np.concatenate([s[b], s[b][sets[b % 2]]])
        T, E = 7, _edges(Ht)
        _, post = oracle.wms_forward(Ht, st, mu, np.full((T, E), 0.625), np.zeros((T, E)))
        ref = oracle.bp(Ht, st, mu, T, 0.625, oracle.RULE_NMS, early_stop=False)
        np.testing.assert_allclose(post, ref["post"], rtol=0, atol=1e-12)


def test_wms_exact_on_trees():
    for trial in range(6):
        rng = np.random.default_rng(300 + trial)
        H = random_tree(rng)
        s = rng.integers(0, 2, H.shape[0]).astype(np.uint8)
        mu = rng.uniform(-1.0, 3.0, H.shape[1])
        _, mc = brute_force(H, s, mu)
        T, E = 2 * H.shape[1], _edges(H)
        _, post = oracle.wms_forward(H, s, mu, np.ones((T, E)), np.zeros((T, E)))
        np.testing.assert_allclose(post, mc, atol=1e-12)


def _random_point(seed, T=6):
    rng = np.random.default_rng(seed)
    c = named_code("bb72")
    H = c.HZ
    sets = oracle.collect_subtrees(H, 3, 2)
    t = sets[seed % 3]
    Ht = np.concatenate([H, H[t]])
    e = random_errors(1, 72, 0.07, seed)[0]
    s = oracle.syndrome(H, e[None])[0]
    st = np.concatenate([s, s[t]])
    mu = rng.uniform(1.5, 3.5, 72)  # distinct magnitudes: no exact ties in the mins
    E = _edges(Ht)
    w = rng.uniform(0.5, 1.0, (T, E))
    g = rng.uniform(0.0, 0.4, (T, E))
    return Ht, st, mu, w, g, e


@pytest.mark.parametrize("seed,all_iters", [(1, False), (2, False), (3, True), (4, True)])
def test_adjoint_matches_finite_differences(seed, all_iters):
    Ht, st, mu, w, g, e = _random_point(seed)
    L, gw, gg = oracle.wms_backward(Ht, st, mu, w, g, e, scale=1.0 / 72, all_iters=all_iters)
    L2, _ = oracle.wms_forward(Ht, st, mu, w, g, e, scale=1.0 / 72, all_iters=all_iters)
    assert L == pytest.approx(L2, rel=1e-14)
    rng = np.random.default_rng(seed)
    h = 1e-6
    checked = 0
    for _ in range(40):
        t = int(rng.integers(0, w.shape[0]))
        k = int(rng.integers(0, w.shape[1]))
        for P, G in ((w, gw), (g, gg)):
            Pp, Pm = P.copy(), P.copy()
            Pp[t, k] += h
            Pm[t, k] -= h
            args = (Pp, g) if P is w else (w, Pp)
            Lp, _ = oracle.wms_forward(Ht, st, mu, *args, e, scale=1.0 / 72, all_iters=all_iters)
            args = (Pm, g) if P is w else (w, Pm)
            Lm, _ = oracle.wms_forward(Ht, st, mu, *args, e, scale=1.0 / 72, all_iters=all_iters)
            fd = (Lp - Lm) / (2 * h)
            # a kink (min or sign switching inside [-h, h]) makes the central
            # difference disagree with both one-sided slopes; skip those points
            L0, _ = oracle.wms_forward(Ht, st, mu, w, g, e, scale=1.0 / 72, all_iters=all_iters)
            right, left = (Lp - L0) / h, (L0 - Lm) / h
            if abs(right - left) > 1e-4 * max(abs(right), abs(left), 1e-8):
                continue
            assert abs(fd - G[t, k]) <= 1e-3 * max(abs(fd), 1e-6), (t, k, fd, G[t, k])
            checked += 1
    assert checked >= 60
