"""Pins of the oracle's syndrome BP (Section II-B).

BP is exact on trees (Section III-A cites Gallager for this), so on random
tree-shaped Tanner graphs:

* sum-product posteriors equal the exact bitwise-MAP log-ratios
  log sum_{He=s, e_i=0} P(e) / sum_{He=s, e_i=1} P(e)  (brute force over 2^n);
* min-sum with alpha = 1 posteriors equal the exact min-cost differences
  min_{He=s, e_i=1} sum mu_j e_j - min_{He=s, e_i=0} sum mu_j e_j.

A dropped term, a wrong sign (syndrome or product) or a wrong exclusion index
changes these values.  Also pinned: the halting rule (H e = s for every
converged output, recomputed here), K = 0 for s = 0, the alpha scaling of the
normalized rule on a single check, and FP32/FP64 agreement on BB codes.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2605_14170_gb300.inputs import named_code, random_errors


def random_tree(rng, max_n=14):
    """Random tree Tanner graph: each new check shares exactly one variable
    with the graph built so far and adds 1-3 new variables."""
    rows = []
    d0 = int(rng.integers(2, 5))
    rows.append(list(range(d0)))
    n = d0
    while True:
        k = int(rng.integers(1, 4))
        if n + k > max_n:
            break
        anchor = int(rng.integers(0, n))
        rows.append([anchor] + list(range(n, n + k)))
        n += k
    H = np.zeros((len(rows), n), np.uint8)
    for r, cols in enumerate(rows):
        H[r, cols] = 1
    return H


def brute_force(H, s, mu):
    m, n = H.shape
    E = np.array(list(itertools.product([0, 1], repeat=n)), np.uint8)
    ok = ((E.astype(np.int64) @ H.T.astype(np.int64)) % 2 == s).all(axis=1)
    E = E[ok]
    cost = E.astype(np.float64) @ mu
    w = np.exp(-(cost - cost.min()))
    lr = np.empty(n)
    mc = np.empty(n)
    for i in range(n):
        z, o = E[:, i] == 0, E[:, i] == 1
        lr[i] = np.log(w[z].sum()) - np.log(w[o].sum())
        mc[i] = cost[o].min() - cost[z].min()
    return lr, mc


@pytest.mark.parametrize("trial", range(12))
def test_tree_exactness_sum_product_and_min_sum(trial):
    rng = np.random.default_rng(100 + trial)
    H = random_tree(rng)
    m, n = H.shape
    s = rng.integers(0, 2, m).astype(np.uint8)
    mu = rng.uniform(-1.0, 3.0, n)
    lr, mc = brute_force(H, s, mu)
    iters = 2 * n  # more than the diameter
    sp = oracle.bp(H, s, mu, iters, 1.0, oracle.RULE_SP, early_stop=False)
    np.testing.assert_allclose(sp["post"], lr, rtol=1e-9, atol=1e-9)
    ms = oracle.bp(H, s, mu, iters, 1.0, oracle.RULE_NMS, early_stop=False)
    np.testing.assert_allclose(ms["post"], mc, rtol=1e-12, atol=1e-12)
    # on a tree the hard decision of min-sum is a minimum-cost solution
    if np.all(np.abs(mc) > 1e-9):
        assert ms["conv"]
        assert np.array_equal((H.astype(int) @ ms["ehat"]) % 2, s)


def test_single_check_closed_forms():
    """One check with three variables: after one iteration the posterior of
    v is mu_v + (-1)^s alpha min_{v' != v} |mu_v'| prod sign (min-sum) and
    mu_v + (-1)^s 2 atanh(prod tanh(mu_v'/2)) (sum-product)."""
    H = np.array([[1, 1, 1]], np.uint8)
    mu = np.array([0.5, -2.0, 3.0])
    for s in (0, 1):
        sg = -1.0 if s else 1.0
        r = oracle.bp(H, np.array([s], np.uint8), mu, 1, 0.75, oracle.RULE_NMS, early_stop=False)
        exp = mu + sg * 0.75 * np.array([-2.0, 0.5, -0.5])
        np.testing.assert_allclose(r["post"], exp, rtol=0, atol=1e-15)
        r = oracle.bp(H, np.array([s], np.uint8), mu, 1, 1.0, oracle.RULE_SP, early_stop=False)
        t = np.tanh(mu / 2)
        exp = mu + sg * 2 * np.arctanh(np.array([t[1] * t[2], t[0] * t[2], t[0] * t[1]]))
        np.testing.assert_allclose(r["post"], exp, rtol=1e-12)


def test_degree_one_row_and_zero_syndrome():
    H = np.array([[1, 0, 0], [0, 1, 1]], np.uint8)
    mu = np.array([2.0, 1.0, 1.5])
    r = oracle.bp(H, np.array([1, 0], np.uint8), mu, 1, 0.5, oracle.RULE_NMS, early_stop=False)
    # the single edge of row 0 receives -alpha * LMAX (syndrome bit 1)
    assert r["post"][0] == pytest.approx(2.0 - 0.5 * oracle.LMAX)
    assert r["ehat"].tolist() == [1, 0, 0] and r["conv"]
    r = oracle.bp(H, np.array([0, 0], np.uint8), mu, 10, 0.5)
    assert r["conv"] and r["K"] == 0 and r["ehat"].sum() == 0


@pytest.mark.parametrize("rule", [oracle.RULE_NMS, oracle.RULE_SP])
def test_halting_rule_on_bb_code(rule):
    c = named_code("bb72")
    H = c.HZ
    sets = oracle.collect_subtrees(H, 4, seed=1)
    e = random_errors(60, H.shape[1], 0.05, 5)
    s = oracle.syndrome(H, e)
    mu = np.full(H.shape[1], np.log(0.95 / 0.05))
    out = oracle.mbbp_decode(H, sets, s, mu, 50, 0.625, rule)
    for b in range(len(s)):
        for t in range(4):
            cand = out["cand"][b, t]
            ok = np.array_equal((H.astype(int) @ cand) % 2, s[b])
            assert bool(out["conv"][b, t]) == ok or out["iters"][b, t] == 50
            if out["conv"][b, t]:
                assert ok
                Ht = np.concatenate([H, H[sets[t]]])
                st = np.concatenate([s[b], s[b][sets[t]]])
                assert np.array_equal((Ht.astype(int) @ cand) % 2, st)
            else:
                assert out["iters"][b, t] == 50
        if out["success"][b]:
            assert np.array_equal((H.astype(int) @ out["ehat"][b]) % 2, s[b])
        else:
            assert out["ehat"][b].sum() == 0 and out["selected"][b] == -1
        if not s[b].any():
            assert (out["iters"][b] == 0).all() and out["ehat"][b].sum() == 0


def test_fp32_matches_fp64_on_bb_code():
    c = named_code("bb144")
    H = c.HZ
    sets = oracle.collect_subtrees(H, 4, seed=2)
    e = random_errors(40, H.shape[1], 0.04, 9)
    s = oracle.syndrome(H, e)
    mu = np.full(H.shape[1], np.log(0.96 / 0.04))
    a = oracle.mbbp_decode(H, sets, s, mu, 3, 0.625, precision="f64", want_post=True)
    b = oracle.mbbp_decode(H, sets, s, mu, 3, 0.625, precision="f32", want_post=True)
    ref = a["post"]
    np.testing.assert_allclose(b["post"], ref, rtol=1e-5, atol=1e-5)
    full64 = oracle.mbbp_decode(H, sets, s, mu, 50, 0.625, precision="f64")
    full32 = oracle.mbbp_decode(H, sets, s, mu, 50, 0.625, precision="f32")
    agree = (full64["ehat"] == full32["ehat"]).all(axis=1).mean()
    assert agree >= 0.95


def _sum_product_tanh_mp(Ht, st, mu, iters):
    """Flooding sum-product BP written with the textbook rule
    m_{c->v} = (-1)^{s_c} 2 atanh(prod_{v' != v} tanh(q_{v'->c} / 2)) in
    50-digit arithmetic (mpmath), with the oracle's readings: q^(0) = mu,
    |m| capped at SPMAX, q clamped to [-LMAX, LMAX]; no early stop.
    Returns (c2v per edge, row by row with columns ascending; posteriors)."""
    mpmath = pytest.importorskip("mpmath")
    mp = mpmath.mp
    mp.dps = 50
    M, n = Ht.shape
    rows = [list(np.nonzero(Ht[r])[0]) for r in range(M)]
    eidx, e = {}, 0
    for r in range(M):
        for v in rows[r]:
            eidx[(r, v)] = e
            e += 1
    cols = [[r for r in range(M) if Ht[r, v]] for v in range(n)]
    mu_mp = [mp.mpf(float(x)) for x in mu]
    v2c = [None] * e
    for (r, v), k in eidx.items():
        v2c[k] = mu_mp[v]
    c2v = [mp.mpf(0)] * e
    spmax, lmax = mp.mpf(oracle.SPMAX), mp.mpf(oracle.LMAX)
    post = list(mu_mp)
    for _ in range(iters):
        for r in range(M):
            ks = [eidx[(r, v)] for v in rows[r]]
            th = [mp.tanh(v2c[k] / 2) for k in ks]
            for j, k in enumerate(ks):
                prod = mp.mpf(1)
                for i, t in enumerate(th):
                    if i != j:
                        prod *= t
                m = 2 * mp.atanh(prod)
                if st[r]:
                    m = -m
                c2v[k] = max(-spmax, min(spmax, m))
        for v in range(n):
            ks = [eidx[(r, v)] for r in cols[v]]
            post[v] = mu_mp[v] + mp.fsum(c2v[k] for k in ks)
            for k in ks:
                q = mu_mp[v] + mp.fsum(c2v[k2] for k2 in ks if k2 != k)
                v2c[k] = max(-lmax, min(lmax, q))
    return np.array([float(x) for x in c2v]), np.array([float(x) for x in post])


@pytest.mark.parametrize("code,R", [("bb72", 2), ("bb144", 1)])
def test_sum_product_phi_form_equals_tanh_rule_on_loopy_graphs(code, R):
    """The oracle evaluates the sum-product rule as prod sign(q) phi(sum
    phi(|q|)) with Gallager's phi.  On the loopy Tanner graphs of the
    representations H^(t) of the BB codes, its FP64 check messages and
    posteriors after 1..5 flooding iterations equal the textbook rule
    2 atanh(prod tanh(q/2)) computed in 50-digit arithmetic, within 1e-9
    relative: the two forms are the same function, and the oracle's
    evaluation adds no error beyond FP64 rounding."""
    c = named_code(code)
    H = c.HZ
    n = H.shape[1]
    sets = oracle.collect_subtrees(H, R, 20260514)
    ex, _ = oracle.sample(20260514, 900, 3, n, 0.06, "depolarizing")
    synd = oracle.syndrome(H, ex)
    mu = np.full(n, np.log((1 - 0.04) / 0.04))
    for t, rows in enumerate(sets):
        Ht = np.vstack([H, H[rows]]).astype(np.uint8)
        for i in range(len(synd)):
            st = np.concatenate([synd[i], synd[i][rows]]).astype(np.uint8)
            for it in (1, 2, 5):
                ref_m, ref_p = _sum_product_tanh_mp(Ht, st, mu, it)
                got = oracle.bp(Ht, st, mu, it, 1.0, oracle.RULE_SP, early_stop=False, precision="f64",
                                want_c2v=True)
                gm = got["c2v"][Ht.astype(bool)]
                assert np.all(np.abs(gm - ref_m) <= 1e-9 * np.maximum(np.abs(ref_m), 1.0)), (code, t, i, it)
                assert np.all(np.abs(got["post"] - ref_p) <= 1e-9 * np.maximum(np.abs(ref_p), 1.0))
