"""Pins of the oracle's Algorithm 2 (maximal subtrees, Section III-A).

* the worked example of Fig. 2 / Example 1, exactly;
* Lemma 1 (|t| <= (|V_v|-1)/(w-1)) and the equality |N(t)| = 1 + (w-1)|t|
  that its proof gives for check-regular graphs;
* every subtree induces a tree (connected, |E| = |V| - 1);
* the subtrees partition the checks;
* maximality: a check assigned later that touches N(t) has >= 2 neighbours
  in N(t), so it would close a cycle;
* every redundant row lies in the GF(2) row space of H.
"""
import numpy as np
import pytest

import oracle
from conftest import read_golden
from paper_2605_14170_gb300.inputs import named_code


def _neighbours(H, rows):
    return set(np.nonzero(H[list(rows)].any(axis=0))[0].tolist())


def _is_tree(H, rows):
    rows = list(rows)
    cols = sorted(_neighbours(H, rows))
    nodes = len(rows) + len(cols)
    edges = int(H[np.ix_(rows, cols)].sum())
    if edges != nodes - 1:
        return False
    # connectivity by BFS over the bipartite graph
    seen_r, seen_c = {rows[0]}, set()
    frontier = [("r", rows[0])]
    rset = set(rows)
    while frontier:
        kind, x = frontier.pop()
        if kind == "r":
            for c in np.nonzero(H[x])[0]:
                if c not in seen_c:
                    seen_c.add(int(c))
                    frontier.append(("c", int(c)))
        else:
            for r in np.nonzero(H[:, x])[0]:
                if r in rset and r not in seen_r:
                    seen_r.add(int(r))
                    frontier.append(("r", int(r)))
    return len(seen_r) == len(rows) and len(seen_c) == len(cols)


def test_fig2_worked_example():
    g = read_golden("fig2_example.txt")
    H = np.array(g["H"], np.uint8)
    perm = np.array(g["pi"][0]) - 1
    cs, order, ns = oracle.subtrees(H, perm)
    assert ns == 2
    t1 = [c for c in order if cs[c] == 1]
    t2 = [c for c in order if cs[c] == 2]
    assert [c + 1 for c in t1] == g["t1"][0]
    assert [c + 1 for c in t2] == g["t2"][0]
    # augmented matrices of Eq. (4), extra rows in acceptance order
    assert np.array_equal(np.concatenate([H, H[t1]]), np.array(g["Ht1"], np.uint8))
    assert np.array_equal(np.concatenate([H, H[t2]]), np.array(g["Ht2"], np.uint8))


@pytest.mark.parametrize("code", ["bb72", "bb144", "bb288"])
@pytest.mark.parametrize("which", ["HX", "HZ"])
def test_lemma1_tree_partition_maximality(code, which):
    c = named_code(code)
    H = getattr(c, which)
    m, n = H.shape
    w = int(H.sum(axis=1)[0])
    assert (H.sum(axis=1) == w).all()
    for j in range(3):
        perm = oracle.permutation(11, j, m)
        cs, order, ns = oracle.subtrees(H, perm)
        # partition: every check in exactly one subtree, order is a permutation
        assert sorted(order.tolist()) == list(range(m))
        assert cs.min() == 1 and cs.max() == ns
        subtrees = [[c for c in order if cs[c] == s] for s in range(1, ns + 1)]
        assert sum(len(t) for t in subtrees) == m
        # the first root is the first entry of the permutation
        assert subtrees[0][0] == perm[0]
        for s, t in enumerate(subtrees, start=1):
            Nt = _neighbours(H, t)
            assert len(t) <= (n - 1) / (w - 1)          # Lemma 1
            assert len(Nt) == 1 + (w - 1) * len(t)      # proof of Lemma 1
            assert _is_tree(H, t)
            # maximality against every check assigned later
            for c2 in range(m):
                if cs[c2] > s:
                    k = len(Nt & set(np.nonzero(H[c2])[0].tolist()))
                    assert k == 0 or k >= 2


def test_lemma1_bound_gb():
    """The 0.4 |V_c| form of Lemma 1 for a weight-6 GB code."""
    c = named_code("gb882")
    H = c.HZ
    m, n = H.shape
    cs, order, ns = oracle.subtrees(H, oracle.permutation(5, 1, m))
    sizes = np.bincount(cs)[1:]
    assert sizes.max() <= (2 * m - 1) / 5 <= 0.4 * m
    assert sizes.sum() == m


@pytest.mark.parametrize("code", ["bb72", "bb144"])
def test_collection_rowspace_and_dedup(code):
    c = named_code(code)
    H = c.HZ
    R = 16
    sets = oracle.collect_subtrees(H, R, seed=3)
    assert len(sets) == R
    keys = [frozenset(s.tolist()) for s in sets]
    assert len(set(keys)) == R
    # the subtrees of the identity order come first, in creation order
    cs, order, ns = oracle.subtrees(H, np.arange(H.shape[0]))
    first = [[c for c in order if cs[c] == s] for s in range(1, ns + 1)]
    for a, b in zip(sets, first):
        assert a.tolist() == b
    rank_H = oracle.gf2_rank(H)
    for s in sets:
        Ht = np.concatenate([H, H[s]])
        assert oracle.gf2_rank(Ht) == rank_H  # redundant rows lie in rowspace(H)
        assert oracle.gf2_rank(np.concatenate([H[s]])) == len(s)  # tree rows are independent


def test_permutations():
    m = 9
    assert oracle.permutation(1, 0, m).tolist() == list(range(m))
    seen = set()
    for j in range(1, 200):
        p = oracle.permutation(1, j, m)
        assert sorted(p.tolist()) == list(range(m))
        seen.add(tuple(p.tolist()))
    assert len(seen) > 190
    # Fisher-Yates gives a uniform position for each element
    m = 4
    counts = np.zeros((m, m))
    for j in range(1, 4001):
        p = oracle.permutation(99, j, m)
        counts[np.arange(m), p] += 1
    assert np.abs(counts / 4000 - 0.25).max() < 0.04


def test_random_small_graphs_are_trees():
    rng = np.random.default_rng(0)
    for _ in range(40):
        m, n = rng.integers(3, 9), rng.integers(4, 12)
        H = (rng.random((m, n)) < 0.35).astype(np.uint8)
        H[H.sum(axis=1) == 0, 0] = 1
        perm = rng.permutation(m).astype(np.int32)
        cs, order, ns = oracle.subtrees(H, perm)
        assert sorted(order.tolist()) == list(range(m))
        for s in range(1, ns + 1):
            t = [c for c in order if cs[c] == s]
            assert _is_tree(H, t)
            Nt = _neighbours(H, t)
            for c2 in range(m):
                if cs[c2] > s:
                    k = len(Nt & set(np.nonzero(H[c2])[0].tolist()))
                    assert k == 0 or k >= 2
