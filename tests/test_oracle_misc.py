"""Pins of the oracle's FWS rule, sampler, GF(2) helpers and logical judge."""
import numpy as np
import pytest

import oracle
from conftest import read_golden
from paper_2605_14170_gb300.inputs import gf2_rank_np, named_code


# ---------------------------------------------------------------- FWS (III-B)

def _cands(rows, n=6):
    return np.array([[int(ch) for ch in r.ljust(n, "0")] for r in rows], np.uint8)


def test_fws_empty_list_is_failure():
    c = _cands(["110000", "000001"])
    ehat, ok, sel = oracle.fws(c, [0, 0])
    assert not ok and sel == -1 and ehat.sum() == 0


def test_fws_frequency_and_weight():
    # A = 110000 (w 2) appears twice: 2/3; B = 100000 (w 1) once: 1/2 -> A
    c = _cands(["100000", "110000", "110000"])
    ehat, ok, sel = oracle.fws(c, [1, 1, 1])
    assert ok and sel == 1 and ehat.tolist() == [1, 1, 0, 0, 0, 0]
    # A = 111000 (w 3) twice: 2/4 ; B = 000000 (w 0) once: 1/1 -> B
    c = _cands(["111000", "000000", "111000"])
    _, ok, sel = oracle.fws(c, [1, 1, 1])
    assert sel == 1
    # non-converged entries are not in the list, however often they repeat
    c = _cands(["000011", "000011", "000011", "100000"])
    _, ok, sel = oracle.fws(c, [0, 0, 0, 1])
    assert sel == 3


def test_fws_ties_go_to_first_occurrence():
    # A = 100000 (w 1) once: 1/2 ; B = 011100 (w 3) twice: 2/4 -> tie
    c = _cands(["011100", "100000", "011100"])
    _, _, sel = oracle.fws(c, [1, 1, 1])
    assert sel == 0
    c = _cands(["100000", "011100", "011100"])
    _, _, sel = oracle.fws(c, [1, 1, 1])
    assert sel == 0
    # equal candidates: the first copy is reported
    c = _cands(["010000", "001000", "001000"])
    _, _, sel = oracle.fws(c, [1, 1, 1])
    assert sel == 1


# --------------------------------------------------------------- sampler

def test_splitmix64_published_values():
    vals = [r[0] for r in read_golden("splitmix64_seed0.txt")[None]]
    assert [oracle.splitmix64_at(0, i + 1) for i in range(3)] == vals


def test_sampler_rates_and_partition_invariance():
    n, batch, p = 50, 4000, 0.06
    ex, ez = oracle.sample(7, 0, batch, n, p, "depolarizing")
    x_only = (ex == 1) & (ez == 0)
    y = (ex == 1) & (ez == 1)
    z_only = (ex == 0) & (ez == 1)
    N = batch * n
    for frac in (x_only.sum() / N, y.sum() / N, z_only.sum() / N):
        assert abs(frac - p / 3) < 4 * np.sqrt(p / 3 / N)
    a, _ = oracle.sample(7, 100, 40, n, p, "depolarizing")
    assert np.array_equal(a, ex[100:140])
    bx, bz = oracle.sample(7, 0, batch, n, p, "bsc")
    assert bz.sum() == 0 and abs(bx.mean() - p) < 4 * np.sqrt(p / N)
    zx, zz = oracle.sample(7, 0, 10, n, 0.0, "depolarizing")
    assert zx.sum() == 0 and zz.sum() == 0


# --------------------------------------------------------------- GF(2) / codes

def test_gf2_rank_against_independent_elimination():
    rng = np.random.default_rng(1)
    assert oracle.gf2_rank(np.eye(7, dtype=np.uint8)) == 7
    assert oracle.gf2_rank(np.ones((5, 9), np.uint8)) == 1
    for _ in range(30):
        r, c = rng.integers(1, 30, 2)
        A = (rng.random((r, c)) < 0.3).astype(np.uint8)
        assert oracle.gf2_rank(A) == gf2_rank_np(A)


@pytest.mark.parametrize("code,n,k", [("bb72", 72, 12), ("bb144", 144, 12), ("bb288", 288, 12)])
def test_bb_codes_parameters(code, n, k):
    """[[72,12,6]], [[144,12,12]], [[288,12,18]]: H_X H_Z^T = 0 (Section II-A)
    and k = n - rank H_X - rank H_Z (the printed code parameters)."""
    c = named_code(code)
    assert c.HX.shape[1] == n
    assert not ((c.HX.astype(int) @ c.HZ.T.astype(int)) % 2).any()
    assert n - oracle.gf2_rank(c.HX) - oracle.gf2_rank(c.HZ) == k
    assert (c.HX.sum(axis=1) == 6).all() and (c.HX.sum(axis=0) == 3).all()


def test_syndrome_of_stabilizers_is_zero():
    c = named_code("bb72")
    s = oracle.syndrome(c.HZ, c.HX)  # X-type stabilizers commute with Z checks
    assert s.sum() == 0
    e = np.zeros((1, 72), np.uint8)
    e[0, 5] = 1
    assert np.array_equal(oracle.syndrome(c.HZ, e)[0], c.HZ[:, 5])


# --------------------------------------------------------------- judge

def test_judge_422_code():
    """[[4,2,2]]: H_X = H_Z = [1 1 1 1]."""
    H = np.ones((1, 4), np.uint8)
    z = np.zeros(4, np.uint8)
    cases = {(1, 1, 1, 1): 0, (1, 1, 0, 0): 2, (1, 0, 0, 0): 1, (0, 0, 0, 0): 0}
    for r, want in cases.items():
        assert oracle.judge(H, H, np.array(r, np.uint8), z)[0] == want


def test_judge_steane_code():
    """Steane code: checks of the [7,4] Hamming code for both types.  Weight-4
    Hamming codewords are stabilizers; weight-3 codewords are logical."""
    H = np.array([[1, 0, 1, 0, 1, 0, 1], [0, 1, 1, 0, 0, 1, 1], [0, 0, 0, 1, 1, 1, 1]], np.uint8)
    import itertools
    for bits in itertools.product([0, 1], repeat=7):
        r = np.array(bits, np.uint8)
        if ((H.astype(int) @ r) % 2).any():
            assert oracle.judge(H, H, r, np.zeros(7, np.uint8))[0] == 1
            continue
        w = int(r.sum())
        want = 0 if w in (0, 4) else 2
        assert oracle.judge(H, H, r, np.zeros(7, np.uint8))[0] == want
