"""Planted mistakes in the oracle must fail its pins.

Each case copies the oracle's C source to a temporary folder, plants one
plausible mistake (a dropped term, a wrong sign, a wrong index, a transposed
operand, an off-by-one in a test), compiles it with gcc and checks that at
least one pin no longer holds.  Everything runs on the CPU.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from conftest import read_golden
from test_oracle_bp import brute_force, random_tree

HERE = os.path.dirname(os.path.abspath(oracle.__file__))


def pins_hold():
    """The pins of test_oracle_*.py in compact form; False if any fails."""
    # Fig. 2
    g = read_golden("fig2_example.txt")
    H = np.array(g["H"], np.uint8)
    cs, order, ns = oracle.subtrees(H, np.array(g["pi"][0]) - 1)
    if ns != 2 or [c + 1 for c in order] != g["t1"][0] + g["t2"][0]:
        return False
    # trees: exact sum-product and min-sum
    for trial in range(6):
        rng = np.random.default_rng(100 + trial)
        Ht = random_tree(rng)
        s = rng.integers(0, 2, Ht.shape[0]).astype(np.uint8)
        mu = rng.uniform(-1.0, 3.0, Ht.shape[1])
        lr, mc = brute_force(Ht, s, mu)
        sp = oracle.bp(Ht, s, mu, 2 * Ht.shape[1], 1.0, oracle.RULE_SP, early_stop=False)
        ms = oracle.bp(Ht, s, mu, 2 * Ht.shape[1], 1.0, oracle.RULE_NMS, early_stop=False)
        if not (np.allclose(sp["post"], lr, atol=1e-9) and np.allclose(ms["post"], mc, atol=1e-12)):
            return False
    # single check, normalized min-sum scaling
    Hs = np.array([[1, 1, 1]], np.uint8)
    r = oracle.bp(Hs, np.array([1], np.uint8), np.array([0.5, -2.0, 3.0]), 1, 0.75,
                  oracle.RULE_NMS, early_stop=False)
    if not np.allclose(r["post"], np.array([0.5, -2.0, 3.0]) - 0.75 * np.array([-2.0, 0.5, -0.5])):
        return False
    # FWS hand-built lists
    def c(rows):
        return np.array([[int(ch) for ch in x] for x in rows], np.uint8)
    if oracle.fws(c(["100000", "110000", "110000"]), [1, 1, 1])[2] != 1:
        return False
    if oracle.fws(c(["111000", "000000", "111000"]), [1, 1, 1])[2] != 1:
        return False
    if oracle.fws(c(["011100", "100000", "011100"]), [1, 1, 1])[2] != 0:
        return False
    # serial schedule: worked examples (Section II-B)
    H3 = np.array([[1, 1, 0, 0], [0, 1, 1, 0], [0, 0, 1, 1]], np.uint8)
    r = oracle.bp(H3, np.array([0, 1, 0], np.uint8), np.array([1.0, -2.0, 3.0, 0.5]), 1, 1.0,
                  oracle.RULE_NMS, early_stop=False, schedule=oracle.SCHEDULE_SERIAL)
    if not np.array_equal(r["post"], [-1.0, -4.5, 4.5, 3.5]):
        return False
    for trial in range(3):
        rng = np.random.default_rng(300 + trial)
        Ht = random_tree(rng)
        s = rng.integers(0, 2, Ht.shape[0]).astype(np.uint8)
        mu = rng.uniform(-1.0, 3.0, Ht.shape[1])
        lr, mc = brute_force(Ht, s, mu)
        for rule, want in ((oracle.RULE_SP, lr), (oracle.RULE_NMS, mc)):
            r = oracle.bp(Ht, s, mu, 2 * Ht.shape[1], 1.0, rule, early_stop=False,
                          schedule=oracle.SCHEDULE_SERIAL)
            if not np.allclose(r["post"], want, atol=1e-9):
                return False
    # LMS hand lists (Section III-A)
    mu6 = np.array([1.0, -2.0, 3.0, 4.0, 5.0, 6.0], np.float32)
    if oracle.lms(c(["001000", "010000", "100000"]), [1, 1, 1], mu6)[2] != 1:
        return False
    if oracle.lms(c(["001000", "000100", "001000"]), [1, 1, 1], np.abs(mu6) * 0 + 1)[2] != 0:
        return False
    # judge on [[4,2,2]]
    H4 = np.ones((1, 4), np.uint8)
    z = np.zeros(4, np.uint8)
    want = {(1, 1, 1, 1): 0, (1, 1, 0, 0): 2, (1, 0, 0, 0): 1}
    for e, w in want.items():
        if oracle.judge(H4, H4, np.array(e, np.uint8), z)[0] != w:
            return False
    return True


MUTATIONS = {
    "syndrome sign dropped (min-sum)": ("bp_body.inc", "int neg = st[r] & 1;", "int neg = 0;"),
    "own edge not excluded (check)": ("bp_body.inc", "if (k == j) continue;\n                            REAL x",
                                      "REAL x"),
    "own edge not excluded (variable)": ("bp_body.inc", "if (k == i) continue;", ""),
    "syndrome sign dropped (sum-product)": ("bp_body.inc", "REAL sum = (REAL)0;\n                        int neg = st[r] & 1;",
                                            "REAL sum = (REAL)0;\n                        int neg = 0;"),
    "sign of q ignored (sum-product)": ("bp_body.inc", "sum = sum + PHI(FABS(v2c[k]));\n                            if (v2c[k] < (REAL)0) neg ^= 1;",
                                        "sum = sum + PHI(FABS(v2c[k]));"),
    "alpha not applied": ("bp_body.inc", "REAL mag = alpha * mn;", "REAL mag = mn;"),
    "eta test off by one": ("mbbp_oracle.c", "if (eta <= 1) {", "if (eta <= 2) {"),
    "FWS operands transposed": ("mbbp_oracle.c", "cnt * (best_w + 1) > best_cnt * (w + 1)",
                                "cnt * (w + 1) > best_cnt * (best_w + 1)"),
    "FWS ties to last": ("mbbp_oracle.c", "cnt * (best_w + 1) > best_cnt * (w + 1)",
                         "cnt * (best_w + 1) >= best_cnt * (w + 1)"),
    "judge rank test inverted": ("mbbp_oracle.c", "> base ? 2 : 0", ">= base ? 2 : 0"),
    "serial: stale check messages": ("bp_body.inc", "                        q = q + c2v[k];\n", ""),
    "serial: own edge not excluded": ("bp_body.inc", "if (k == j) continue;\n                        q = q + c2v[k];",
                                      "q = q + c2v[k];"),
    "serial: syndrome sign dropped": ("bp_body.inc", "int neg = st[r] & 1;\n                    if (rule == OR_RULE_NMS) {",
                                      "int neg = 0;\n                    if (rule == OR_RULE_NMS) {"),
    "serial: layers ignore shared variables": ("bp_body.inc", "if (used[(size_t)L * (n + 1) + edge_col[k]]) clash = 1;",
                                               "if (used[(size_t)L * (n + 1) + edge_col[k]]) clash = 0;"),
    "LMS ties to last": ("mbbp_oracle.c", "mt < best_m", "mt <= best_m"),
    "LMS metric drops the sign of mu": ("mbbp_oracle.c", "mt = mt + mu[v];", "mt = mt + fabsf(mu[v]);"),
}


@pytest.fixture(autouse=True)
def _restore():
    yield
    oracle.use_library(None)


def test_unmutated_oracle_holds_pins():
    assert pins_hold()


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_is_caught(name, tmp_path):
    fname, old, new = MUTATIONS[name]
    for f in ("mbbp_oracle.c", "bp_body.inc"):
        shutil.copy(os.path.join(HERE, f), tmp_path / f)
    src = (tmp_path / fname).read_text()
    assert old in src, name
    (tmp_path / fname).write_text(src.replace(old, new, 1))
    so = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                           str(tmp_path / "mbbp_oracle.c"), "-o", str(so), "-lm"])
    oracle.use_library(str(so))
    assert not pins_hold(), f"planted mistake not caught: {name}"
