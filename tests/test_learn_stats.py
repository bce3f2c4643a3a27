"""Host-side statistics of the learned-weight comparison (no GPU): the
Wilson interval and the one-sided two-proportion z statistic, against
their closed forms and scipy's normal distribution."""
import math

import pytest


def test_two_proportion_z_closed_form_and_symmetry():
    from paper_2605_14170_gb300 import learn
    n = 1_000_000
    # 700 vs 525 failures: pooled rate 612.5 / 1e6
    pp = 612.5e-6
    want = (175 / n) / math.sqrt(2 * pp * (1 - pp) / n)
    assert learn.two_proportion_z(700, 525, n) == pytest.approx(want, rel=1e-12)
    assert learn.two_proportion_z(525, 700, n) == pytest.approx(-want, rel=1e-12)
    assert learn.two_proportion_z(0, 0, n) == 0.0
    assert learn.two_proportion_z(10, 10, 100) == 0.0


def test_wilson_interval_matches_normal_quantile():
    scipy_stats = pytest.importorskip("scipy.stats")
    from paper_2605_14170_gb300 import learn
    z = float(scipy_stats.norm.ppf(0.975))
    for k, n in ((0, 100), (5, 100), (50, 100), (100, 100), (3, 10**6)):
        lo, hi = learn.wilson(k, n, z)
        ph = k / n
        # the interval's ends solve |ph - x| = z sqrt(x (1 - x) / n)
        for x in (lo, hi):
            if 1e-9 < x < 1.0 - 1e-9:
                assert abs(ph - x) == pytest.approx(z * math.sqrt(x * (1 - x) / n), rel=1e-9, abs=1e-15)
        assert lo <= ph <= hi
        if k == 0:
            assert lo == pytest.approx(0.0, abs=1e-12)
        if k == n:
            assert hi == pytest.approx(1.0, abs=1e-12)
