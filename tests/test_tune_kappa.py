"""Host logic of the kappa tuning (paper_1710_06198_gb300.tune_kappa.find_crossing) on model
sigma(m0) curves: the first crossing from above is found whether the walk lands below the target
or steps over a narrow dip (sigma ~ |m0 - m_c| near a real eigenvalue of the Wilson operator)."""
import pytest

from paper_1710_06198_gb300.tune_kappa import find_crossing


@pytest.mark.parametrize("m_c", [-0.7465, -0.7123, -0.83])
def test_dip_between_walk_points(m_c):
    target = 5e-4
    sig = lambda m: abs(m - m_c) + 0.0 * m + (0.3 if m < -1.0 else 0.0)
    m0, ev = find_crossing(sig, target, start_m0=-0.6, step=0.05)
    assert abs(ev[m0] - target) <= 0.02 * target
    assert m0 > m_c                                   # the upper branch: first crossing from above
    assert len(ev) < 45


def test_monotone_curve_crossed_by_the_walk():
    target = 1e-3
    sig = lambda m: max(0.0, m + 0.9) * 2.0 + 1e-5
    m0, ev = find_crossing(sig, target, start_m0=0.0, step=0.1)
    assert abs(ev[m0] - target) <= 0.02 * target and m0 > -0.9
