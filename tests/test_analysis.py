"""Slope fitting of separation time series (host side)."""
import math

import numpy as np

from paper_2208_01525_gb300 import analysis as A


def test_slope_recovers_a_line_and_ignores_points_outside_the_window():
    eta = np.linspace(0, 100, 201)
    y = 0.25 * eta + 3.0
    y[eta < 40] = -7.0           # outside the window, must not matter
    y[150] = np.inf              # non-finite points are dropped
    s, b, n = A.slope(eta, y, 50.0, 100.0)
    assert abs(s - 0.25) < 1e-12 and abs(b - 3.0) < 1e-10 and n == 100


def test_scaling_slopes_from_records():
    recs = []
    for k in range(20):
        eta = 10.0 + k
        s = {key: 0.0 for key in A.SERIES}
        s.update(eta=eta, xi_p=0.3 * eta, xi_q=0.28 * eta + 1, xi_pq=2.0 * eta, xi_w=0.2 * eta)
        d = {key: 0.0 for key in A.DIAG_SERIES}
        d.update(xi_l=0.19 * eta, xi_l_p=0.31 * eta, xi_l_q=0.29 * eta)
        recs.append((s, d))
    sl = A.scaling_slopes(recs, 12.0, 28.0)
    for k, v in (("xi_p", 0.3), ("xi_q", 0.28), ("xi_pq", 2.0), ("xi_w", 0.2), ("xi_l", 0.19),
                 ("xi_l_p", 0.31), ("xi_l_q", 0.29)):
        assert math.isclose(sl[k], v, rel_tol=1e-12), k
    assert math.isnan(A.slope([1.0], [2.0], 0, 5)[0])
