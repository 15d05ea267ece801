"""Time-series analysis of detection records (host side, numpy).

The paper's scaling results are the slopes of the mean string separations
in conformal time over a late window, e.g. eta in [950, 1024] for the 4096^3
runs (Sec. V), and the asymptotic velocities; these helpers turn a list of
records (Lattice.read_records) into series and fit xi-dot per species by
least squares over a window.
"""
from __future__ import annotations

import numpy as np

SERIES = ("xi_p", "xi_q", "xi_pq", "xi_w", "f_total", "f_p")
DIAG_SERIES = ("xi_l", "xi_l_p", "xi_l_q", "v2_l", "v2_pq")


def series(records) -> dict:
    """Arrays over the records: eta plus the string and diagnostic fields."""
    out = {"eta": np.array([s["eta"] for s, _ in records], dtype=np.float64)}
    for k in SERIES:
        out[k] = np.array([s[k] for s, _ in records], dtype=np.float64)
    for k in DIAG_SERIES:
        out[k] = np.array([d[k] for _, d in records], dtype=np.float64)
    return out


def slope(eta, y, lo: float, hi: float):
    """Least-squares line y = s eta + b over lo <= eta <= hi (finite points
    only); returns (s, b, number of points)."""
    eta = np.asarray(eta, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    m = (eta >= lo) & (eta <= hi) & np.isfinite(y)
    if m.sum() < 2:
        return float("nan"), float("nan"), int(m.sum())
    A = np.stack([eta[m], np.ones(int(m.sum()))], axis=1)
    (s, b), *_ = np.linalg.lstsq(A, y[m], rcond=None)
    return float(s), float(b), int(m.sum())


def scaling_slopes(records, lo: float, hi: float) -> dict:
    """xi-dot of every separation estimator over the window [lo, hi]."""
    ser = series(records)
    return {k: slope(ser["eta"], ser[k], lo, hi)[0]
            for k in ("xi_p", "xi_q", "xi_pq", "xi_w", "xi_l", "xi_l_p", "xi_l_q")}
