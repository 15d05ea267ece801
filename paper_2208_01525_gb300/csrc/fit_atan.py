"""Coefficients of the FP32 edge-phase routine (arctangent on [0, 1]).

The FP32 kernels compute the gauge-invariant edge phase chi = arg(z) of
z = conj(phi(x)) U_i(x) phi(x+i) (Sec. III.A) by octant reduction,
t = min(|Re z|, |Im z|) / max(|Re z|, |Im z|) in [0, 1], and an odd
polynomial atan(t) ~ t * P(t^2).  This script derives P: the Remez exchange
algorithm for the minimax approximation of atan on [0, 1] among odd
polynomials of degree 2*DEG+1, run in double precision on a dense grid.

    python paper_2208_01525_gb300/csrc/fit_atan.py

prints the coefficients (lowest order first) and the maximum absolute error
of the exact-arithmetic polynomial; they are pasted into site_math.cuh.
"""
import numpy as np

DEG = 7  # P has DEG + 1 coefficients: atan(t) ~ sum_k c_k t^(2k+1), k = 0..DEG


def remez(deg: int, iters: int = 40):
    n = deg + 1
    m = n + 1  # reference points: n coefficients + the levelled error
    x = 0.5 - 0.5 * np.cos(np.pi * np.arange(m) / (m - 1))
    x[0] = 1e-3  # the error vanishes at t = 0; start the reference just above it
    grid = np.linspace(1e-6, 1.0, 400001)
    c = None
    for _ in range(iters):
        a = np.zeros((m, n + 1))
        for k in range(n):
            a[:, k] = x ** (2 * k + 1)
        a[:, n] = (-1.0) ** np.arange(m)
        sol = np.linalg.solve(a, np.arctan(x))
        c = sol[:n]
        err = np.arctan(grid) - grid * np.polyval(c[::-1], grid * grid)
        runs = np.split(np.arange(grid.size), np.where(np.diff(np.sign(err)) != 0)[0] + 1)
        pts = np.array([r[np.argmax(np.abs(err[r]))] for r in runs])
        if pts.size < m:
            break
        if pts.size > m:
            best = max(range(pts.size - m + 1), key=lambda i: np.min(np.abs(err[pts[i:i + m]])))
            pts = pts[best:best + m]
        x = grid[pts]
    err = np.arctan(grid) - grid * np.polyval(c[::-1], grid * grid)
    return c, float(np.max(np.abs(err)))


if __name__ == "__main__":
    coef, e = remez(DEG)
    for k, v in enumerate(coef):
        print(f"c{k} = {v:.9e}f")
    print(f"max |atan(t) - t P(t^2)| on [0, 1] = {e:.3e}")
