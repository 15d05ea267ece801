"""Table of the FP64 link-phase routine (sine and cosine of theta = dx A).

The FP64 kernels evaluate cos(theta) and sin(theta) of every link angle by
the table-driven method (Tang 1989): theta = m h + r with h = 2 pi / N,
m = rint(theta / h) and |r| <= h / 2; sin(m h) and cos(m h) come from an
N-entry table indexed by m mod N, and sin r, cos r from short Taylor
polynomials, combined by the angle-addition formulas.  This script writes
the table and the reduction constants, each correctly rounded to double
from 40-digit values (mpmath), into sincos_table.cuh:

    python paper_2208_01525_gb300/csrc/gen_sincos_table.py

h is split as h1 + h2 (Cody & Waite 1980): h1 keeps the top H1_BITS bits of
h so that m * h1 is exact for |m| < 2**(53 - H1_BITS), and h2 = h - h1
rounded to double.
"""
import os

import mpmath

N = 1024
H1_BITS = 30
mpmath.mp.dps = 40

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "sincos_table.cuh")


def hexd(v) -> str:
    return float(v).hex()


def main():
    two_pi = 2 * mpmath.pi
    h = two_pi / N
    # h1: h truncated to H1_BITS significant bits
    e = int(mpmath.floor(mpmath.log(h, 2)))
    scale = mpmath.mpf(2) ** (H1_BITS - 1 - e)
    h1 = mpmath.floor(h * scale) / scale
    h2 = h - h1
    inv_h = N / two_pi
    lines = [
        "// Generated by gen_sincos_table.py: sin and cos of m * 2 pi / "
        f"{N} for m = 0 .. {N - 1},",
        "// correctly rounded to double, and the constants of the reduction",
        "// theta = m h + r (h = 2 pi / N split as h1 + h2, h1 with "
        f"{H1_BITS} significant bits).",
        "#pragma once",
        "",
        "namespace u1u1 {",
        "",
        f"constexpr int SINCOS_TAB_N = {N};",
        f"constexpr double SINCOS_TAB_INV_H = {hexd(inv_h)};  // N / (2 pi)",
        f"constexpr double SINCOS_TAB_H1 = {hexd(h1)};",
        f"constexpr double SINCOS_TAB_H2 = {hexd(h2)};",
        f"// |m| below this keeps m * h1 exact: |theta| < 2^{53 - H1_BITS} h",
        f"constexpr double SINCOS_TAB_MAX_ARG = {hexd(mpmath.mpf(2) ** (53 - H1_BITS) * h1)};",
        "",
        "// {sin(m h), cos(m h)}",
        f"__device__ const double2 k_sincos_tab[{N}] = {{",
    ]
    for m in range(N):
        a = m * h
        lines.append(f"    {{{hexd(mpmath.sin(a))}, {hexd(mpmath.cos(a))}}},")
    lines += ["};", "", "}  // namespace u1u1", ""]
    with open(OUT, "w") as f:
        f.write("\n".join(lines))
    print(f"wrote {OUT}: h1 = {float(h1)!r}, h2 = {float(h2)!r}")


if __name__ == "__main__":
    main()
