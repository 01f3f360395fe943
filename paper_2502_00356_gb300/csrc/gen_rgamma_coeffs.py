"""Write bk_rgamma_coeffs.inc: Taylor coefficients of the reciprocal gamma
function, 1/Gamma(z) = sum_{k>=1} c_k z^k, split for Temme's series.

With them, for |mu| <= 1/2,
    G2(mu) = [1/Gamma(1-mu) + 1/Gamma(1+mu)] / 2 =  sum_{k odd}  c_k mu^{k-1},
    G1(mu) = [1/Gamma(1-mu) - 1/Gamma(1+mu)] / (2 mu) = -sum_{k even} c_k mu^{k-2},
    1/Gamma(1 +- mu) = G2 -+ mu G1,
which is how the GPU series evaluates G1 without the cancellation of its
defining difference near mu = 0.  The coefficients come from mpmath at 50
digits (mpmath.taylor of mpmath.rgamma), rounded once to double; terms up to
k = 29 (the first dropped term is below 1e-20 at |mu| = 1/2).

    python paper_2502_00356_gb300/csrc/gen_rgamma_coeffs.py
"""
from __future__ import annotations

import os

K_MAX = 29


def coefficients() -> list[float]:
    import mpmath
    mpmath.mp.dps = 50
    c = mpmath.taylor(mpmath.rgamma, 0, K_MAX)
    return [float(v) for v in c]  # c[0] = 0, c[k] for k = 1..K_MAX


def main() -> str:
    c = coefficients()
    odd = [c[k] for k in range(1, K_MAX + 1, 2)]       # G2: c_1, c_3, ... (powers mu^0, mu^2, ...)
    even = [-c[k] for k in range(2, K_MAX + 1, 2)]     # G1: -c_2, -c_4, ...
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "bk_rgamma_coeffs.inc")
    lines = ["// Taylor coefficients of 1/Gamma(z) for Temme's G1, G2 in powers of mu^2;",
             "// written by gen_rgamma_coeffs.py (mpmath, 50 digits).",
             f"constexpr int kG2Terms = {len(odd)};",
             "static __constant__ double kG2Coef[kG2Terms] = {"]
    lines += [f"    {v.hex()}," for v in odd]
    lines += ["};", f"constexpr int kG1Terms = {len(even)};",
              "static __constant__ double kG1Coef[kG1Terms] = {"]
    lines += [f"    {v.hex()}," for v in even]
    lines += ["};"]
    with open(out, "w") as f:
        f.write("\n".join(lines) + "\n")
    return out


if __name__ == "__main__":
    print(main())
