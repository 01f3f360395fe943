"""Write bk_exp2_table.inc: 2^{j/4096}, j = 0..4095, as C hex-float literals.

Each value is computed with 80-digit decimal arithmetic and rounded once to
the nearest double (float() of a decimal string rounds correctly), so every
entry is the correctly rounded 2^{j/4096}.  The table backs the table-driven
exponential of the FP64 kernels (bk_math64.cuh).

    python paper_2502_00356_gb300/csrc/gen_exp2_table.py
"""
from __future__ import annotations

import os
from decimal import Decimal, getcontext

N = 4096


def values() -> list[float]:
    getcontext().prec = 80
    ln2 = Decimal(2).ln()
    return [float(str((ln2 * j / N).exp())) for j in range(N)]


def main() -> str:
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "bk_exp2_table.inc")
    v = values()
    lines = ["// 2^{j/4096}, j = 0..4095, correctly rounded; written by gen_exp2_table.py."]
    for a in range(0, N, 4):
        lines.append("    " + ", ".join(x.hex() for x in v[a:a + 4]) + ",")
    with open(out, "w") as f:
        f.write("\n".join(lines) + "\n")
    return out


if __name__ == "__main__":
    print(main())
