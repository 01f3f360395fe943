"""Write bk_cosh_table.inc: 2 cosh(h) for the quantised quadrature steps
h = 2^e (1 + k/256), e = -12..0, k = 0..255 (3,328 entries, index
(e + 12) * 256 + k), as C hex-float literals.

Each value is computed with 60-digit decimal arithmetic and rounded once to
the nearest double (float() of a decimal string rounds correctly), so every
entry is the correctly rounded 2 cosh(h).  The table backs the step of the
plain form's common node loop (bk_math64.cuh), whose h is rounded up to
8 significand bits.

    python paper_2502_00356_gb300/csrc/gen_cosh_table.py
"""
from __future__ import annotations

import os
from decimal import Decimal, getcontext

E_MIN, E_MAX, BITS = -12, 0, 8


def steps() -> list[Decimal]:
    return [Decimal(2) ** e * (1 + Decimal(k) / (1 << BITS))
            for e in range(E_MIN, E_MAX + 1) for k in range(1 << BITS)]


def values() -> list[float]:
    getcontext().prec = 60
    return [float(str(h.exp() + (-h).exp())) for h in steps()]


def main() -> str:
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "bk_cosh_table.inc")
    v = values()
    lines = [f"// 2 cosh(2^e (1 + k/256)), e = {E_MIN}..{E_MAX}, k = 0..255, correctly rounded;"
             " written by gen_cosh_table.py."]
    for a in range(0, len(v), 4):
        lines.append("    " + ", ".join(x.hex() for x in v[a:a + 4]) + ",")
    with open(out, "w") as f:
        f.write("\n".join(lines) + "\n")
    return out


if __name__ == "__main__":
    print(main())
