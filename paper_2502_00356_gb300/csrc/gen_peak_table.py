"""Write bk_peak_table.inc: for the quantised shift points s = k/64,
k = 0..1024 (s in [0, 16]), the values the FP32 forms need at the point their
quadrature is centred on:

    cosh s as a double-float (hi, lo), sinh s, e^{-s}

as a float4 initialiser per entry (C hex-float literals).  Each value is
computed with 60-digit decimal arithmetic; hi is the value rounded to a
double and then to a float, lo the rest rounded the same way, so hi + lo
carries cosh s to about 2^-48 relative.  sinh s and e^{-s} are rounded
to float the same way (within an ulp).

    python paper_2502_00356_gb300/csrc/gen_peak_table.py
"""
from __future__ import annotations

import os
import struct
from decimal import Decimal, getcontext

STEPS, K_MAX = 64, 1024


def to_f32(v) -> float:
    """The float nearest to the double nearest to v (as a Python float)."""
    return struct.unpack("f", struct.pack("f", float(v)))[0]


def values() -> list[tuple[float, float, float, float]]:
    getcontext().prec = 60
    out = []
    for k in range(K_MAX + 1):
        s = Decimal(k) / STEPS
        e, r = s.exp(), (-s).exp()
        ch = (e + r) / 2
        hi = to_f32(str(ch))
        lo = to_f32(str(ch - Decimal(hi)))
        out.append((hi, lo, to_f32(str((e - r) / 2)), to_f32(str(r))))
    return out


def literal(x: float) -> str:
    return ("-" if x < 0 else "") + abs(x).hex() + "f" if x != 0 else "0.0f"


def main() -> str:
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "bk_peak_table.inc")
    lines = [f"// (cosh s as hi, lo), sinh s, e^-s at s = k/{STEPS}, k = 0..{K_MAX};"
             " written by gen_peak_table.py."]
    for v in values():
        lines.append("    {" + ", ".join(literal(x) for x in v) + "},")
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")
    return path


if __name__ == "__main__":
    print(main())
