"""The constant tables compiled into the CUDA library are exactly what their
committed generator scripts write (so a table can be regenerated and
reviewed from its definition), and each agrees with an independent
evaluation of the function it tabulates."""
import importlib.util
import math
import os
import re

import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_2502_00356_gb300", "csrc")
HEX = re.compile(r"-?0x[0-9a-f]\.[0-9a-f]+p[+-]\d+")


def load(name):
    spec = importlib.util.spec_from_file_location(name, os.path.join(CSRC, name + ".py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def parse(inc):
    with open(os.path.join(CSRC, inc)) as f:
        return [float.fromhex(h) for h in HEX.findall(f.read())]


def ulps(a, b):
    return abs(a - b) / math.ulp(b)


def test_exp2_table_is_the_generators():
    gen = load("gen_exp2_table")
    table = parse("bk_exp2_table.inc")
    assert len(table) == gen.N == 4096
    assert table == gen.values()
    for j in range(0, 4096, 37):  # correctly rounded 2^{j/4096}: within half an ulp of libm's
        assert ulps(table[j], 2.0 ** (j / 4096)) <= 1.0


def test_cosh_step_table_is_the_generators():
    gen = load("gen_cosh_table")
    table = parse("bk_cosh_table.inc")
    assert len(table) == 3328 == len(gen.steps())
    assert table == gen.values()
    for k in range(0, 3328, 13):
        e, j = k // 256 - 12, k % 256
        h = math.ldexp(1.0 + j / 256.0, e)
        assert float(gen.steps()[k]) == h  # the step the kernels index: 2^e (1 + j/256)
        assert ulps(table[k], 2.0 * math.cosh(h)) <= 1.0


def test_rgamma_coefficients_are_the_generators():
    pytest.importorskip("mpmath")
    gen = load("gen_rgamma_coeffs")
    c = gen.coefficients()
    want = [c[k] for k in range(1, gen.K_MAX + 1, 2)] + [-c[k] for k in range(2, gen.K_MAX + 1, 2)]
    assert parse("bk_rgamma_coeffs.inc") == want
    # 1/Gamma(z) from the coefficients at a few points against the library gamma
    for z in (0.1, 0.37, 0.5, -0.45):
        s = sum(ck * z ** k for k, ck in enumerate(c))
        assert abs(s * math.gamma(z) - 1.0) <= 1e-14


def test_peak_table_is_the_generators():
    """kPeakTab: cosh s as hi + lo, sinh s, e^-s at s = k/64."""
    import struct
    gen = load("gen_peak_table")
    with open(os.path.join(CSRC, "bk_peak_table.inc")) as f:
        rows = [line for line in f if line.strip().startswith("{")]
    vals = gen.values()
    assert len(rows) == len(vals) == 1025

    def lit(tok):
        tok = tok.strip().rstrip("f")
        return 0.0 if tok in ("0.0", "-0.0") else float.fromhex(tok)

    f32 = lambda v: struct.unpack("f", struct.pack("f", v))[0]
    ulp32 = lambda v: math.ldexp(1.0, math.frexp(v)[1] - 24)  # float spacing at v
    for k in range(0, 1025, 7):
        got = tuple(lit(t) for t in rows[k].strip().strip("{},").split(","))
        assert got == vals[k]
        s = k / 64.0
        ch = 1.0 + 2.0 * math.sinh(s / 2) ** 2  # cosh s
        assert abs((got[0] + got[1]) - ch) <= 1e-13 * ch
        assert all(v == f32(v) for v in got)  # every entry is a float
        assert abs(got[2] - math.sinh(s)) <= ulp32(math.sinh(s)) if k else got[2] == 0.0
        assert abs(got[3] - math.exp(-s)) <= ulp32(math.exp(-s))
