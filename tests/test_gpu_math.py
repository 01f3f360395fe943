"""The plain form's device math helpers, evaluated as the kernels compute
them (bk_math_probe), against 50-digit decimal references: the table-driven
exponentials of the node loops and of the final normalisation, the table
log, the exact integer-pipe rounding and remainder, the 2 cosh tiers of the
recurrences and the seeded square root.  Each bound is the one the helper's
own documentation states."""
import math
from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np
import pytest

import paper_2502_00356_gb300 as bk

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

getcontext().prec = 50
LN2 = Decimal(2).ln()


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    bk.build()
    return torch.device("cuda:0")


def probe(fn, x, dev):
    out = bk.bk_math_probe(fn, torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64), device=dev))
    torch.cuda.synchronize()
    return out.cpu().numpy()


def rel_err(got, ref):
    return abs(Decimal(float(got)) / ref - 1)


def test_final_exponential(dev):
    rng = np.random.default_rng(61)
    a = np.concatenate([rng.uniform(-707.9, 707.9, 1500), rng.uniform(-20, 20, 500),
                        [0.0, 1e-300, -1e-300, 0.5 * math.log(2) / 4096, 707.99, -707.99]])
    got = probe("exp", a, dev)
    for ai, gi in zip(a, got):
        ref = Decimal(float(ai)).exp()
        # the rounding of u = a 4096/ln2 and of 4096/ln2 itself (1.3e-16 |a|)
        # plus the cubic and two roundings
        assert rel_err(gi, ref) <= Decimal(abs(float(ai)) * 1.5e-16 + 4e-16), (ai, gi)
    # the range-checked path: overflow, deep underflow, NaN
    edge = probe("exp", np.array([709.0, 709.9, -740.0, -746.0, np.nan, np.inf, -np.inf]), dev)
    assert rel_err(edge[0], Decimal(709).exp()) < Decimal(1e-15)
    assert np.isposinf(edge[1]) and edge[3] == 0.0 and np.isnan(edge[4])
    assert 0.0 < edge[2] < 1e-320 and np.isposinf(edge[5]) and edge[6] == 0.0


def test_final_exponential_integer_pipe(dev):
    """The Matern entries' final exponential, e^a = 2^{u/4096} with u = a
    4096/ln 2 formed in table units and evaluated on the integer pipe (the
    cubic in fixed point, the table product as a 64-bit significand)."""
    rng = np.random.default_rng(66)
    a = np.concatenate([rng.uniform(-707.3, 707.3, 1500), rng.uniform(-20, 20, 500),
                        rng.uniform(-1e-3, 1e-3, 200),
                        [0.0, 1e-300, -1e-300, 0.5 * math.log(2) / 4096, -0.5 * math.log(2) / 4096,
                         707.3, -707.3, 1.0, -1.0]])
    got = probe("exp_units", a, dev)
    for ai, gi in zip(a, got):
        ref = Decimal(float(ai)).exp()
        # the rounding of u = a 4096/ln2 (1.3e-16 |a|), the cubic's truncation
        # (3e-18), the fixed-point terms (below 2^-58) and the truncated
        # significand product and renormalisation (below 2^-52)
        assert rel_err(gi, ref) <= Decimal(abs(float(ai)) * 1.5e-16 + 4e-16), (ai, gi)
    edge = probe("exp_units", np.array([709.0, 709.9, -740.0, -746.0, np.nan, np.inf, -np.inf]), dev)
    assert rel_err(edge[0], Decimal(709).exp()) < Decimal(1e-15)
    assert np.isposinf(edge[1]) and edge[3] == 0.0 and np.isnan(edge[4])
    assert 0.0 < edge[2] < 1e-320 and np.isposinf(edge[5]) and edge[6] == 0.0


def test_table_log(dev):
    rng = np.random.default_rng(62)
    a = np.concatenate([np.exp(rng.uniform(-690, 690, 1500)), 1.0 + rng.uniform(-1e-6, 1e-6, 200),
                        [1.0, 2.0, 0.5, 5e-324, 1e-310, 1.7976931348623157e308, 1 + 2**-52]])
    got = probe("log", a, dev)
    for ai, gi in zip(a, got):
        ref = Decimal(float(ai)).ln()
        # ln2/4096 rounded once times |4096 e + j| (below |log a| 2^-53) plus
        # the series and two roundings
        assert abs(Decimal(float(gi)) - ref) <= abs(ref) * Decimal(1.2e-16) + Decimal(3e-19) + \
            abs(ref) * Decimal(2.3e-16), (ai, gi)


def test_table_log_parts(dev):
    """log a as the Matern entries form it: nd = 4096 e + j and log1p(d)
    from the integer pipe (d from a 64-bit significand product, the series in
    fixed point), assembled here by one FMA with ln2/4096."""
    rng = np.random.default_rng(67)
    a = np.concatenate([np.exp(rng.uniform(-690, 690, 1500)), 1.0 + rng.uniform(-1e-6, 1e-6, 200),
                        np.exp(rng.uniform(-12, 5, 500)),
                        [1.0, 2.0, 0.5, 5e-324, 1e-310, 1.7976931348623157e308, 1 + 2**-52,
                         2 - 2**-52, 1.5, 0.1, 14.1]])
    got = probe("log_parts", a, dev)
    for ai, gi in zip(a, got):
        ref = Decimal(float(ai)).ln()
        # ln2/4096 rounded once times |nd| (below |log a| 2^-53) and two
        # roundings, relative; absolute: the table value's own rounding (2^-53
        # in d, as for the FP64 table log), the series' truncation (2e-17) and
        # its fixed-point terms (2^-62)
        assert abs(Decimal(float(gi)) - ref) <= abs(ref) * Decimal(3.5e-16) + Decimal(1.3e-16), (ai, gi)
    # the same values as the FP64 table log to within its rounding
    old = probe("log", a, dev)
    assert np.all(np.abs(got - old) <= 2.3e-16 * np.abs(old) + 2e-17)


def test_node_exponentials(dev):
    rng = np.random.default_rng(63)
    # results stay normal for u >= -1022 * 4096 (4,186,112)
    u = np.concatenate([rng.uniform(-3e5, 3e5, 1500), rng.uniform(-4.18e6, 4.18e6, 300),
                        np.arange(-5, 6) * 0.5, [2**21 + 0.5, -(2**21 + 0.5), 1e-300, 0.0]])
    got = probe("exp2s_node", u, dev)
    for ui, gi in zip(u, got):
        ref = (Decimal(float(ui)) * LN2 / 4096).exp()
        assert rel_err(gi, ref) <= Decimal(3e-14), (ui, gi)  # the quadratic: 2.6e-14
    # the uncentred loop's node exponent D = K x cosh t (x >= 1e-4: D >= 0.59,
    # x cosh t <= 690: D < 4.08e6) truncated to units of 2^-40 (1.7e-16
    # relative in the result) and the fixed-point exponential
    D = np.concatenate([rng.uniform(0.25, 4.08e6, 1500), rng.uniform(0.25, 8, 300),
                        np.arange(1, 12) * 0.5, [0.25, 4096.0, 4096.5, 2**21 + 0.5, 4.08e6]])
    got = probe("exp2s_neg", D, dev)
    for di, gi in zip(D, got):
        ref = (-Decimal(float(di)) * LN2 / 4096).exp()
        assert rel_err(gi, ref) <= Decimal(3e-14), (di, gi)


def test_fixed_point_node_exponential(dev):
    """The node loop's exponential of a signed fixed-point exponent U = D -
    G (units of 2^-40), over the loop's range: results in [2^-1000, 2^1000],
    halves rounding up, the renormalisation at both ends of the table."""
    rng = np.random.default_rng(68)
    a = np.concatenate([rng.uniform(-4.09e6, 4.09e6, 1500), rng.uniform(-8, 8, 500),
                        np.arange(-9, 10) * 0.5, np.arange(-3, 4) * 4096.0,
                        [2.0**-41, -2.0**-41, 3 * 2.0**-41, 1e-20, 4095.5, -4095.5]])
    got = probe("exp2s_fix", a, dev)
    for ai, gi in zip(a, got):
        u40 = round(Fraction(float(ai)) * 2**40)  # the probe's rounding: to nearest, ties to even
        ref = (-Decimal(u40) / Decimal(2**40) * LN2 / 4096).exp()
        assert rel_err(gi, ref) <= Decimal(3e-14), (ai, gi)  # the quadratic: 2.6e-14


def test_fixed_point_geometric_factor(dev):
    """1 + W_j from W_j in units of 2^-63 (truncated) rounded to a double, and
    the ratio r in units of 2^-64 (truncated, clamped below 2^64)."""
    rng = np.random.default_rng(69)
    w = np.concatenate([rng.uniform(0, 1, 2000), rng.uniform(0, 1e-10, 200),
                        [0.0, 1.0, 0.5, 0.25, 1 - 2**-53, 2**-60, 2**-64, 1e-300]])
    got = probe("one_plus_w", w, dev)
    for wi, gi in zip(w, got):
        assert abs(Fraction(float(gi)) - 1 - Fraction(float(wi))) <= Fraction(1, 2**53) + Fraction(1, 2**63), (wi, gi)
    assert got[-8] == 1.0 and got[-7] == 2.0 and got[-6] == 1.5 and got[-5] == 1.25
    r = np.concatenate([rng.uniform(0, 1, 2000), [0.0, 1.0, 0.5, 1 - 2**-53, 2**-64, 2**-70, 1e-300]])
    got = probe("fix64", r, dev)
    for ri, gi in zip(r, got):
        q = min(math.floor(Fraction(float(ri)) * 2**64), 2**64 - 1)
        assert gi == float(q) * 2.0**-64, (ri, gi)


def test_integer_rounding_is_exact(dev):
    rng = np.random.default_rng(64)
    v = np.concatenate([rng.uniform(0, 2**22 - 1, 4000), rng.uniform(0, 4, 1000),
                        np.floor(rng.uniform(0, 2**22 - 1, 1000)) + 0.5,
                        np.nextafter(np.floor(rng.uniform(1, 2**22 - 1, 500)) + 0.5, 0),
                        [0.0, 5e-324, 1e-300, 0.25, 0.5, 0.75, 1.0, 2**22 - 0.5]])
    got = probe("round_rem", v, dev)
    for vi, (m, r) in zip(v, got):
        want_m = math.floor(Fraction(float(vi)) + Fraction(1, 2))  # halves round up
        assert m == want_m, (vi, m, want_m)
        assert Fraction(float(r)) == Fraction(float(vi)) - want_m, (vi, r)


def test_two_cosh_tiers(dev):
    rng = np.random.default_rng(65)
    v = np.concatenate([rng.uniform(0, 0.35, 700), rng.uniform(0.35, 0.75, 700),
                        rng.uniform(0.75, 20, 300),
                        [0.0, 1e-10, 0.35, np.nextafter(0.35, 1), 0.75, np.nextafter(0.75, 1)]])
    for order in (v, np.sort(v)):  # mixed tiers in a warp, and warp-uniform tiers
        got = probe("two_cosh", order, dev)
        for vi, gi in zip(order, got):
            x = Decimal(float(vi))
            ref = x.exp() + (-x).exp()
            # series tiers: about an ulp; the exponential path: a few
            bound = 3.4e-16 if vi <= 0.75 else 1e-15
            assert rel_err(gi, ref) <= Decimal(bound), (vi, gi)


def test_seeded_square_root(dev):
    rng = np.random.default_rng(66)
    a = np.concatenate([np.exp(rng.uniform(-80, 80, 2000)),
                        [1e-300, 5e-324, 1e300, 2.0, 0.5, 1.0, 4.0, 2.0**-120, 2.0**120]])
    got = probe("sqrt", a, dev)
    want = np.sqrt(a)
    ulp = np.spacing(want)
    assert np.all(np.abs(got - want) <= ulp), np.max(np.abs(got - want) / ulp)


def test_integer_square_root(dev):
    """The Matern entries' square root on the integer pipe (an FP32 seed,
    one correction from an exact 64-bit residual, one from an exact 128-bit
    residual): within an ulp on the whole normal range, both exponent
    parities and the significand ends."""
    rng = np.random.default_rng(68)
    a = np.concatenate([np.exp(rng.uniform(-700, 700, 3000)), np.exp(rng.uniform(-5, 5, 2000)),
                        (1 + rng.uniform(0, 1e-12, 300)) * 2.0 ** rng.integers(-60, 60, 300),
                        (4 - rng.uniform(0, 1e-12, 300)) * 2.0 ** rng.integers(-60, 60, 300),
                        [2.0**-1022, 1.7976931348623157e308, 2.0, 0.5, 1.0, 4.0, 3.9999999999999996,
                         1.0000000000000002, 5e-324, 1e-310]])
    got = probe("sqrt_int", a, dev)
    want = np.sqrt(a)
    ulp = np.spacing(want)
    assert np.all(np.abs(got - want) <= ulp), np.max(np.abs(got - want) / ulp)


def test_setup_exponential(dev):
    rng = np.random.default_rng(67)
    a = np.concatenate([rng.uniform(-707, 707, 1000), rng.uniform(-1, 1, 300), [0.0]])
    got = probe("exp_acc", a, dev)
    for ai, gi in zip(a, got):
        assert rel_err(gi, Decimal(float(ai)).exp()) <= Decimal(4.5e-16), (ai, gi)
