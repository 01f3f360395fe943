// FP32 precision form of the integrand (Sec. IV-B): window search and
// quadrature in FP32 on the FMA and MUFU pipes, with FP64 kept for the
// search outside the stated region, for cosh(t_max) and for the log-domain
// normalisation.  Window rule with eps = 2^-23 (the FP32 machine epsilon).
#pragma once

#include "bk_math64.cuh"

namespace bk {

constexpr float kLog2ef = 1.44269504f;
constexpr float kLn2f = 0.693147181f;
constexpr float kLogInvEps32 = 15.9423857f;  // -log(2^-23)
// ln(2 / tol) with tol = 2e-7 for the strip-bound node count of the FP32 form.
constexpr float kF32Log2OverTol = 16.1181f;
constexpr int kF32MaxNodes = 256;

// 2^v and 1/v on the MUFU unit (ex2.approx / rcp.approx, about 2 ulp).
__device__ __forceinline__ float mufu_ex2(float v) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}
__device__ __forceinline__ float mufu_rcp(float v) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}
__device__ __forceinline__ float mufu_lg2(float v) {
  float r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}
__device__ __forceinline__ float exp_f32(float a) { return mufu_ex2(a * kLog2ef); }
// a / b from the MUFU reciprocal (about 2 ulp; moderate normal b), for
// Newton steps, first guesses and low-order corrections, where a rounded
// quotient is not needed (an IEEE division is a ~10-instruction sequence).
__device__ __forceinline__ float fast_div(float a, float b) { return a * mufu_rcp(b); }
// sqrt v for v > 0 from the MUFU reciprocal square root (about 2 ulp), where
// the root is a first guess or is corrected afterwards.
__device__ __forceinline__ float fast_sqrt_pos(float v) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return v * r;
}

// sinh with small relative error for all |y| <= ~80: the odd Taylor
// polynomial to y^7 below 0.35 (truncation < 1e-9 relative), (e^y - e^-y)/2
// above (cancellation costs at most a factor coth(0.35) ~ 3 in ulps).
__device__ __forceinline__ float sinh_f32(float y) {
  const float ay = fabsf(y), y2 = y * y;
  const float poly = y * fmaf(y2, fmaf(y2, fmaf(y2, 1.0f / 5040.0f, 1.0f / 120.0f), 1.0f / 6.0f), 1.0f);
  const float e = mufu_ex2(ay * kLog2ef);
  const float big = copysignf(0.5f * (e - mufu_rcp(e)), y);
  return ay < 0.35f ? poly : big;
}

struct Window32 {
  float ts, t0, t1;
  float cs;  // cosh ts (window_f32 only)
};

// a3 in FP32: the same bracketed Newton as peak_f64 (g' concave on t > 0,
// negative at asinh(nu/x)); the right end is inflated slightly so that the
// FP32 value stays right of the root.
__device__ __forceinline__ float peak_f32(float x, float nu, Tally& tl) {
  const float nu2 = nu * nu;
  if (!(nu2 > x)) return 0.0f;
  const float q = fast_div(nu, x);
  float hi = kLn2f * mufu_lg2(q + fast_sqrt_pos(fmaf(q, q, 1.0f)));
  hi = fmaf(hi, 1.0e-4f, hi) + 1.0e-6f;
  float lo = 0.0f;
  const float tc2 = (nu2 - x) / fmaf(nu2 * nu2, 1.0f / 3.0f, x * (1.0f / 6.0f));
  float t = (tc2 < hi * hi) ? fast_sqrt_pos(tc2) : hi;
  for (int it = 0; it < 40; ++it) {
    ++tl.peak_iters;
    const float e = mufu_ex2(t * kLog2ef);
    const float ch = 0.5f * (e + mufu_rcp(e));
    const float sh = sinh_f32(t);
    const float w = mufu_ex2(-2.0f * kLog2ef * nu * t);
    const float r1 = mufu_rcp(1.0f + w);
    const float gp = fmaf(nu * (1.0f - w), r1, -x * sh);
    const float gpp = fmaf(nu2 * 4.0f * w, r1 * r1, -x * ch);
    if (gp > 0.0f) lo = t; else hi = t;
    float tn;
    if (gpp < 0.0f) {
      tn = t - fast_div(gp, gpp);
      if (tn > hi) tn = hi;
      if (!(tn > lo)) tn = 0.5f * (lo + hi);
    } else {
      tn = 0.5f * (lo + hi);
    }
    const float dt = tn - t;
    t = tn;
    if (fabsf(dt) <= 2e-6f * t) break;
  }
  return t;
}

// cosh t - cosh ts = 2 sinh((t + ts)/2) sinh((t - ts)/2): no cancellation.
__device__ __forceinline__ float dcosh_f32(float t, float ts) {
  return 2.0f * sinh_f32(0.5f * (t + ts)) * sinh_f32(0.5f * (t - ts));
}

// a4 in FP32 with the bound F of window_f64 (see there), L = -log eps
// (2^-23 for the FP32 forms; 2^-52 where the plain form takes its FP64
// Newton starts from here).
__device__ __forceinline__ Window32 window_f32(float x, float nu, float L, Tally& tl) {
  Window32 w;
  const float ts = peak_f32(x, nu, tl);
  w.ts = ts;
  const float es = mufu_ex2(ts * kLog2ef);
  const float cs = 0.5f * (es + mufu_rcp(es));
  w.cs = cs;
  const float ss = sinh_f32(ts);
  {
    const float a = x * cs, b = nu - x * ss;
    float t = ts + fast_div(b + fast_sqrt_pos(fmaf(b, b, 2.0f * a * L)), a);
    t = fmaf(t, 1.0e-4f, t);
    float tb = kLn2f * mufu_lg2(fast_div(2.0f * (L + a + nu * t), x));
    tb = fmaf(tb, 1.0e-4f, tb);
    if (tb < t) t = tb;
    for (int it = 0; it < 40; ++it) {
      ++tl.iters;
      const float F = fmaf(nu, t - ts, -x * dcosh_f32(t, ts)) + L;
      const float Fp = fmaf(-x, sinh_f32(t), nu);
      const float dt = fast_div(F, Fp);
      t -= dt;
      if (fabsf(dt) <= 1e-5f * t) break;
    }
    w.t1 = t;
  }
  w.t0 = 0.0f;
  if (ts > 0.0f) {
    const float Lp = L + kLn2f;
    const float G0 = fmaf(-nu, ts, x * (cs - 1.0f)) + Lp;
    if (G0 < 0.0f) {
      float t = fmaxf(0.0f, ts - fast_div(Lp, nu));
      for (int it = 0; it < 40; ++it) {
        ++tl.iters;
        const float G = fmaf(nu, t - ts, -x * dcosh_f32(t, ts)) + Lp;
        const float Gp = fmaf(-x, sinh_f32(t), nu);
        float tn = t - fast_div(G, Gp);
        if (tn < 0.0f) tn = 0.0f;
        const bool done = fabsf(tn - t) <= 1e-5f * fmaxf(tn, 1e-3f);
        t = tn;
        if (done) break;
      }
      w.t0 = t;
    }
  }
  return w;
}

// e^y - 1 and e^{-y} - 1 together, both with small relative error:
// em = e^y - 1 from its Taylor polynomial to y^7 for |y| < 0.35 (truncation
// < 2e-8 relative), else E - 1 with E = e^y on the MUFU (exact for E in [1/2, 2] by
// Sterbenz, no cancellation beyond a factor ~3 in ulps elsewhere), and
// e^{-y} - 1 = -em / (1 + em) from one rcp (1 + em reproduces E there).  One
// polynomial, one ex2 and one rcp for both.
__device__ __forceinline__ void expm1_pm_f32(float y, float& em, float& emn) {
  const float p =
      y * fmaf(y, fmaf(y, fmaf(y, fmaf(y, fmaf(y, fmaf(y, 1.0f / 5040.0f, 1.0f / 720.0f),
                                               1.0f / 120.0f), 1.0f / 24.0f), 1.0f / 6.0f),
                   0.5f), 1.0f);
  const float e = mufu_ex2(y * kLog2ef);
  em = fabsf(y) < 0.35f ? p : e - 1.0f;
  emn = -em * mufu_rcp(1.0f + em);
}

// The searched window of the FP32 form: FP32 search inside x in [1e-4, 1e4],
// nu <= 40, the FP64 search (with the FP32 eps) outside, where FP32 sinh /
// cosh of the window ends lose too much.  x is the FP32 argument, x64 the
// full one, produced by x64_of() only on the FP64 path (a conversion between
// FP64 and FP32 costs an FP64-pipe slot on this GPU, like an FMA).
template <class X64>
__device__ __forceinline__ Window32 search_window_f32(float x, X64 x64_of, float nu,
                                                     const double* __restrict__ tab, Tally& tl) {
  Window32 w;
  if (x >= 1e-4f && x <= 1e4f && nu <= 40.0f) {
    w = window_f32(x, nu, kLogInvEps32, tl);
  } else {
    const Window64 w64 = window_f64(x64_of(), (double)nu, (double)kLogInvEps32, tab, tl);
    w.ts = (float)w64.ts;
    w.t0 = (float)w64.t0;
    w.t1 = (float)w64.t1;
  }
  return w;
}

// e^t for |t| < ~80 in FP32 without a large exponential argument:
// t = k ln2 + r with ln 2 split into 16 + remaining bits (k ln2_hi exact for
// |k| < 2^8) and e^{+-r} from the Taylor polynomial of degree 7 on
// |r| <= ln2/2 (truncation < 6e-9 relative); returns 2^k e^r and 2^-k e^-r.
__device__ __forceinline__ float exp_taylor7_f32(float r) {
  return fmaf(r, fmaf(r, fmaf(r, fmaf(r, fmaf(r, fmaf(r, fmaf(r, 1.0f / 5040.0f, 1.0f / 720.0f),
                                                          1.0f / 120.0f), 1.0f / 24.0f),
                                            1.0f / 6.0f), 0.5f), 1.0f), 1.0f);
}
__device__ __forceinline__ void exp_pm_f32(float t, float& ep, float& em) {
  const float kf = rintf(t * kLog2ef);
  const int k = (int)kf;
  float r = fmaf(-kf, 0.693145751953125f, t);
  r = fmaf(-kf, 1.428606765330187e-06f, r);
  ep = exp_taylor7_f32(r) * __int_as_float((127 + k) << 23);
  em = exp_taylor7_f32(-r) * __int_as_float((127 - k) << 23);
}

// ---------------------------------------------------------------------------
// Double-float arithmetic (an unevaluated sum hi + lo of two floats, ~44
// significant bits) from error-free transformations (Knuth's two-sum, the FMA
// two-product), so that the FP32 forms can keep distances and log-domain sums
// accurate without FP64 instructions.
struct DF {
  float hi, lo;
};

__device__ __forceinline__ DF two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return DF{s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ DF quick_two_sum(float a, float b) {  // |a| >= |b|
  const float s = a + b;
  return DF{s, b - (s - a)};
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
  const DF s = two_sum(a.hi, b.hi);
  return quick_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ DF df_add_f(DF a, float b) {
  const DF s = two_sum(a.hi, b);
  return quick_two_sum(s.hi, s.lo + a.lo);
}
__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const float p = a.hi * b.hi;
  const float e = fmaf(a.hi, b.hi, -p);
  return quick_two_sum(p, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e)));
}
__device__ __forceinline__ DF df_mul_f(DF a, float b) {
  const float p = a.hi * b;
  const float e = fmaf(a.hi, b, -p);
  return quick_two_sum(p, fmaf(a.lo, b, e));
}
__device__ __forceinline__ DF df_neg(DF a) { return DF{-a.hi, -a.lo}; }

// ln 2 as a double-float, and split for range reduction (k ln2_hi exact for
// |k| < 2^8): ln2_hi has 16 significant bits.
constexpr float kLn2HiF = 0.693145751953125f;
constexpr float kLn2LoF = 1.428606765330187e-06f;
constexpr float kLn2DfHi = 0.693147182464599609375f;  // float nearest to ln 2
constexpr float kLn2DfLo = -1.904654323148236e-09f;   // ln 2 - kLn2DfHi

// log of a double-float z > 0 (normal floats): z = 2^e m, m in [sqrt(1/2),
// sqrt(2)), log m = 2 atanh(s), s = (m - 1)/(m + 1) from its series to s^13
// (truncation < 1e-9 absolute), plus e ln 2 and the first-order lo term.
__device__ __forceinline__ DF df_log(DF z) {
  // z.hi = m 2^e with m in [0.5, 1), from the bits (z.hi is a positive normal float)
  const int bits = __float_as_int(z.hi);
  int e = ((bits >> 23) & 0xff) - 126;
  float m = __int_as_float((bits & 0x007fffff) | 0x3f000000);
  if (m < 0.70710678f) {
    m *= 2.0f;
    e -= 1;
  }
  // s = (m - 1)/(m + 1) from the MUFU reciprocal and one Newton correction
  const float rp = mufu_rcp(m + 1.0f);
  float s = (m - 1.0f) * rp;
  s = fmaf(fmaf(-s, m + 1.0f, m - 1.0f), rp, s);
  const float s2 = s * s;
  const float q = fmaf(s2, fmaf(s2, fmaf(s2, fmaf(s2, fmaf(s2, fmaf(s2, 1.0f / 13.0f, 1.0f / 11.0f),
                                                          1.0f / 9.0f), 1.0f / 7.0f), 1.0f / 5.0f),
                                1.0f / 3.0f), 1.0f);
  const float lm = 2.0f * s * q;
  const float ef = (float)e;
  DF r = quick_two_sum(ef * kLn2HiF, fmaf(ef, kLn2LoF, lm));  // e ln2_hi exact
  return df_add_f(r, fast_div(z.lo, z.hi));
}

// Distance as a double-float from the double-float coordinates: the hi-part
// differences are made exact with two-sum, squares with the FMA two-product.
// r.hi == 0 exactly when both FP64 coordinates agree.
__device__ __forceinline__ DF df_hypot_diff(float axh, float axl, float ayh, float ayl, float bxh,
                                            float bxl, float byh, float byl) {
  DF dx = two_sum(bxh, -axh);
  dx = two_sum(dx.hi, dx.lo + (bxl - axl));  // renormalise: the hi parts may cancel
  DF dy = two_sum(byh, -ayh);
  dy = two_sum(dy.hi, dy.lo + (byl - ayl));
  DF px = DF{dx.hi * dx.hi, 0.0f};
  px.lo = fmaf(dx.hi, dx.hi, -px.hi);
  px.lo = fmaf(2.0f * dx.hi, dx.lo, px.lo);
  DF py = DF{dy.hi * dy.hi, 0.0f};
  py.lo = fmaf(dy.hi, dy.hi, -py.hi);
  py.lo = fmaf(2.0f * dy.hi, dy.lo, py.lo);
  const DF r2 = df_add(px, py);
  if (r2.hi == 0.0f && dx.hi == 0.0f && dy.hi == 0.0f && dx.lo == 0.0f && dy.lo == 0.0f)
    return DF{0.0f, 0.0f};
  const float rh = fast_sqrt_pos(r2.hi);  // its error is in the lo term below
  return DF{rh, (fmaf(-rh, rh, r2.hi) + r2.lo) * fast_div(0.5f, rh)};
}

// e^a * s for a double-float a with FP32 accuracy, as a float (the FP32
// output case; underflows to 0 below the float range and overflows to
// s * inf above it, where the two power-of-two factors would leave the
// exponent field).
__device__ __forceinline__ float df_exp_times(DF a, float s) {
  if (a.hi < -103.0f) return 0.0f;
  if (a.hi > 100.0f) return s * __int_as_float(0x7f800000);
  const float kf = rintf(a.hi * kLog2ef);
  float r = fmaf(-kf, kLn2HiF, a.hi);
  r = fmaf(-kf, kLn2LoF, r) + a.lo;
  const int k = (int)kf;
  const int k1 = k >> 1;  // split so both factors stay normal floats
  return (exp_taylor7_f32(r) * s) * __int_as_float((127 + k1) << 23) *
         __int_as_float((127 + k - k1) << 23);
}

// ---------------------------------------------------------------------------
// Conversions and functions for the FP32 forms without FP64 instructions.
// (On this GPU FP64 <-> FP32 conversions run at the FP64 rate, 2 per clock
// and SM, like an FMA; integer <-> FP32 conversions run on the MUFU pipe.)

// A double as a double-float by integer operations: hi = v rounded to 24
// significant bits, lo = the rest rounded to float (|v - hi - lo| <= 2^-48
// |v|).  ok = false (and the caller takes an FP64 path) outside
// |v| in [2^-70, 2^100] or for zero, denormal, infinite and NaN v.
__device__ __forceinline__ DF df_from_bits(double v, bool& ok) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int e = (int)((b >> 52) & 0x7ff) - 1023;
  ok = (e >= -70 && e <= 100);
  const unsigned long long m = (b & 0xfffffffffffffull) | (1ull << 52);
  unsigned long long q = (m + (1ull << 28)) >> 29;  // 24 significant bits (25 on carry)
  const long long r = (long long)m - (long long)(q << 29);  // |r| <= 2^28
  int eh = e;
  if (q >> 24) {
    q >>= 1;
    ++eh;
  }
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const float hi = __int_as_float((int)(sign | ((unsigned)(eh + 127) << 23) | ((unsigned)q & 0x7fffffu)));
  // r 2^(e-52): the exponent can fall below the float range; split the scale
  const int s1 = (e - 52) / 2, s2 = (e - 52) - s1;
  const float lo = (float)r * __int_as_float((s1 + 127) << 23) * __int_as_float((s2 + 127) << 23);
  return DF{hi, __int_as_float(__float_as_int(lo) ^ (int)sign)};
}

// e^t as a double-float, ~2e-14 relative for t in [-70, 88] (below -70 the
// low part leaves the float range and the result has FP32 accuracy): t = k ln 2 + r
// with ln 2 split into 16 + 24 + 24 bits (k ln2_hi exact for |k| < 128, the
// second product kept exact by the FMA), |r| <= ln2/2, e^r by its Taylor
// series to r^11 (truncation < 7e-15) in double-float with double-float
// coefficients up to 1/720.
constexpr float kLn2Lo2F = 5.4979231e-14f;  // ln 2 - kLn2HiF - kLn2LoF (to float)
__device__ __forceinline__ DF df_exp(float t) {
  const float kf = rintf(t * kLog2ef);
  const float r0 = fmaf(-kf, kLn2HiF, t);            // exact
  const float p1 = kf * kLn2LoF;
  const float p1e = fmaf(kf, kLn2LoF, -p1);
  DF r = two_sum(r0, -p1);
  r = df_add_f(r, -fmaf(kf, kLn2Lo2F, p1e));
  float c = 1.0f / 39916800.0f;                        // 1/11!
  c = fmaf(c, r.hi, 1.0f / 3628800.0f);
  c = fmaf(c, r.hi, 1.0f / 362880.0f);
  c = fmaf(c, r.hi, 1.0f / 40320.0f);
  c = fmaf(c, r.hi, 1.0f / 5040.0f);                   // tail to r^7 in FP32 (its error < 1e-14)
  DF p = df_add(df_mul_f(r, c), DF{0x1.6c16c2p-10f, -0x1.27d27ep-35f});  // + 1/720
  p = df_add(df_mul(p, r), DF{0x1.111112p-7f, -0x1.dddddep-32f});          // + 1/120
  p = df_add(df_mul(p, r), DF{0x1.555556p-5f, -0x1.555556p-30f});         // + 1/24
  p = df_add(df_mul(p, r), DF{0x1.555556p-3f, -0x1.555556p-28f});         // + 1/6
  p = df_add_f(df_mul(p, r), 0.5f);
  p = df_add_f(df_mul(p, r), 1.0f);
  p = df_add_f(df_mul(p, r), 1.0f);
  const int k = (int)kf;
  const float sc = __int_as_float((127 + k) << 23);
  return DF{p.hi * sc, p.lo * sc};
}

// 1 / a for a double-float a > 0 (one Newton step on the FP32 reciprocal).
__device__ __forceinline__ DF df_rcp(DF a) {
  const float y = 1.0f / a.hi;
  const DF e = df_add_f(df_neg(df_mul_f(a, y)), 1.0f);  // 1 - a y
  return df_add_f(df_mul_f(e, y), y);
}

// cosh t - 1 for t >= 0 as a double-float (~1e-13 relative): for t < 1/2
// (t^2/2)(1 + (t^2/12) q(t^2)) with q's tail in FP32, else (e^t + e^-t)/2 - 1.
__device__ __forceinline__ DF df_cosh_m1(float t) {
  if (t < 0.5f) {
    // cosh t - 1 = (y/2)(1 + (y/12)(1 + y q(y))), y = t^2,
    // q = 1/30 + y/1680 + y^2/151200 (next term below 1e-9 of q)
    const DF y = DF{t * t, fmaf(t, t, -(t * t))};  // t^2 exactly
    const float q = fmaf(y.hi, fmaf(y.hi, 1.0f / 151200.0f, 1.0f / 1680.0f), 1.0f / 30.0f);
    const DF inner = df_add_f(df_mul_f(y, q), 1.0f);
    const DF corr = df_mul(df_mul(inner, y), DF{0x1.555556p-4f, -0x1.555556p-29f});  // / 12
    return df_mul(DF{0.5f * y.hi, 0.5f * y.lo}, df_add_f(corr, 1.0f));
  }
  const DF e = df_exp(t);
  const DF c = df_add(e, df_rcp(e));  // 2 cosh t
  return df_add_f(DF{0.5f * c.hi, 0.5f * c.lo}, -1.0f);
}

// The FP32 quadrature of one evaluation on a given window: h S, the shift
// point s its terms are centred on and cosh s - 1 there (NaN h S when the
// node bound is exceeded).
struct Quad32 {
  float hS;
  float ts;    // the shift point s (the window's peak rounded to the grid of kPeakTab)
  DF ch;       // cosh s as a double-float
  float amax;  // largest node exponent g(t_j) - g(s) (up to the e^{-2 nu t} factor)
};

// The shift points of the FP32 quadrature: the peak ts rounded to the grid
// k/64 (k <= 1024), where kPeakTab holds cosh s (double-float), sinh s and
// e^{-s} (gen_peak_table.py).  Any shift point is exact (it scales the
// terms, and log K adds it back); one within 1/128 of the peak keeps the
// largest scaled term at e^{|g''| / 32768} ~ 1.  The table takes the place
// of per-evaluation FP32 exponentials of ts and of a double-float cosh ts - 1.
constexpr int kPeakTabSize = 1025;
static __device__ const float4 kPeakTab[kPeakTabSize] = {
#include "bk_peak_table.inc"
};

// s, cosh s, D = x sinh s and B = x e^{-s}/2 for the peak ts: from the
// table on its grid, else (ts >= 16, or not a number) at ts itself from FP32
// and double-float exponentials.
__device__ __forceinline__ void shift_f32(float x, float ts, float& s, DF& ch, float& B,
                                          float& D) {
  if (ts >= 0.0f && ts < 16.0f) {
    const float r = rintf(ts * 64.0f);
    s = r * 0.015625f;
    const float4 e = __ldg(&kPeakTab[__float2int_rn(r)]);
    ch = DF{e.x, e.y};
    D = x * e.z;
    B = 0.5f * x * e.w;
  } else {
    s = ts;
    float ep, emx;
    exp_pm_f32(ts, ep, emx);
    B = 0.5f * x * emx;
    D = 0.5f * x * (ep - emx);  // no cancellation at ts >= 16
    ch = df_add_f(df_cosh_m1(ts), 1.0f);
  }
}

// ---------------------------------------------------------------------------
// The FP32 quadrature (a6).  The scaled trapezoid sum, with the weights of
// Eq. (refined):
//   S = sum_j c_j exp(a_j) (1 + e^{-2 nu t_j}),  c_0 = c_N = 1/2,
//   a_j = nu tau_j - x (cosh t_j - cosh s),  tau_j = t_j - s = (t0 - s) + j h,
// centred on the shift point s (a grid point next to the peak, see
// shift_f32; any s is exact, it only scales the terms).  Peak-relative nodes
// keep nu tau_j and the spacing accurate near the peak.  The cosh difference
// is written so that no large argument enters an FP32 exponential and
// nothing cancels, for every s >= 0 alike: with em = e^tau - 1 and
// emn = e^{-tau} - 1 (so em emn = -(em + emn)), D = x sinh s and
// B = x e^{-s}/2,
//   x (cosh t - cosh s) = x e^s/2 em + B emn = em (D - B emn),
// where D - B emn >= D/2 > 0 for t >= 0 (tau >= -s).  e^{-2 nu t_j} follows
// a geometric recurrence; the sums are Kahan-compensated.  The order enters
// as nu_hi + nu_lo (the FP64 order split into two floats): rounding nu itself
// to FP32 would integrate K of a neighbouring order, off by
// ulp(nu) d(log K)/d nu ~ ulp(nu) ln(2 nu/x), ~1e-5 at x ~ 1e-3, nu ~ 18.
//
// The node loop can be split over L lanes (L = 1, 2, 4, 8) for evaluations
// whose node counts differ from lane to lane (random (x, nu) pairs).  Every
// lane first prepares its own evaluation's job (window, node count, shift
// point); the warp then takes the 32 jobs in L passes of 32/L jobs, each job
// on a group of L consecutive lanes: lane r of a group evaluates nodes
// j = r, r + L, ..., and the group adds its partial sums by a compensated
// butterfly (__shfl_xor_sync, two-sum in FP32).  With L = 1 every lane runs
// its own job and no lane waits for another (no shuffle).

// One evaluation's quadrature job: nodes t_j = t0 + j h, j = 0..N, centred on
// s (N < 0: no job).
struct Job32 {
  float t0, h, s, nu, nu_lo, B, D;
  int N;
};

__device__ __forceinline__ Job32 no_job32() { return Job32{0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, -1}; }

// The job of quad_f32 on window w; q receives the shift point (q.hS is NaN and
// the job empty when the node bound is exceeded).
__device__ __forceinline__ Job32 job_f32(float x, float nu, float nu_lo, const Window32& w,
                                         Quad32& q, Tally& tl) {
  const int N = strip_node_count(x, nu, w.t1 - w.t0, kF32Log2OverTol, kF32MaxNodes);
  q.amax = 0.0f;
  if (N > kF32MaxNodes) {
    ++tl.fail;
    q.hS = __int_as_float(0x7fc00000);
    q.ts = w.ts;
    q.ch = DF{1.0f, 0.0f};
    return no_job32();
  }
  Job32 jb;
  shift_f32(x, w.ts, q.ts, q.ch, jb.B, jb.D);
  jb.t0 = w.t0;
  jb.h = fast_div(w.t1 - w.t0, (float)N);
  jb.s = q.ts;
  jb.nu = nu;
  jb.nu_lo = nu_lo;
  jb.N = N;
  tl.nodes += N + 1;
  return jb;
}

// One node's term of the FP32 sum (the node arithmetic above): the scaled
// integrand at tau = t - s times (1 + e^{-2 nu t}) (W = e^{-2 nu t}); am
// receives the largest exponent when kAmax.
template <bool kAmax>
__device__ __forceinline__ float node_f32(const Job32& jb, float tau, float W, float& am) {
  float em, emn;
  expm1_pm_f32(tau, em, emn);
  const float a = fmaf(jb.nu, tau, fmaf(jb.nu_lo, tau, -em * fmaf(-jb.B, emn, jb.D)));
  if constexpr (kAmax) am = fmaxf(am, a);
  const float f = exp_f32(a);
  return fmaf(f, W, f);
}

// Runs the 32 jobs of the warp on groups of L lanes; for L > 1 every lane of
// the warp must call it (L = 1 runs this lane's job alone).  Each lane
// receives h S and, when kAmax, the largest node exponent of its own job (0
// and -3e38 for no job).  A lane's first node is taken before its loop and
// its last node's term kept, so that the end weights 1/2 need no test per
// node.
template <int L, bool kAmax = true>
__device__ __forceinline__ void coop_trapezoid_f32(const Job32& my, float& hS, float& amax) {
  static_assert(L == 1 || L == 2 || L == 4 || L == 8, "lanes per job");
  constexpr int G = 32 / L;  // jobs per pass
  constexpr unsigned kAll = 0xffffffffu;
  const int lane = threadIdx.x & 31, g = lane / L, r = lane - g * L;
  hS = 0.0f;
  amax = -3.0e38f;
#pragma unroll 1
  for (int p = 0; p < L; ++p) {
    Job32 jb = my;
    if constexpr (L > 1) {
      const int owner = p * G + g;
      jb.t0 = __shfl_sync(kAll, my.t0, owner);
      jb.h = __shfl_sync(kAll, my.h, owner);
      jb.s = __shfl_sync(kAll, my.s, owner);
      jb.nu = __shfl_sync(kAll, my.nu, owner);
      jb.nu_lo = __shfl_sync(kAll, my.nu_lo, owner);
      jb.B = __shfl_sync(kAll, my.B, owner);
      jb.D = __shfl_sync(kAll, my.D, owner);
      jb.N = __shfl_sync(kAll, my.N, owner);
    }
    float S = 0.0f, c = 0.0f, ends = 0.0f, am = -3.0e38f;
    if (r <= jb.N) {
      const float tau0 = jb.t0 - jb.s;
      const float l2n = -2.0f * kLog2ef * jb.nu;
      float W = mufu_ex2(l2n * fmaf((float)r, jb.h, jb.t0));  // e^{-2 nu t_r}
      const float rho = mufu_ex2(l2n * ((float)L * jb.h));    // e^{-2 nu L h}
      float f = node_f32<kAmax>(jb, fmaf((float)r, jb.h, tau0), W, am);
      const float f_first = f;
      S = f;
      float jf = (float)(r + L);
#pragma unroll 2
      for (int j = r + L; j <= jb.N; j += L, jf += (float)L) {
        W *= rho;
        f = node_f32<kAmax>(jb, fmaf(jf, jb.h, tau0), W, am);
        const float y = f - c;  // Kahan
        const float s2 = S + y;
        c = (s2 - S) - y;
        S = s2;
      }
      // end weights 1/2: node 0 is this lane's first if r = 0; node N its
      // last if N - r is a multiple of L
      ends = (r == 0 ? f_first : 0.0f) + (((jb.N - r) & (L - 1)) == 0 ? f : 0.0f);
    }
    // this lane's part as hi + lo, then the group's butterfly
    DF v = two_sum(S, -c);
    v.lo = fmaf(-0.5f, ends, v.lo);
#pragma unroll
    for (int o = 1; o < L; o <<= 1) {
      const float oh = __shfl_xor_sync(kAll, v.hi, o), ol = __shfl_xor_sync(kAll, v.lo, o);
      const DF t = two_sum(v.hi, oh);
      v = quick_two_sum(t.hi, t.lo + (v.lo + ol));
      if constexpr (kAmax) am = fmaxf(am, __shfl_xor_sync(kAll, am, o));
    }
    const float tot = jb.h * (v.hi + v.lo);
    if constexpr (L == 1) {
      hS = tot;
      amax = am;
    } else {
      // the owner of group g' in pass p is lane p G + g'; group g' holds its sum
      const float got = __shfl_sync(kAll, tot, (lane % G) * L);
      const float gam = kAmax ? __shfl_sync(kAll, am, (lane % G) * L) : 0.0f;
      if (lane / G == p) {
        hS = got;
        amax = gam;
      }
    }
  }
}

// The FP32 quadrature of one evaluation on window w, on this lane alone:
// h S, the shift point and cosh s - 1 there (NaN h S when the node bound is
// exceeded).
__device__ __forceinline__ Quad32 quad_f32(float x, float nu, float nu_lo, const Window32& w,
                                           Tally& tl) {
  Quad32 q;
  const Job32 jb = job_f32(x, nu, nu_lo, w, q, tl);
  if (jb.N >= 0) coop_trapezoid_f32<1>(jb, q.hS, q.amax);
  return q;
}

// log f_s = nu s - x cosh(s) - ln 2 in FP64 (nu s reaches ~200), s the
// quadrature's shift point.
__device__ __forceinline__ double log_scale_from(double x64, double nu64, const Quad32& q) {
  return fma(nu64, (double)q.ts, -x64 * ((double)q.ch.hi + (double)q.ch.lo)) - kLn2;
}

// The same log f_s = nu s - x cosh(s) - ln 2 as a double-float from the
// double-float x and nu, without FP64 instructions.
__device__ __forceinline__ DF df_log_scale(DF x, DF nu, const Quad32& q) {
  const DF a = df_add(df_mul_f(nu, q.ts), df_neg(df_mul(x, q.ch)));
  return df_add(a, DF{-kLn2DfHi, -kLn2DfLo});
}

// e^a for a FP64 argument with FP32 accuracy (MUFU ex2 on the reduced
// argument); NaN propagates, |a| beyond the double range is not handled.
__device__ __forceinline__ double exp_fast(double a) {
  double kd = fma(a, kLog2e, kRoundMagic);
  const int k = __double2loint(kd);
  kd -= kRoundMagic;
  double r = fma(-kd, kLn2Hi, a);
  r = fma(-kd, kLn2Lo, r);
  const int k1 = k >> 1;
  return ((double)mufu_ex2((float)r * kLog2ef) * pow2i(k1)) * pow2i(k - k1);
}

// ---------------------------------------------------------------------------
// Learned window (a10).  The window network's outputs (t*, t* - t0,
// t1 - t*, ln N) are tabulated by the inference kernel on a grid over
// (ln x, nu) and interpolated bilinearly here; the window is widened by a
// relative and an absolute margin and then checked:
//   F(t1) = nu (t1 - t^) - x (cosh t1 - cosh t^) + L <= 0 and, if t0 > 0,
//   F(t0) + ln 2 <= 0, with t^ the predicted peak and L = -log eps.
// F bounds g(t) - g(t^) + L from above on each side (see window_f64), and
// g(t^) <= g(t*), so a window that passes contains the eps-window of the
// unimodal integrand; anything else takes the searched window (fallback).
constexpr int kTabX = 512;   // ln x in [ln 1e-3, ln 140]
constexpr int kTabNu = 256;  // nu in [0.05, 20]
constexpr float kTabLx0 = -6.90775528f, kTabLx1 = 4.94164242f;
constexpr float kTabNu0 = 0.05f, kTabNu1 = 20.0f;

struct LearnedView {
  const float4* table;  // kTabNu rows of kTabX entries (t*, left, right, ln N)
  float margin_rel, margin_abs;
};

__device__ __forceinline__ bool learned_window_f32(const LearnedView& lv, float x, float nu,
                                                   Window32& w, unsigned& repairs) {
  const float lx = kLn2f * mufu_lg2(x);
  const float fx = (lx - kTabLx0) * ((kTabX - 1) / (kTabLx1 - kTabLx0));
  const float fn = (nu - kTabNu0) * ((kTabNu - 1) / (kTabNu1 - kTabNu0));
  if (!(fx >= 0.0f && fx <= (float)(kTabX - 1) && fn >= 0.0f && fn <= (float)(kTabNu - 1)))
    return false;
  const int ix = min((int)fx, kTabX - 2), in = min((int)fn, kTabNu - 2);
  const float ax = fx - (float)ix, an = fn - (float)in;
  const float4 p00 = __ldg(lv.table + in * kTabX + ix), p01 = __ldg(lv.table + in * kTabX + ix + 1);
  const float4 p10 = __ldg(lv.table + (in + 1) * kTabX + ix);
  const float4 p11 = __ldg(lv.table + (in + 1) * kTabX + ix + 1);
  const float b00 = (1.0f - ax) * (1.0f - an), b01 = ax * (1.0f - an), b10 = (1.0f - ax) * an,
              b11 = ax * an;
  const float ts = fmaxf(b00 * p00.x + b01 * p01.x + b10 * p10.x + b11 * p11.x, 0.0f);
  const float left = fmaxf(b00 * p00.y + b01 * p01.y + b10 * p10.y + b11 * p11.y, 0.0f);
  const float right = fmaxf(b00 * p00.z + b01 * p01.z + b10 * p10.z + b11 * p11.z, 0.0f);
  float t0 = fmaxf(0.0f, ts - fmaf(left, 1.0f + lv.margin_rel, lv.margin_abs));
  float t1 = ts + fmaf(right, 1.0f + lv.margin_rel, lv.margin_abs);
  const float L = kLogInvEps32;
  // Right end.  F is concave and decreasing past its maximum at asinh(nu/x):
  // a point with F > 0 and F' < 0 lies left of the root, and one Newton step
  // from there lands right of it (the tangent lies above F).
  const float F1 = fmaf(nu, t1 - ts, -x * dcosh_f32(t1, ts)) + L;
  if (F1 > 0.0f) {
    const float Fp = fmaf(-x, sinh_f32(t1), nu);
    if (!(Fp < 0.0f)) return false;
    t1 -= fast_div(F1, Fp);
    ++repairs;
  }
  // Left end (only when interior): G = F + ln 2 is concave and increasing on
  // [0, ts]; from a point with G > 0 one Newton step lands left of the root.
  if (t0 > 0.0f) {
    const float G = fmaf(nu, t0 - ts, -x * dcosh_f32(t0, ts)) + L + kLn2f;
    if (G > 0.0f) {
      const float Gp = fmaf(-x, sinh_f32(t0), nu);
      if (!(Gp > 0.0f)) return false;
      t0 = fmaxf(0.0f, t0 - fast_div(G, Gp));
      ++repairs;
    }
  }
  w.ts = ts;
  w.t0 = t0;
  w.t1 = t1;
  return true;
}

}  // namespace bk
