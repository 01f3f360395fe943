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

// e^a in FP64 range with FP32 accuracy: a = k ln 2 + r in FP64, e^r on MUFU.
__device__ __forceinline__ double exp_split(double a) {
  if (a != a) return a;
  if (a > 709.782712893384) return __longlong_as_double(0x7ff0000000000000LL);
  if (a < -745.2) return 0.0;
  double kd = fma(a, kLog2e, kRoundMagic);
  const int k = __double2loint(kd);
  kd -= kRoundMagic;
  double r = fma(-kd, kLn2Hi, a);
  r = fma(-kd, kLn2Lo, r);
  const double er = (double)mufu_ex2((float)r * kLog2ef);
  const int k1 = k >> 1;
  return (er * pow2i(k1)) * pow2i(k - k1);
}

struct Window32 {
  float ts, t0, t1;
};

// a3 in FP32: the same bracketed Newton as peak_f64 (g' concave on t > 0,
// negative at asinh(nu/x)); the right end is inflated slightly so that the
// FP32 value stays right of the root.
__device__ __forceinline__ float peak_f32(float x, float nu, Tally& tl) {
  const float nu2 = nu * nu;
  if (!(nu2 > x)) return 0.0f;
  const float q = nu / x;
  float hi = kLn2f * mufu_lg2(q + sqrtf(fmaf(q, q, 1.0f)));
  hi = fmaf(hi, 1.0e-4f, hi) + 1.0e-6f;
  float lo = 0.0f;
  const float tc2 = (nu2 - x) / fmaf(nu2 * nu2, 1.0f / 3.0f, x * (1.0f / 6.0f));
  float t = (tc2 < hi * hi) ? sqrtf(tc2) : hi;
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
      tn = t - gp / gpp;
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

// a4 in FP32 with the bound F of window_f64 (see there), eps = 2^-23.
__device__ __forceinline__ Window32 window_f32(float x, float nu, Tally& tl) {
  Window32 w;
  const float L = kLogInvEps32;
  const float ts = peak_f32(x, nu, tl);
  w.ts = ts;
  const float es = mufu_ex2(ts * kLog2ef);
  const float cs = 0.5f * (es + mufu_rcp(es));
  const float ss = sinh_f32(ts);
  {
    const float a = x * cs, b = nu - x * ss;
    float t = ts + (b + sqrtf(fmaf(b, b, 2.0f * a * L))) / a;
    t = fmaf(t, 1.0e-4f, t);
    float tb = kLn2f * mufu_lg2(2.0f * (L + a + nu * t) / x);
    tb = fmaf(tb, 1.0e-4f, tb);
    if (tb < t) t = tb;
    for (int it = 0; it < 40; ++it) {
      ++tl.iters;
      const float F = fmaf(nu, t - ts, -x * dcosh_f32(t, ts)) + L;
      const float Fp = fmaf(-x, sinh_f32(t), nu);
      const float dt = F / Fp;
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
      float t = fmaxf(0.0f, ts - Lp / nu);
      for (int it = 0; it < 40; ++it) {
        ++tl.iters;
        const float G = fmaf(nu, t - ts, -x * dcosh_f32(t, ts)) + Lp;
        const float Gp = fmaf(-x, sinh_f32(t), nu);
        float tn = t - G / Gp;
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

// Scaled trapezoid sum of the FP32 form, with the weights of Eq. (refined):
//   S = sum_j c_j exp(nu (t_j - ts) - x (cosh t_j - cosh ts)) (1 + e^{-2 nu t_j}),
// c_0 = c_N = 1/2, the exponent in the difference form, e^{-2 nu t_j} by a
// geometric recurrence and a Kahan-compensated sum.  Returns h S.
__device__ __forceinline__ float trapezoid_f32(float x, float nu, const Window32& w, int N,
                                               Tally& tl) {
  const float h = (w.t1 - w.t0) / (float)N;
  float W = mufu_ex2(-2.0f * kLog2ef * nu * w.t0);
  const float rho = mufu_ex2(-2.0f * kLog2ef * nu * h);
  float S = 0.0f, c = 0.0f;
  const float x2 = 2.0f * x;
  const bool at_zero = (w.ts == 0.0f);
  for (int j = 0; j <= N; ++j) {
    const float t = fmaf((float)j, h, w.t0);
    float a;
    if (at_zero) {
      const float s = sinh_f32(0.5f * t);
      a = fmaf(-x2 * s, s, nu * t);
    } else {
      a = fmaf(-x2 * sinh_f32(0.5f * (t + w.ts)), sinh_f32(0.5f * (t - w.ts)), nu * (t - w.ts));
    }
    float f = exp_f32(a);
    f = fmaf(f, W, f);
    if (j == 0 || j == N) f *= 0.5f;
    const float y = f - c;  // Kahan
    const float s2 = S + y;
    c = (s2 - S) - y;
    S = s2;
    W *= rho;
  }
  tl.nodes += N + 1;
  return h * S;
}

// Everything of one K_nu evaluation in the FP32 form except the final
// normalisation: returns h S (FP32) and the FP64 log-scale
// log f_s = nu ts - x cosh(ts) - ln 2, so that K = e^{log f_s} h S.
// Outside x in [1e-4, 1e4], nu <= 40 the FP64 window search is used.
// On failure (node bound exceeded) returns NaN scale.
__device__ __forceinline__ double log_scale_f32(double x64, float nu, float& hS, Tally& tl) {
  const float x = (float)x64;
  Window32 w;
  if (x >= 1e-4f && x <= 1e4f && nu <= 40.0f) {
    w = window_f32(x, nu, tl);
  } else {
    const Window64 w64 = window_f64(x64, (double)nu, (double)kLogInvEps32, tl);
    w.ts = (float)w64.ts;
    w.t0 = (float)w64.t0;
    w.t1 = (float)w64.t1;
  }
  const int N = strip_node_count(x, nu, w.t1 - w.t0, kF32Log2OverTol, kF32MaxNodes);
  if (N > kF32MaxNodes) {
    ++tl.fail;
    hS = 0.0f;
    return __longlong_as_double(0x7ff8000000000000LL);
  }
  hS = trapezoid_f32(x, nu, w, N, tl);
  double cs = 1.0;
  if (w.ts > 0.0f) {  // cosh of the (FP32) peak in FP64: x cosh(ts) can be ~1e2
    const double e = exp_bounded((double)w.ts);
    cs = 0.5 * (e + 1.0 / e);
  }
  return fma((double)nu, (double)w.ts, -x64 * cs) - kLn2;
}

}  // namespace bk
