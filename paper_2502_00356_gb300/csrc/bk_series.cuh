// Temme's series with Campbell's forward recurrence (Sec. IV-A), the small-x
// branch of the paper's refined algorithm (Algorithm 2: x < 0.1), FP64.
//
// For nu = mu + M, M = floor(nu + 1/2), |mu| <= 1/2:
//   K_mu = sum_k c_k f_k,  K_{mu+1} = (2/x) sum_k c_k h_k,  c_k = (x^2/4)^k / k!,
//   h_k = p_k - k f_k,  p_k = p_{k-1}/(k - mu),  q_k = q_{k-1}/(k + mu),
//   f_k = (k f_{k-1} + p_{k-1} + q_{k-1}) / (k^2 - mu^2),
//   p_0 = (1/2)(x/2)^{-mu} Gamma(1+mu),  q_0 = (1/2)(x/2)^{mu} Gamma(1-mu),
//   f_0 = (mu pi / sin(mu pi)) [cosh(s) G1(mu) + (sinh(s)/s) ln(2/x) G2(mu)],
// with s = mu ln(2/x) and Temme's G1, G2 (the paper leaves them undefined).
// G1 and G2 come from the Taylor series of 1/Gamma in mu^2
// (bk_rgamma_coeffs.inc), which avoids the cancellation of G1's defining
// difference near mu = 0; 1/Gamma(1 -+ mu) = G2 +- mu G1.  The sum stops when
// both new terms are below 2^-54 of their sums (at most 15,000 terms, the
// paper's cap), then K_{eta+1} = (2 eta / x) K_eta + K_{eta-1} runs upward to
// nu, rescaled by 2^-800 whenever it passes 2^800 so that large orders at tiny
// x do not overflow.  The transcendental functions here are CUDA's: this
// branch is not on the integration hot path.
#pragma once

#include "bk_math64.cuh"

namespace bk {

#include "bk_rgamma_coeffs.inc"

// log K_nu(x) for x > 0 (intended for x below ~2, where the series converges
// quickly); terms receives the number of series terms used.
static __device__ __noinline__ double series_log_k(double x, double nu, unsigned& terms) {
  nu = fabs(nu);
  const double M = floor(nu + 0.5);
  const double mu = nu - M;
  const double m2 = mu * mu;
  double g2 = kG2Coef[kG2Terms - 1];
  for (int i = kG2Terms - 2; i >= 0; --i) g2 = fma(g2, m2, kG2Coef[i]);
  double g1 = kG1Coef[kG1Terms - 1];
  for (int i = kG1Terms - 2; i >= 0; --i) g1 = fma(g1, m2, kG1Coef[i]);
  const double rg_plus = fma(-mu, g1, g2);  // 1/Gamma(1 + mu)
  const double rg_minus = fma(mu, g1, g2);  // 1/Gamma(1 - mu)
  const double lx = log(2.0 / x);
  const double s = mu * lx;
  const double fact = (mu == 0.0) ? 1.0 : (3.141592653589793 * mu) / sinpi(mu);
  const double shs = (s == 0.0) ? 1.0 : sinh(s) / s;
  double f = fact * fma(cosh(s), g1, shs * lx * g2);
  const double es = exp(s);
  double p = 0.5 * es / rg_plus;
  double q = 0.5 / (es * rg_minus);
  double c = 1.0;
  const double y = 0.25 * x * x;
  double sum_f = f, sum_h = p;
  int k = 1;
  for (; k <= 15000; ++k) {
    const double kd = (double)k;
    f = (fma(kd, f, p) + q) / fma(kd, kd, -m2);
    p = p / (kd - mu);
    q = q / (kd + mu);
    c = c * y / kd;
    const double tf = c * f;
    const double th = c * fma(-kd, f, p);
    sum_f += tf;
    sum_h += th;
    if (fabs(tf) <= 0x1p-54 * fabs(sum_f) && fabs(th) <= 0x1p-54 * fabs(sum_h)) break;
  }
  terms = (unsigned)min(k, 15000);
  const int m = (int)M;
  if (m == 0) return log(sum_f);
  double prev = sum_f, cur = (2.0 / x) * sum_h;  // K_mu, K_{mu+1}
  double log_scale = 0.0;
  for (int j = 1; j < m; ++j) {
    const double next = fma(2.0 * (mu + (double)j) / x, cur, prev);
    prev = cur;
    cur = next;
    if (cur > 0x1p800) {
      prev *= 0x1p-800;
      cur *= 0x1p-800;
      log_scale += 800.0 * kLn2;
    }
  }
  return log(cur) + log_scale;
}

}  // namespace bk
