// Per-matrix constants and staged locations shared by the Matern kernels and
// the arithmetic forms.
#pragma once

#include <cmath>
#include <cstdint>

#include "bk_math64.cuh"

namespace bk {

constexpr double kInf = __builtin_huge_val();

// Output conversion of a double result (FP32 outputs round once).
template <typename T>
__device__ __forceinline__ T to_out(double v);
template <>
__device__ __forceinline__ double to_out<double>(double v) { return v; }
template <>
__device__ __forceinline__ float to_out<float>(double v) { return (float)v; }


// a1: log of the Matern prefactor sigma^2 / (2^{nu-1} Gamma(nu)) (Sec. III-A).
__device__ __forceinline__ double matern_log_prefactor(double sigma2, double nu) {
  const double ls = (sigma2 > 0.0) ? log_pos(sigma2) : -kInf;
  return ls - (nu - 1.0) * kLn2 - lgamma(nu);
}

// Per-matrix constants of one Matern launch (a1 and the order split).
struct MaternParams {
  double sigma2, beta, nu, log_pref, inv_beta;
  double nu_k;                     // nu times K = 4096/ln 2 (exp_units_full's units)
  double log_pref_kh;              // K (a1 + nu ln(2 ln 2)): the exponent's constant for log(xh 2^-12)
  double xh_c2;                    // (K/2 / beta)^2: xh = x K/2 = sqrt(r^2 xh_c2)
  float inv_beta_f, nu_hi, nu_lo;  // nu = nu_hi + nu_lo (two floats)
  float inv_beta_lo;               // 1/beta = inv_beta_f + inv_beta_lo
  float log_pref_hi, log_pref_lo;  // a1 as two floats
  float log_pref_m_ln2_hi, log_pref_m_ln2_lo;  // a1 - ln 2 as two floats (FP32 forms)
  float sigma2_f;                  // sigma^2 as a float (the FP32 diagonal)
};

__device__ __forceinline__ MaternParams matern_params(double sigma2, double beta, double nu) {
  MaternParams p;
  p.sigma2 = sigma2;
  p.beta = beta;
  p.nu = nu;
  p.log_pref = matern_log_prefactor(sigma2, nu);
  p.nu_k = nu * kExpScale;
  p.log_pref_kh = fma(nu, 0.32663425997828094, p.log_pref) * kExpScale;  // ln(2 ln 2)
  p.inv_beta = 1.0 / beta;
  const double hb = (0.5 * kExpScale) * p.inv_beta;
  p.xh_c2 = hb * hb;
  p.inv_beta_f = (float)p.inv_beta;
  p.nu_hi = (float)nu;
  p.nu_lo = (float)(nu - (double)p.nu_hi);
  p.inv_beta_lo = (float)(p.inv_beta - (double)p.inv_beta_f);
  p.log_pref_hi = (float)p.log_pref;
  p.log_pref_lo = (float)(p.log_pref - (double)p.log_pref_hi);
  const double lpm = p.log_pref - kLn2;
  p.log_pref_m_ln2_hi = (float)lpm;
  p.log_pref_m_ln2_lo = (float)(lpm - (double)p.log_pref_m_ln2_hi);
  p.sigma2_f = (float)sigma2;
  return p;
}

// The same constants computed on the host (std::log, std::lgamma) for the
// single-matrix launches, so that their many blocks start without per-block
// setup arithmetic.
inline MaternParams matern_params_host(double sigma2, double beta, double nu) {
  MaternParams p;
  p.sigma2 = sigma2;
  p.beta = beta;
  p.nu = nu;
  p.log_pref = (sigma2 > 0.0 ? std::log(sigma2) : -kInf) - (nu - 1.0) * kLn2 - std::lgamma(nu);
  p.nu_k = nu * kExpScale;
  p.log_pref_kh = std::fma(nu, std::log(2.0 * kLn2), p.log_pref) * kExpScale;
  p.inv_beta = 1.0 / beta;
  const double hb = (0.5 * kExpScale) * p.inv_beta;
  p.xh_c2 = hb * hb;
  p.inv_beta_f = (float)p.inv_beta;
  p.nu_hi = (float)nu;
  p.nu_lo = (float)(nu - (double)p.nu_hi);
  p.inv_beta_lo = (float)(p.inv_beta - (double)p.inv_beta_f);
  p.log_pref_hi = (float)p.log_pref;
  p.log_pref_lo = (float)(p.log_pref - (double)p.log_pref_hi);
  const double lpm = p.log_pref - kLn2;
  p.log_pref_m_ln2_hi = (float)lpm;
  p.log_pref_m_ln2_lo = (float)(lpm - (double)p.log_pref_m_ln2_hi);
  p.sigma2_f = (float)sigma2;
  return p;
}

// A location as staged in shared memory: FP64 coordinates and the same
// coordinates as float pairs (hi + lo), so that FP32 forms can form exact-ish
// differences without FP64 instructions.
struct Loc {
  double x, y;
  float xh, xl, yh, yl;
};

__device__ __forceinline__ void split_f(double v, float& h, float& l) {
  h = (float)v;
  l = (float)(v - (double)h);
}

}  // namespace bk
