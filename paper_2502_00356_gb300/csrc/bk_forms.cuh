// The two arithmetic forms of one K_nu evaluation and one Matern entry, as
// policies for the kernels of bk_tiles.cuh:
//  * FormF64, the plain form: FP64 search and quadrature (bk_math64.cuh);
//  * FormF32, the precision form: FP32 search and quadrature on the FMA and
//    MUFU pipes (bk_math32.cuh), FP64 distance and log-domain normalisation.
#pragma once

#include "bk.h"
#include "bk_math32.cuh"
#include "bk_math64.cuh"

namespace bk {

struct FormF64 {
  __device__ __forceinline__ double eval(double x, double nu, Tally& tl, unsigned& evals,
                                                double& log_k) const {
    ++evals;
    log_k = log_kv_f64(x, nu, kPlainLog2OverTol, kPlainMaxNodes, tl);
    return exp_full(log_k);
  }

  // a2 + a3..a7 for one entry: distance, x = r / beta, log K_nu(x),
  // M = exp(log prefactor + nu log x + log K).  sigma^2 where r == 0
  // (Algorithm 3 tests the computed distance for exact zero).
  __device__ __forceinline__ double matern(double xi, double yi, double xj, double yj,
                                                  double sigma2, double beta, double nu,
                                                  double log_pref, Tally& tl, unsigned& evals) const {
    const double dx = xj - xi, dy = yj - yi;
    const double r = sqrt(fma(dx, dx, dy * dy));
    if (r == 0.0) return sigma2;
    const double z = r / beta;
    ++evals;
    const double lk = log_kv_f64(z, nu, kPlainLog2OverTol, kPlainMaxNodes, tl);
    return exp_full(fma(nu, log_pos(z), log_pref) + lk);
  }
};

struct FormF32 {
  __device__ __forceinline__ double eval(double x, double nu, Tally& tl, unsigned& evals,
                                                double& log_k) const {
    ++evals;
    float hS;
    const double scale = log_scale_f32(x, nu, hS, tl);
    log_k = scale + (double)(kLn2f * mufu_lg2(hS));
    return exp_split(scale) * (double)hS;
  }

  // a2 in FP64; a3..a6 in FP32; a7 as the FP64 sum
  // log prefactor + nu log x + log f_s, exponentiated and scaled by h S.
  __device__ __forceinline__ double matern(double xi, double yi, double xj, double yj,
                                                  double sigma2, double beta, double nu,
                                                  double log_pref, Tally& tl, unsigned& evals) const {
    const double dx = xj - xi, dy = yj - yi;
    const double r = sqrt(fma(dx, dx, dy * dy));
    if (r == 0.0) return sigma2;
    const double z = r / beta;
    ++evals;
    float hS;
    const double scale = log_scale_f32(z, nu, hS, tl);
    // log x in FP64 near r -> 0, where nu log x cancels against log K_nu
    const double lz = (z < 1.0) ? log_pos(z) : (double)(kLn2f * mufu_lg2((float)z));
    return exp_split(fma(nu, lz, log_pref) + scale) * (double)hS;
  }
};

// Device view (table and margins) of a window network with weights.
LearnedView learned_view(const bk_learned* m);

// FP32 form with the learned window (a10): the window comes from the
// tabulated network when it passes the in-kernel check, else from the search
// (counted as a fallback).  A non-finite sum (a badly placed predicted peak
// can overflow the scaled nodes) also falls back.
struct FormF32Learned {
  LearnedView lv;

  __device__ __forceinline__ double scale(double x, double nu, float& hS, Tally& tl) const {
    Window32 w;
    if (learned_window_f32(lv, (float)x, (float)nu, w)) {
      const double sc = scale_from_window_f32(x, nu, w, hS, tl);
      if (isfinite(hS) && hS > 0.0f && sc == sc) return sc;
    }
    ++tl.fallback;
    return log_scale_f32(x, nu, hS, tl);
  }

  __device__ __forceinline__ double eval(double x, double nu, Tally& tl, unsigned& evals,
                                         double& log_k) const {
    ++evals;
    float hS;
    const double sc = scale(x, nu, hS, tl);
    log_k = sc + (double)(kLn2f * mufu_lg2(hS));
    return exp_split(sc) * (double)hS;
  }

  __device__ __forceinline__ double matern(double xi, double yi, double xj, double yj,
                                           double sigma2, double beta, double nu,
                                           double log_pref, Tally& tl, unsigned& evals) const {
    const double dx = xj - xi, dy = yj - yi;
    const double r = sqrt(fma(dx, dx, dy * dy));
    if (r == 0.0) return sigma2;
    const double z = r / beta;
    ++evals;
    float hS;
    const double sc = scale(z, nu, hS, tl);
    const double lz = (z < 1.0) ? log_pos(z) : (double)(kLn2f * mufu_lg2((float)z));
    return exp_split(fma(nu, lz, log_pref) + sc) * (double)hS;
  }
};

}  // namespace bk
