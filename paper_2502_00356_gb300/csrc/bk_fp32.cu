// FP32 precision form: the integrand, window search and node count in FP32
// (bk_math32.cuh); distance, cosh(t_max) and the log-domain normalisation in
// FP64 where cancellation or large magnitudes need it.
#include <cuda_runtime.h>

#include <cstdint>

#include "bk_internal.h"
#include "bk_math32.cuh"
#include "bk_tiles.cuh"

namespace bk {

struct FormF32 {
  static __device__ __forceinline__ double eval(double x, double nu, Tally& tl, unsigned& evals,
                                                double& log_k) {
    ++evals;
    float hS;
    const double scale = log_scale_f32(x, (float)nu, hS, tl);
    log_k = scale + (double)(kLn2f * mufu_lg2(hS));
    return exp_split(scale) * (double)hS;
  }

  // a2 in FP64; a3..a6 in FP32; a7 as the FP64 sum
  // log prefactor + nu log x + log f_s, exponentiated and scaled by h S.
  static __device__ __forceinline__ double matern(double xi, double yi, double xj, double yj,
                                                  double sigma2, double beta, double nu,
                                                  double log_pref, Tally& tl, unsigned& evals) {
    const double dx = xj - xi, dy = yj - yi;
    const double r = sqrt(fma(dx, dx, dy * dy));
    if (r == 0.0) return sigma2;
    const double z = r / beta;
    ++evals;
    float hS;
    const double scale = log_scale_f32(z, (float)nu, hS, tl);
    // log x in FP64 near r -> 0, where nu log x cancels against log K_nu
    const double lz = (z < 1.0) ? log_pos(z) : (double)(kLn2f * mufu_lg2((float)z));
    return exp_split(fma(nu, lz, log_pref) + scale) * (double)hS;
  }
};

cudaError_t launch_eval_f32(const double* x, const double* nu, void* out, void* log_out,
                            bk_dtype out_t, int64_t n, unsigned long long* ctr, cudaStream_t s) {
  return launch_eval_form<FormF32>(x, nu, out, log_out, out_t, n, ctr, s);
}

cudaError_t launch_matern_sym_f32(const double* locs, int64_t n, double sigma2, double beta,
                                  double nu, void* out, int64_t ld, bk_dtype out_t,
                                  unsigned long long* ctr, cudaStream_t s) {
  return launch_matern_sym_form<FormF32>(locs, n, sigma2, beta, nu, out, ld, out_t, ctr, s);
}

cudaError_t launch_matern_block_f32(const double* locs1, int64_t m, const double* locs2,
                                    int64_t n, double sigma2, double beta, double nu, void* out,
                                    int64_t ld, bk_dtype out_t, unsigned long long* ctr,
                                    cudaStream_t s) {
  return launch_matern_block_form<FormF32>(locs1, m, locs2, n, sigma2, beta, nu, out, ld, out_t,
                                           ctr, s);
}

}  // namespace bk
