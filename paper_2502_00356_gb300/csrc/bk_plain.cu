// Plain FP64 form: K_nu evaluation and the fused Matern tile writer
// (distance -> r/beta -> K_nu -> normalisation -> store), Algorithm 3 and
// Sec. IV-B, with the window search, strip-bound node count and log-domain
// trapezoid of bk_math64.cuh.  One thread evaluates one K_nu.
#include <cuda_runtime.h>

#include <cstdint>

#include "bk_internal.h"
#include "bk_math64.cuh"
#include "bk_tiles.cuh"

namespace bk {

struct FormF64 {
  static __device__ __forceinline__ double eval(double x, double nu, Tally& tl, unsigned& evals,
                                                double& log_k) {
    ++evals;
    log_k = log_kv_f64(x, nu, kPlainLog2OverTol, kPlainMaxNodes, tl);
    return exp_full(log_k);
  }

  // a2 + a3..a7 for one entry: distance, x = r / beta, log K_nu(x),
  // M = exp(log prefactor + nu log x + log K).  sigma^2 where r == 0
  // (Algorithm 3 tests the computed distance for exact zero).
  static __device__ __forceinline__ double matern(double xi, double yi, double xj, double yj,
                                                  double sigma2, double beta, double nu,
                                                  double log_pref, Tally& tl, unsigned& evals) {
    const double dx = xj - xi, dy = yj - yi;
    const double r = sqrt(fma(dx, dx, dy * dy));
    if (r == 0.0) return sigma2;
    const double z = r / beta;
    ++evals;
    const double lk = log_kv_f64(z, nu, kPlainLog2OverTol, kPlainMaxNodes, tl);
    return exp_full(fma(nu, log_pos(z), log_pref) + lk);
  }
};

int grid_for(int64_t work_items, int per_sm) {
  const int64_t cap = (int64_t)current_sm_count() * per_sm;
  return (int)(work_items < cap ? (work_items > 0 ? work_items : 1) : cap);
}

cudaError_t launch_eval_f64(const double* x, const double* nu, void* out, void* log_out,
                            bk_dtype out_t, int64_t n, unsigned long long* ctr, cudaStream_t s) {
  return launch_eval_form<FormF64>(x, nu, out, log_out, out_t, n, ctr, s);
}

cudaError_t launch_matern_sym_f64(const double* locs, int64_t n, double sigma2, double beta,
                                  double nu, void* out, int64_t ld, bk_dtype out_t,
                                  unsigned long long* ctr, cudaStream_t s) {
  return launch_matern_sym_form<FormF64>(locs, n, sigma2, beta, nu, out, ld, out_t, ctr, s);
}

cudaError_t launch_matern_block_f64(const double* locs1, int64_t m, const double* locs2,
                                    int64_t n, double sigma2, double beta, double nu, void* out,
                                    int64_t ld, bk_dtype out_t, unsigned long long* ctr,
                                    cudaStream_t s) {
  return launch_matern_block_form<FormF64>(locs1, m, locs2, n, sigma2, beta, nu, out, ld, out_t,
                                           ctr, s);
}

}  // namespace bk
