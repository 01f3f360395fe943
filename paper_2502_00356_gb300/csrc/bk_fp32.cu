// FP32 precision form: the integrand, window search and node count in FP32
// (bk_math32.cuh); distance, cosh(t_max) and the log-domain normalisation in
// FP64 where cancellation or large magnitudes need it.
#include <cuda_runtime.h>

#include <cstdint>

#include "bk_internal.h"
#include "bk_forms.cuh"
#include "bk_tiles.cuh"

namespace bk {

cudaError_t launch_eval_f32(const double* x, const double* nu, void* out, void* log_out,
                            bk_dtype out_t, int64_t n, unsigned long long* ctr, cudaStream_t s,
                            int lanes) {
  return launch_eval_form(FormF32{nullptr}, x, nu, out, log_out, out_t, n, ctr, s, lanes);
}

cudaError_t launch_matern_sym_f32(const double* locs, int64_t n, double sigma2, double beta,
                                  double nu, void* out, int64_t ld, bk_dtype out_t,
                                  unsigned long long* ctr, cudaStream_t s, const SymRange& range) {
  return launch_matern_sym_form(FormF32{nullptr}, locs, n, sigma2, beta, nu, out, ld, out_t, ctr, s,
                                range);
}

cudaError_t launch_matern_block_f32(const double* locs1, int64_t m, const double* locs2,
                                    int64_t n, double sigma2, double beta, double nu, void* out,
                                    int64_t ld, bk_dtype out_t, unsigned long long* ctr,
                                    cudaStream_t s) {
  return launch_matern_block_form(FormF32{nullptr}, locs1, m, locs2, n, sigma2, beta, nu, out, ld, out_t,
                                           ctr, s);
}

}  // namespace bk
