// Plain FP64 form: K_nu evaluation and the fused Matern tile writer
// (distance -> r/beta -> K_nu -> normalisation -> store), Algorithm 3 and
// Sec. IV-B, with the window search, strip-bound node count and log-domain
// trapezoid of bk_math64.cuh.  One thread evaluates one K_nu.
#include <cuda_runtime.h>

#include <cstdint>

#include "bk_internal.h"
#include "bk_forms.cuh"
#include "bk_tiles.cuh"

namespace bk {

int grid_for(int64_t work_items, int per_sm) {
  const int64_t cap = (int64_t)current_sm_count() * per_sm;
  return (int)(work_items < cap ? (work_items > 0 ? work_items : 1) : cap);
}

cudaError_t launch_eval_f64(const double* x, const double* nu, void* out, void* log_out,
                            bk_dtype out_t, int64_t n, bool search_f64, unsigned long long* ctr,
                            cudaStream_t s) {
  return launch_eval_form(FormF64{nullptr, search_f64}, x, nu, out, log_out, out_t, n, ctr, s);
}

cudaError_t launch_matern_sym_f64(const double* locs, int64_t n, double sigma2, double beta,
                                  double nu, void* out, int64_t ld, bk_dtype out_t,
                                  bool search_f64, unsigned long long* ctr, cudaStream_t s) {
  return launch_matern_sym_form(FormF64{nullptr, search_f64}, locs, n, sigma2, beta, nu, out, ld,
                                out_t, ctr, s);
}

cudaError_t launch_matern_block_f64(const double* locs1, int64_t m, const double* locs2,
                                    int64_t n, double sigma2, double beta, double nu, void* out,
                                    int64_t ld, bk_dtype out_t, bool search_f64,
                                    unsigned long long* ctr, cudaStream_t s) {
  return launch_matern_block_form(FormF64{nullptr, search_f64}, locs1, m, locs2, n, sigma2, beta, nu,
                                  out, ld, out_t, ctr, s);
}

}  // namespace bk
