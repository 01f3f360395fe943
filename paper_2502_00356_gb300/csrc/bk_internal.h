// Internal declarations shared by the library's translation units (not part
// of the public C-ABI in include/bk.h).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "bk.h"

namespace bk {

// Number of SMs of the current device (cached per device ordinal).
int current_sm_count();

// Records a message for bk_last_error() on this thread and returns `st`.
bk_status set_error(bk_status st, const char* fmt, ...);

// Converts a CUDA error into BK_ERR_CUDA with a message (BK_OK if none).
bk_status check_cuda(cudaError_t e, const char* what);

// A range of block-columns [j0, j1) of a symmetric matrix (32-wide blocks),
// written in block-column order; j1 < 0 means the whole matrix.  fill_table:
// whether a launch of the plain form refills the caller's e^{-2 nu h} table
// (a caller writing several ranges of one matrix fills it with the first).
struct SymRange {
  int64_t j0 = 0, j1 = -1;
  bool fill_table = true;
};

// ---- plain FP64 form (bk_plain.cu) ----
cudaError_t launch_eval_f64(const double* x, const double* nu, void* out, void* log_out,
                            bk_dtype out_t, int64_t n, const bk_opts& o, cudaStream_t s);

// Full symmetric n x n matrix: lower-triangle tiles, each written twice.
cudaError_t launch_matern_sym_f64(const double* locs, int64_t n, double sigma2, double beta,
                                  double nu, void* out, int64_t ld, bk_dtype out_t,
                                  const bk_opts& o, cudaStream_t s,
                                  const SymRange& range = SymRange{});

// General m x n block between two location sets.
cudaError_t launch_matern_block_f64(const double* locs1, int64_t m, const double* locs2,
                                    int64_t n, double sigma2, double beta, double nu, void* out,
                                    int64_t ld, bk_dtype out_t, const bk_opts& o, cudaStream_t s);

// K, dK/dx, dK/dnu of the plain form (outputs may be null).
cudaError_t launch_eval_grad_f64(const double* x, const double* nu, double* k, double* dkdx,
                                 double* dkdnu, int64_t n, const bk_opts& o, cudaStream_t s);

// The Gaussian log-likelihood steps (Cholesky, log det, forward
// substitution, reduction) on `s`; see bk_gaussian_loglik.
cudaError_t launch_loglik(double* a, int64_t n, int64_t ld, const double* z, double* y,
                          double* out, unsigned long long* ctr, cudaStream_t s);

// Option checks shared by every entry point that takes bk_opts (sets the
// error message and returns the status).
bk_status check_opts(const bk_opts* o);

// Lanes per evaluation of the FP32 forms' bare evaluations: opts.lanes, else
// bk_eval_autotune's choice for the current device, else the default.
int eval_lanes(const bk_opts& o, bk_dtype out_dtype);

// ---- FP32 precision form (bk_fp32.cu) ----
cudaError_t launch_eval_f32(const double* x, const double* nu, void* out, void* log_out,
                            bk_dtype out_t, int64_t n, unsigned long long* ctr, cudaStream_t s,
                            int lanes);
cudaError_t launch_matern_sym_f32(const double* locs, int64_t n, double sigma2, double beta,
                                  double nu, void* out, int64_t ld, bk_dtype out_t,
                                  unsigned long long* ctr, cudaStream_t s,
                                  const SymRange& range = SymRange{});
cudaError_t launch_matern_block_f32(const double* locs1, int64_t m, const double* locs2,
                                    int64_t n, double sigma2, double beta, double nu, void* out,
                                    int64_t ld, bk_dtype out_t, unsigned long long* ctr,
                                    cudaStream_t s);

// ---- learned window (bk_learned.cu); `m` must have weights (learned_ready)
bool learned_ready(const bk_learned* m);
cudaError_t launch_eval_learned(const bk_learned* m, const double* x, const double* nu, void* out,
                                void* log_out, bk_dtype out_t, int64_t n, unsigned long long* ctr,
                                cudaStream_t s, int lanes);
cudaError_t launch_matern_sym_learned(const bk_learned* m, const double* locs, int64_t n,
                                      double sigma2, double beta, double nu, void* out, int64_t ld,
                                      bk_dtype out_t, unsigned long long* ctr, cudaStream_t s,
                                      const SymRange& range = SymRange{});
cudaError_t launch_matern_block_learned(const bk_learned* m, const double* locs1, int64_t m_,
                                        const double* locs2, int64_t n, double sigma2,
                                        double beta, double nu, void* out, int64_t ld,
                                        bk_dtype out_t, unsigned long long* ctr, cudaStream_t s);

}  // namespace bk
