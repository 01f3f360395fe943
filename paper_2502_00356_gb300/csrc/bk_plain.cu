// Plain FP64 form: K_nu evaluation and the fused Matern tile writer
// (distance -> r/beta -> K_nu -> normalisation -> store), Algorithm 3 and
// Sec. IV-B, with the window search, strip-bound node count and log-domain
// trapezoid of bk_math64.cuh, or the paper's fixed window (Algorithm 2), and
// Temme's series for small x when asked.  One thread evaluates one K_nu.
#include <cuda_runtime.h>

#include <cstdint>

#include "bk_internal.h"
#include "bk_forms.cuh"
#include "bk_tiles.cuh"

namespace bk {

namespace {

// Fills the per-launch table of e^{-2 nu h} on kCoshTab's steps.
__global__ void __launch_bounds__(256) decay_table_kernel(double nu, double* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < kCoshTabSize) out[k] = decay_entry(nu, k, kExp2Tab);
}

// Runs launch(form) for a Matern tile writer of the searched-window form with
// form.wnu pointing at the caller's table (bk_opts.d_cosh_table), first
// filled on s with e^{-2 nu h} for this launch's nu.  Without a table the
// kernels compute the values themselves; forms without the table run as
// they are.  Allocates nothing.
// fill = false: the table already holds this nu's values (an earlier launch
// for the same matrix filled it on s).
template <class Form, class Launch>
cudaError_t with_decay_table(Form form, double nu, double* table, cudaStream_t s,
                               Launch&& launch, bool fill = true) {
  if constexpr (Form::kDecayTable) {
    if (table != nullptr) {
      static_assert(kCoshTabSize == BK_COSH_TABLE_LEN, "table length");
      if (fill) decay_table_kernel<<<(kCoshTabSize + 255) / 256, 256, 0, s>>>(nu, table);
      form.wnu = table;
    }
  }
  return launch(form);
}

}  // namespace

int grid_for(int64_t work_items, int per_sm) {
  const int64_t cap = (int64_t)current_sm_count() * per_sm;
  return (int)(work_items < cap ? (work_items > 0 ? work_items : 1) : cap);
}

// Calls launch(form) with the plain form the options select: the paper's
// fixed window (Algorithm 2) or the searched window, each with the optional
// series branch for small x.
template <class Launch>
cudaError_t with_plain_form(const bk_opts& o, Launch&& launch) {
  if (o.window == BK_WIN_FIXED)
    return launch(FormF64Fixed{nullptr, o.fixed_t1, o.fixed_bins, o.series_below});
  if (o.series_below > 0.0) return launch(FormF64Series{nullptr, o.search_f64 != 0, o.series_below});
  return launch(FormF64{nullptr, o.search_f64 != 0, 0.0});
}

cudaError_t launch_eval_f64(const double* x, const double* nu, void* out, void* log_out,
                            bk_dtype out_t, int64_t n, const bk_opts& o, cudaStream_t s) {
  return with_plain_form(o, [&](const auto& form) {
    return launch_eval_form(form, x, nu, out, log_out, out_t, n, o.d_counters, s);
  });
}

cudaError_t launch_matern_sym_f64(const double* locs, int64_t n, double sigma2, double beta,
                                  double nu, void* out, int64_t ld, bk_dtype out_t,
                                  const bk_opts& o, cudaStream_t s, const SymRange& range) {
  if (n == 0) return cudaSuccess;
  return with_plain_form(o, [&](const auto& form) {
    return with_decay_table(
        form, nu, o.d_cosh_table, s,
        [&](const auto& f) {
          return launch_matern_sym_form(f, locs, n, sigma2, beta, nu, out, ld, out_t,
                                        o.d_counters, s, range);
        },
        range.fill_table);
  });
}

cudaError_t launch_matern_block_f64(const double* locs1, int64_t m, const double* locs2,
                                    int64_t n, double sigma2, double beta, double nu, void* out,
                                    int64_t ld, bk_dtype out_t, const bk_opts& o, cudaStream_t s) {
  if (m == 0 || n == 0) return cudaSuccess;
  return with_plain_form(o, [&](const auto& form) {
    return with_decay_table(form, nu, o.d_cosh_table, s, [&](const auto& f) {
      return launch_matern_block_form(f, locs1, m, locs2, n, sigma2, beta, nu, out, ld, out_t,
                                      o.d_counters, s);
    });
  });
}

cudaError_t launch_eval_grad_f64(const double* x, const double* nu, double* k, double* dkdx,
                                 double* dkdnu, int64_t n, const bk_opts& o, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int grid = one_wave_grid(n, 4);
  eval_grad_kernel<FormF64><<<grid, 128, 0, s>>>(FormF64{nullptr, o.search_f64 != 0, 0.0}, x, nu,
                                                 k, dkdx, dkdnu, n, o.d_counters);
  return cudaGetLastError();
}

}  // namespace bk
