// The C-ABI of libbesselk (include/bk.h): host-side argument checks, option
// handling and dispatch to the kernels.  Nothing here allocates device memory
// or synchronises, except bk_sync.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <numeric>
#include <vector>

#include "bk_internal.h"

namespace bk {

namespace {
thread_local char g_err[512] = "";
// lanes per evaluation chosen by bk_eval_autotune, per device, FP32 form
// (searched, learned window) and output dtype; 0 = not tuned.
std::mutex g_lanes_mutex;
int g_eval_lanes[64][2][2] = {};
std::mutex g_sm_mutex;
int g_sm_count[64] = {0};
}  // namespace

bk_status set_error(bk_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return st;
}

bk_status check_cuda(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return BK_OK;
  return set_error(BK_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

int current_sm_count() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 132;
  std::lock_guard<std::mutex> lk(g_sm_mutex);
  if (g_sm_count[dev] == 0) {
    int c = 0;
    if (cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || c <= 0)
      c = 132;
    g_sm_count[dev] = c;
  }
  return g_sm_count[dev];
}

namespace {
bool finite(double v) { return std::isfinite(v); }
}  // namespace

int eval_lanes(const bk_opts& o, bk_dtype out_dtype) {
  if (o.lanes != 0) return o.lanes;
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64) {
    std::lock_guard<std::mutex> lk(g_lanes_mutex);
    const int t = g_eval_lanes[dev][o.window == BK_WIN_LEARNED ? 1 : 0][out_dtype == BK_F32 ? 1 : 0];
    if (t != 0) return t;
  }
  return BK_EVAL_LANES_DEFAULT;
}

bk_status check_opts(const bk_opts* o) {
  if (o->window != BK_WIN_SEARCH && o->window != BK_WIN_LEARNED && o->window != BK_WIN_FIXED)
    return set_error(BK_ERR_INVALID_ARG, "opts.window: unknown value %d", (int)o->window);
  if (o->compute != BK_F64 && o->compute != BK_F32)
    return set_error(BK_ERR_INVALID_ARG, "opts.compute: unknown dtype %d", (int)o->compute);
  if (!finite(o->series_below) || o->series_below < 0.0 || o->series_below > 2.0)
    return set_error(BK_ERR_INVALID_ARG, "opts.series_below must be in [0, 2] (got %g)",
                     o->series_below);
  if (o->series_below > 0.0 && o->compute != BK_F64)
    return set_error(BK_ERR_UNSUPPORTED, "opts.series_below needs compute = BK_F64");
  if (o->window == BK_WIN_FIXED) {
    if (o->fixed_bins < 1 || o->fixed_bins > 100000 || !(o->fixed_t1 > 0.0) ||
        !(o->fixed_t1 <= 700.0))
      return set_error(BK_ERR_INVALID_ARG,
                       "opts: the fixed window needs 1 <= fixed_bins <= 100000 and "
                       "0 < fixed_t1 <= 700");
    if (o->compute != BK_F64)
      return set_error(BK_ERR_UNSUPPORTED, "the fixed window needs compute = BK_F64");
  }
  if (o->lanes != 0 && o->lanes != 1 && o->lanes != 2 && o->lanes != 4 && o->lanes != 8)
    return set_error(BK_ERR_INVALID_ARG, "opts.lanes must be 0, 1, 2, 4 or 8 (got %d)", o->lanes);
  if (o->window == BK_WIN_LEARNED) {
    if (o->compute != BK_F32)
      return set_error(BK_ERR_UNSUPPORTED, "the learned window needs compute = BK_F32 "
                                           "(the network is trained on eps = 2^-23 windows)");
    if (!learned_ready(o->learned))
      return set_error(BK_ERR_NOT_LOADED, "opts.learned has no trained or loaded weights");
  }
  return BK_OK;
}

namespace {

bk_status check_dtype(bk_dtype d) {
  if (d != BK_F64 && d != BK_F32)
    return set_error(BK_ERR_INVALID_ARG, "dtype: unknown value %d", (int)d);
  return BK_OK;
}

bk_status check_theta(double sigma2, double beta, double nu) {
  if (!finite(sigma2) || sigma2 < 0.0)
    return set_error(BK_ERR_INVALID_ARG, "sigma2 must be finite and >= 0 (got %g)", sigma2);
  if (!finite(beta) || !(beta > 0.0))
    return set_error(BK_ERR_INVALID_ARG, "beta must be finite and > 0 (got %g)", beta);
  if (!finite(nu) || !(nu > 0.0))
    return set_error(BK_ERR_INVALID_ARG, "nu must be finite and > 0 (got %g)", nu);
  return BK_OK;
}

bk_status check_matrix(const void* out, int64_t rows, int64_t cols, int64_t ld) {
  if (rows < 0 || cols < 0) return set_error(BK_ERR_INVALID_ARG, "negative matrix size");
  if (rows == 0 || cols == 0) return BK_OK;
  if (out == nullptr) return set_error(BK_ERR_INVALID_ARG, "out is NULL");
  if (ld < rows) return set_error(BK_ERR_INVALID_ARG, "ld (%lld) < rows (%lld)", (long long)ld,
                                  (long long)rows);
  if (cols > INT64_MAX / ld) return set_error(BK_ERR_INVALID_ARG, "ld * cols overflows int64");
  return BK_OK;
}

}  // namespace
}  // namespace bk

using namespace bk;

extern "C" {

void bk_opts_default(bk_opts* o) {
  if (o == nullptr) return;
  std::memset(o, 0, sizeof(*o));
  o->window = BK_WIN_SEARCH;
  o->compute = BK_F64;
  o->fixed_bins = 40;
  o->fixed_t1 = 9.0;
  o->search_f64 = 0;
  o->series_below = 0.0;
  o->d_counters = nullptr;
  o->learned = nullptr;
  o->d_cosh_table = nullptr;
  o->lanes = 0;
}

const char* bk_version(void) { return "libbesselk 0.1.0 (sm_103a)"; }

const char* bk_last_error(void) { return g_err; }

const char* bk_status_string(bk_status s) {
  switch (s) {
    case BK_OK: return "BK_OK";
    case BK_ERR_INVALID_ARG: return "BK_ERR_INVALID_ARG";
    case BK_ERR_CUDA: return "BK_ERR_CUDA";
    case BK_ERR_NOMEM: return "BK_ERR_NOMEM";
    case BK_ERR_UNSUPPORTED: return "BK_ERR_UNSUPPORTED";
    case BK_ERR_NOT_CONVERGED: return "BK_ERR_NOT_CONVERGED";
    case BK_ERR_NOT_LOADED: return "BK_ERR_NOT_LOADED";
  }
  return "BK_UNKNOWN_STATUS";
}

bk_status bk_sync(bk_stream_t stream) {
  return check_cuda(cudaStreamSynchronize((cudaStream_t)stream), "bk_sync");
}

bk_status bk_eval_ex(const double* x, const double* nu, void* out, void* log_out,
                     bk_dtype out_dtype, int64_t n, const bk_opts* opts, bk_stream_t stream) {
  bk_opts o;
  bk_opts_default(&o);
  if (opts != nullptr) o = *opts;
  if (n < 0) return set_error(BK_ERR_INVALID_ARG, "n must be >= 0 (got %lld)", (long long)n);
  bk_status st = check_dtype(out_dtype);
  if (st != BK_OK) return st;
  if ((st = check_opts(&o)) != BK_OK) return st;
  if (n == 0) return BK_OK;
  if (x == nullptr || nu == nullptr || out == nullptr)
    return set_error(BK_ERR_INVALID_ARG, "x, nu and out must be non-NULL when n > 0");
  cudaStream_t s = (cudaStream_t)stream;
  const int lanes = eval_lanes(o, out_dtype);
  const cudaError_t e =
      (o.window == BK_WIN_LEARNED)
          ? launch_eval_learned(o.learned, x, nu, out, log_out, out_dtype, n, o.d_counters, s,
                                lanes)
      : (o.compute == BK_F64)
          ? launch_eval_f64(x, nu, out, log_out, out_dtype, n, o, s)
          : launch_eval_f32(x, nu, out, log_out, out_dtype, n, o.d_counters, s, lanes);
  return check_cuda(e, "bk_eval launch");
}

bk_status bk_eval_autotune(const double* x, const double* nu, void* out, bk_dtype out_dtype,
                           int64_t n, const bk_opts* opts, bk_stream_t stream, int* best_lanes) {
  bk_opts o;
  bk_opts_default(&o);
  if (opts != nullptr) o = *opts;
  if (o.compute != BK_F32 || o.window == BK_WIN_FIXED)
    return set_error(BK_ERR_UNSUPPORTED, "bk_eval_autotune: FP32 forms only (compute = BK_F32)");
  if (best_lanes == nullptr) return set_error(BK_ERR_INVALID_ARG, "best_lanes is NULL");
  if (n < 1) return set_error(BK_ERR_INVALID_ARG, "bk_eval_autotune needs n >= 1");
  const int64_t m = n < ((int64_t)1 << 20) ? n : ((int64_t)1 << 20);
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e != cudaSuccess) {
    if (a) cudaEventDestroy(a);
    return check_cuda(e, "bk_eval_autotune: cudaEventCreate");
  }
  int best = 0;
  float best_ms = 0.0f;
  bk_status st = BK_OK;
  for (int lanes : {1, 2, 4, 8}) {
    o.lanes = lanes;
    for (int rep = 0; rep < 4 && st == BK_OK; ++rep) {  // one warm-up, three timed
      if (rep == 1) cudaEventRecord(a, s);
      st = bk_eval_ex(x, nu, out, nullptr, out_dtype, m, &o, stream);
    }
    if (st != BK_OK) break;
    cudaEventRecord(b, s);
    e = cudaEventSynchronize(b);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e != cudaSuccess) {
      st = check_cuda(e, "bk_eval_autotune: timing");
      break;
    }
    if (best == 0 || ms < best_ms) {
      best = lanes;
      best_ms = ms;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (st != BK_OK) return st;
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64) {
    std::lock_guard<std::mutex> lk(g_lanes_mutex);
    g_eval_lanes[dev][o.window == BK_WIN_LEARNED ? 1 : 0][out_dtype == BK_F32 ? 1 : 0] = best;
  }
  *best_lanes = best;
  return BK_OK;
}

bk_status bk_eval_grad(const double* x, const double* nu, double* k, double* dk_dx,
                       double* dk_dnu, int64_t n, const bk_opts* opts, bk_stream_t stream) {
  bk_opts o;
  bk_opts_default(&o);
  if (opts != nullptr) o = *opts;
  if (n < 0) return set_error(BK_ERR_INVALID_ARG, "n must be >= 0 (got %lld)", (long long)n);
  bk_status st = check_opts(&o);
  if (st != BK_OK) return st;
  if (o.compute != BK_F64 || o.window != BK_WIN_SEARCH || o.series_below != 0.0)
    return set_error(BK_ERR_UNSUPPORTED, "bk_eval_grad: the plain form only (compute = BK_F64, "
                                         "window = BK_WIN_SEARCH, series_below = 0)");
  if (n == 0) return BK_OK;
  if (x == nullptr || nu == nullptr)
    return set_error(BK_ERR_INVALID_ARG, "x and nu must be non-NULL when n > 0");
  if (k == nullptr && dk_dx == nullptr && dk_dnu == nullptr)
    return set_error(BK_ERR_INVALID_ARG, "bk_eval_grad: all outputs are NULL");
  return check_cuda(launch_eval_grad_f64(x, nu, k, dk_dx, dk_dnu, n, o, (cudaStream_t)stream),
                    "bk_eval_grad launch");
}

bk_status bk_gaussian_loglik(double* a, int64_t n, int64_t ld, const double* z, double* y,
                             double* out, const bk_opts* opts, bk_stream_t stream) {
  bk_opts o;
  bk_opts_default(&o);
  if (opts != nullptr) o = *opts;
  bk_status st = check_opts(&o);
  if (st != BK_OK) return st;
  if (out == nullptr) return set_error(BK_ERR_INVALID_ARG, "out is NULL");
  if (n < 0) return set_error(BK_ERR_INVALID_ARG, "n must be >= 0 (got %lld)", (long long)n);
  cudaStream_t s = (cudaStream_t)stream;
  if (n == 0)
    return check_cuda(cudaMemsetAsync(out, 0, 3 * sizeof(double), s), "bk_gaussian_loglik");
  if ((st = check_matrix(a, n, n, ld)) != BK_OK) return st;
  if (z == nullptr || y == nullptr) return set_error(BK_ERR_INVALID_ARG, "z and y must be non-NULL");
  if (n > (int64_t)65535 * 64)
    return set_error(BK_ERR_INVALID_ARG, "n too large for the tile grid (max %lld)",
                     (long long)65535 * 64);
  return check_cuda(launch_loglik(a, n, ld, z, y, out, o.d_counters, s), "bk_gaussian_loglik");
}

bk_status bk_eval(const double* x, const double* nu, double* out, int64_t n, bk_stream_t stream) {
  return bk_eval_ex(x, nu, out, nullptr, BK_F64, n, nullptr, stream);
}

bk_status bk_matern_tile_ex(const double* locs, int64_t n, double sigma2, double beta, double nu,
                            void* out, int64_t ld, bk_dtype dtype, const bk_opts* opts,
                            bk_stream_t stream) {
  bk_opts o;
  bk_opts_default(&o);
  if (opts != nullptr) o = *opts;
  bk_status st;
  if ((st = check_dtype(dtype)) != BK_OK) return st;
  if ((st = check_theta(sigma2, beta, nu)) != BK_OK) return st;
  if ((st = check_matrix(out, n, n, ld)) != BK_OK) return st;
  if (opts == nullptr) o.compute = dtype;  // the output dtype picks the form by default
  if ((st = check_opts(&o)) != BK_OK) return st;
  if (n == 0) return BK_OK;
  if (locs == nullptr) return set_error(BK_ERR_INVALID_ARG, "locs is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  const cudaError_t e =
      (o.window == BK_WIN_LEARNED)
          ? launch_matern_sym_learned(o.learned, locs, n, sigma2, beta, nu, out, ld, dtype,
                                      o.d_counters, s)
      : (o.compute == BK_F64)
          ? launch_matern_sym_f64(locs, n, sigma2, beta, nu, out, ld, dtype, o, s)
          : launch_matern_sym_f32(locs, n, sigma2, beta, nu, out, ld, dtype, o.d_counters, s);
  return check_cuda(e, "bk_matern_tile launch");
}

bk_status bk_matern_tile(const double* locs, int64_t n, double sigma2, double beta, double nu,
                         void* out, int64_t ld, bk_dtype dtype, bk_stream_t stream) {
  return bk_matern_tile_ex(locs, n, sigma2, beta, nu, out, ld, dtype, nullptr, stream);
}

bk_status bk_matern_tile2(const double* locs1, int64_t m, const double* locs2, int64_t n,
                          double sigma2, double beta, double nu, void* out, int64_t ld,
                          bk_dtype dtype, const bk_opts* opts, bk_stream_t stream) {
  bk_opts o;
  bk_opts_default(&o);
  bk_status st;
  if ((st = check_dtype(dtype)) != BK_OK) return st;
  if (opts != nullptr) o = *opts; else o.compute = dtype;
  if ((st = check_theta(sigma2, beta, nu)) != BK_OK) return st;
  if ((st = check_matrix(out, m, n, ld)) != BK_OK) return st;
  if ((st = check_opts(&o)) != BK_OK) return st;
  if (m == 0 || n == 0) return BK_OK;
  if (locs1 == nullptr || locs2 == nullptr)
    return set_error(BK_ERR_INVALID_ARG, "locs1 and locs2 must be non-NULL");
  cudaStream_t s = (cudaStream_t)stream;
  const cudaError_t e =
      (o.window == BK_WIN_LEARNED)
          ? launch_matern_block_learned(o.learned, locs1, m, locs2, n, sigma2, beta, nu, out, ld,
                                        dtype, o.d_counters, s)
      : (o.compute == BK_F64)
          ? launch_matern_block_f64(locs1, m, locs2, n, sigma2, beta, nu, out, ld, dtype, o,
                                    s)
          : launch_matern_block_f32(locs1, m, locs2, n, sigma2, beta, nu, out, ld, dtype,
                                    o.d_counters, s);
  return check_cuda(e, "bk_matern_tile2 launch");
}

bk_status bk_morton_order(const double* locs, int64_t n, int64_t* perm) {
  if (n < 0) return set_error(BK_ERR_INVALID_ARG, "n must be >= 0");
  if (n == 0) return BK_OK;
  if (locs == nullptr || perm == nullptr)
    return set_error(BK_ERR_INVALID_ARG, "locs and perm must be non-NULL");
  std::vector<uint32_t> code((size_t)n);
  for (int64_t i = 0; i < n; ++i) {
    uint32_t q[2];
    for (int d = 0; d < 2; ++d) {
      double c = std::floor(locs[d * n + i] * 65536.0);
      if (!(c > 0.0)) c = 0.0;  // also maps NaN to 0
      if (c > 65535.0) c = 65535.0;
      q[d] = (uint32_t)c;
    }
    uint32_t z = 0;
    for (int b = 0; b < 16; ++b) {
      z |= ((q[0] >> b) & 1u) << (2 * b);
      z |= ((q[1] >> b) & 1u) << (2 * b + 1);
    }
    code[(size_t)i] = z;
  }
  std::iota(perm, perm + n, (int64_t)0);
  std::stable_sort(perm, perm + n, [&](int64_t a, int64_t b) { return code[(size_t)a] < code[(size_t)b]; });
  return BK_OK;
}

}  // extern "C"
