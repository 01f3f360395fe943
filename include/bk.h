/*
 * libbesselk: the modified Bessel function of the second kind K_nu(x) and the
 * Matern covariance matrices built on it, on one NVIDIA GB300 (sm_103a).
 *
 * Method (arXiv 2502.00356, Sec. IV-B): K_nu(x) is the integral of Eq.
 * (integral), K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt, evaluated in the
 * log domain of Eq. (logintegrand), g(t) = log cosh(nu t) - x cosh t, by a
 * trapezoid rule (Eq. (refined), weights multiplying the exponential) over
 * the peak-centred window [t0, t1] = {t : g(t) >= log(eps) + g(t_max)}.
 * The Matern entry is Sec. III-A's
 *   M(r) = sigma^2 / (2^{nu-1} Gamma(nu)) (r/beta)^nu K_nu(r/beta),
 * with M = sigma^2 where r == 0 (Algorithm 3).
 *
 * Conventions for every entry point:
 *  - Array arguments are DEVICE pointers owned by the caller, unless a
 *    parameter says "host".  Nothing is retained after the call returns.
 *  - Work is enqueued on `stream` (NULL = the legacy default stream) and the
 *    call returns without synchronising.  Kernel-side faults surface as
 *    BK_ERR_CUDA from a later call or from bk_sync().
 *  - Argument errors are detected on the host before any launch and return
 *    BK_ERR_INVALID_ARG; nothing is enqueued in that case.
 *  - bk_last_error() returns a thread-local message for the last failure.
 *  - Locations use the structure-of-arrays layout [x_0..x_{n-1}, y_0..y_{n-1}]
 *    (the paper passes the x and y vectors separately, Algorithm 3).
 *  - Matrices are column-major: entry (i, j) at out[i + j * ld], ld >= rows.
 *
 * Element-wise domain (both forms): x == 0 gives +inf; x < 0 or NaN gives
 * NaN; nu < 0 uses |nu| (K_{-nu} = K_nu, Eq. (integral) holds for real nu).
 * Accuracy is stated for x in [1e-3, 140], |nu| <= 20 (the region of Sec.
 * IV-C); other finite inputs are computed but not covered by that statement.
 * A point whose bounded root search does not converge gives NaN and, when
 * counters are supplied, increments BK_CTR_FAIL.
 */
#ifndef BESSELK_BK_H
#define BESSELK_BK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;
typedef struct CUstream_st* bk_stream_t; /* same type as cudaStream_t */

typedef enum {
  BK_OK = 0,
  BK_ERR_INVALID_ARG = 1,   /* rejected on the host, nothing launched */
  BK_ERR_CUDA = 2,          /* a CUDA runtime error (message in bk_last_error) */
  BK_ERR_NOMEM = 3,         /* a workspace or plan is too small */
  BK_ERR_UNSUPPORTED = 4,   /* option combination not available */
  BK_ERR_NOT_CONVERGED = 5, /* reserved for host-side iterative helpers */
  BK_ERR_NOT_LOADED = 6     /* the learned window has no weights */
} bk_status;

typedef enum { BK_F64 = 0, BK_F32 = 1 } bk_dtype;

/* How the integration window [t0, t1] and the node count are found. */
typedef enum {
  BK_WIN_SEARCH = 0,  /* per-point peak and bound search (Sec. IV-B) */
  BK_WIN_LEARNED = 1, /* predicted by the window network, checked, with fallback */
  BK_WIN_FIXED = 2    /* the paper's fixed [0, t1] with b bins and no search (Algorithm 2,
                         Sec. IV-C); plain FP64 form only */
} bk_window;

/* Indices into the optional device counter array bk_opts.d_counters. */
enum {
  BK_CTR_FALLBACK = 0, /* windows of a fast path (the learned network, or the plain
                          form's FP32 roots) replaced by the full window search */
  BK_CTR_FAIL = 1,     /* points returned as NaN because a search did not converge */
  BK_CTR_NODES = 2,    /* integrand evaluations (quadrature nodes) */
  BK_CTR_ITERS = 3,    /* window-end root-finder iterations */
  BK_CTR_EVALS = 4,    /* K_nu evaluations */
  BK_CTR_PEAK_ITERS = 5, /* peak (t_max) root-finder iterations */
  BK_CTR_REPAIR = 6,   /* learned window ends moved by one Newton step after the check */
  BK_CTR_SERIES = 7,   /* evaluations taken by Temme's series (bk_opts.series_below) */
  BK_NUM_COUNTERS = 8
};

typedef struct {
  bk_window window;  /* default BK_WIN_SEARCH */
  bk_dtype compute;  /* arithmetic of the integrand: BK_F64 (plain) or BK_F32 */
  int fixed_bins;    /* BK_WIN_FIXED: number of bins b, 1..100000 (paper: 40) */
  double fixed_t1;   /* BK_WIN_FIXED: upper bound, (0, 700] (paper: 9) */
  /* Optional device array of BK_NUM_COUNTERS unsigned 64-bit counters that
     kernels add to (never reset by the library).  NULL = no counting. */
  unsigned long long* d_counters;
  /* BK_WIN_LEARNED: the window network (trained or loaded); must outlive
     every call and plan that uses it. */
  const struct bk_learned* learned;
  /* Plain form (BK_F64, BK_WIN_SEARCH) only.  0 (default): the peak and the
     window ends are the FP32 roots of the bound F (inside x in [1e-4, 1e4],
     nu <= 40; widened by 2e-5 relative), and the window is checked in FP64
     on the quadrature's own end nodes (integrand below eps = 2^-52 times its
     peak value); a failing window is replaced by the FP64 search
     (BK_CTR_FALLBACK).  1: the FP64 Newton search from its own bounds for
     every point. */
  int search_f64;
  /* Plain form (BK_F64) only: x below which K_nu(x) comes from Temme's series
     with Campbell's forward recurrence (Sec. IV-A) instead of the integral;
     0 (default) = never, at most 2.  The paper's refined algorithm
     (Algorithm 2) is window = BK_WIN_FIXED, fixed_bins = 40, fixed_t1 = 9,
     series_below = 0.1.  Evaluations taken by the series are counted in
     BK_CTR_SERIES (their series terms in BK_CTR_NODES). */
  double series_below;
  /* Optional device scratch of BK_COSH_TABLE_LEN doubles for the plain
     form's Matern writers (bk_matern_tile_ex, bk_matern_tile2 with compute
     BK_F64 and the searched window): each call first fills it, on its
     stream, with e^{-2 nu h} over the quantised quadrature steps of the
     node loop (the ratio of its geometric factor e^{-2 nu t_j}), a per-call
     table that saves an accurate exponential (about 9 FP64 operations) per
     entry.  Caller-owned; one buffer must not serve two calls that can
     overlap on the GPU.  NULL (default): the kernels compute the values.
     No call allocates either way. */
  double* d_cosh_table;
  /* Bare evaluations (bk_eval_ex) of the FP32 forms only: lanes that share
     one evaluation's quadrature nodes, 1, 2, 4 or 8 (the node loops of a
     warp's 32 evaluations then run in `lanes` passes on groups of that many
     lanes, partial sums combined by a compensated shuffle reduction).
     0 (default): the choice bk_eval_autotune made for this device, form and
     output dtype in this process, else BK_EVAL_LANES_DEFAULT.  Other entry
     points ignore it (the Matern writers' warps evaluate 32 neighbouring
     entries of similar cost, one per lane). */
  int lanes;
} bk_opts;

/* lanes per evaluation when bk_opts.lanes is 0 and nothing was autotuned. */
#define BK_EVAL_LANES_DEFAULT 1

/* Length (doubles) of bk_opts.d_cosh_table. */
#define BK_COSH_TABLE_LEN 3328

/* Fills *o with the defaults: BK_WIN_SEARCH, BK_F64, b = 40, t1 = 9, no
   counters, no network, search_f64 = 0, series_below = 0, lanes = 0. */
void bk_opts_default(bk_opts* o);

const char* bk_version(void);
const char* bk_last_error(void);
const char* bk_status_string(bk_status s);

/* Waits for `stream` and reports any pending CUDA error as BK_ERR_CUDA. */
bk_status bk_sync(bk_stream_t stream);

/*
 * bk_eval: out[i] = K_{nu[i]}(x[i]) for i < n, FP64 in and out, the plain
 * FP64 form (per-point peak search, eps = 2^-52 window, self-checked
 * trapezoid).  Cites Eq. (integral), Eq. (logintegrand), Eq. (refined) and
 * the window of Sec. IV-B.  x, nu, out: device, n doubles each; out may alias
 * neither input.  n == 0 is a no-op; n < 0 or a NULL pointer with n > 0 is
 * BK_ERR_INVALID_ARG.
 */
bk_status bk_eval(const double* x, const double* nu, double* out, int64_t n, bk_stream_t stream);

/*
 * bk_eval_ex: as bk_eval with options.  out_dtype selects FP64 or FP32
 * output; opts == NULL means bk_opts_default.  With opts->compute == BK_F32
 * the integrand is evaluated in FP32 (the precision form).  When
 * `log_out` is non-NULL it receives log K_nu(x) in the same dtype (useful
 * where K_nu overflows, e.g. tiny x with large nu).
 */
bk_status bk_eval_ex(const double* x, const double* nu, void* out, void* log_out,
                     bk_dtype out_dtype, int64_t n, const bk_opts* opts, bk_stream_t stream);

/*
 * bk_eval_autotune: times bk_eval_ex of the FP32 forms (opts->compute =
 * BK_F32, searched or learned window) with 1, 2, 4 and 8 lanes per
 * evaluation on the first min(n, 2^20) pairs of the caller's x, nu (device,
 * as bk_eval_ex; out receives results), keeps the fastest for this device,
 * form and output dtype (used by later calls with opts->lanes == 0) and
 * returns it in *best_lanes (host).  The lane split is the multi-threaded
 * evaluation of K_nu that Sec. VI names as future work, on the node loop of
 * Algorithm 2.  Synchronises `stream`; allocates no device memory.  Errors:
 * BK_ERR_UNSUPPORTED for the FP64 forms, BK_ERR_INVALID_ARG as bk_eval_ex.
 */
bk_status bk_eval_autotune(const double* x, const double* nu, void* out, bk_dtype out_dtype,
                           int64_t n, const bk_opts* opts, bk_stream_t stream, int* best_lanes);

/* Derivatives of K_nu(x) with K itself, from one quadrature (not in the
 * paper; for gradient-based maximum likelihood): differentiating Eq.
 * (integral) of Sec. IV-B under the integral sign,
 *   dK/dx  = -int_0^inf cosh(t) e^{-x cosh t} cosh(nu t) dt,
 *   dK/dnu =  int_0^inf t sinh(nu t) e^{-x cosh t} dt,
 * evaluated on the nodes of the plain FP64 form over the union of the
 * eps-windows of the orders nu and nu + 1 (the dK/dx integrand decays like
 * that of K_{nu+1}).  x, nu: n FP64 values (device); k, dk_dx, dk_dnu: n FP64
 * outputs each (device), any of them NULL to skip.  Domain: x = 0 gives
 * (+inf, -inf, NaN), x = +inf gives zeros, x < 0, NaN or non-finite nu give
 * NaN; dK/dnu is odd in nu.  opts: only the plain form (compute BK_F64,
 * window BK_WIN_SEARCH, series_below 0; search_f64 and counters apply), else
 * BK_ERR_UNSUPPORTED.  Asynchronous on `stream`; allocates nothing. */
bk_status bk_eval_grad(const double* x, const double* nu, double* k, double* dk_dx,
                       double* dk_dnu, int64_t n, const bk_opts* opts, bk_stream_t stream);

/*
 * bk_matern_tile: the full n x n Matern matrix of `n` locations (Sec. III-A,
 * Algorithm 3), column-major with leading dimension ld >= n, written as
 * FP64 (dtype BK_F64, plain FP64 form) or FP32 (BK_F32, precision form).
 * Each unordered pair is evaluated once and written to (i, j) and (j, i);
 * the diagonal and any pair at distance exactly 0 get sigma^2.
 * locs: device, 2n doubles (SoA).  out: device, ld * n elements of dtype.
 * Requires sigma2 >= 0, beta > 0, nu > 0, all finite.  Asynchronous on
 * `stream`; allocates nothing (the options' d_cosh_table is the caller's).
 */
bk_status bk_matern_tile(const double* locs, int64_t n, double sigma2, double beta, double nu,
                         void* out, int64_t ld, bk_dtype dtype, bk_stream_t stream);

/* bk_matern_tile with options (window mode, counters). */
bk_status bk_matern_tile_ex(const double* locs, int64_t n, double sigma2, double beta, double nu,
                            void* out, int64_t ld, bk_dtype dtype, const bk_opts* opts,
                            bk_stream_t stream);

/*
 * bk_matern_tile2: the m x n block between row locations locs1 (m points) and
 * column locations locs2 (n points): out[i + j*ld] = M(|l2_j - l1_i|), the
 * single-tile kernel of Algorithm 3 (GenerateMaternCovariance(l1, l2, ...)).
 * ld >= m.  sigma^2 wherever the distance is exactly 0.
 */
bk_status bk_matern_tile2(const double* locs1, int64_t m, const double* locs2, int64_t n,
                          double sigma2, double beta, double nu, void* out, int64_t ld,
                          bk_dtype dtype, const bk_opts* opts, bk_stream_t stream);

/*
 * bk_matern_tile_host: the matrix of bk_matern_tile_ex delivered to HOST
 * memory, with the host <-> device transfers inside the call (Sec. III-A,
 * Algorithm 3; the paper's matrices are consumed by a host-side runtime).
 *   h_locs:  HOST, 2n doubles (SoA), copied into d_work on `stream`.
 *   h_out:   HOST, ld * n elements of dtype, column-major, ld >= n.
 *   mode:    BK_HOST_AUTO or BK_HOST_STAGED (below).
 *   d_work:  DEVICE workspace, 256-byte aligned, caller-owned; one workspace
 *            must not serve two calls that can overlap on the GPU.
 * BK_HOST_AUTO: when the device can address h_out (cudaHostGetDevicePointer
 * accepts it: page-locked memory from cudaHostAlloc, cudaMallocHost or
 * cudaHostRegister, and on GB300, whose GPU reaches host page tables through
 * ATS, pageable memory as well), the tile writer stores the matrix straight
 * into h_out over the GPU-CPU link (NVLink-C2C) and d_work needs only
 * bk_matern_tile_host_workspace(n, dtype, 0) bytes (locations and the plain
 * form's e^{-2 nu h} table).  Otherwise, and always with BK_HOST_STAGED,
 * the matrix is staged in d_work, which then needs
 * bk_matern_tile_host_workspace(n, dtype, 1) bytes: it is generated in up to
 * 16 panels of block-columns, and each finished panel's columns are copied to
 * h_out on a library-owned copy stream (one per device, created on first use
 * with its events) while later panels are generated; with pageable h_out each
 * copy blocks the calling thread until it is done.  Either way `stream` waits
 * for the last write to h_out before any later work: h_out is complete once
 * `stream` reaches the end of the call (e.g. after bk_sync(stream)).  Options
 * as bk_matern_tile_ex (opts == NULL: compute = dtype).  Not for stream
 * capture.  Allocates no device memory.  Errors: BK_ERR_INVALID_ARG for bad
 * sizes, parameters, mode, NULL pointers or an unaligned workspace;
 * BK_ERR_NOMEM when work_bytes is too small for the way h_out is written.
 */
enum { BK_HOST_AUTO = 0, BK_HOST_STAGED = 1 };
size_t bk_matern_tile_host_workspace(int64_t n, bk_dtype dtype, int staged);
bk_status bk_matern_tile_host(const double* h_locs, int64_t n, double sigma2, double beta,
                              double nu, void* h_out, int64_t ld, bk_dtype dtype,
                              const bk_opts* opts, int mode, void* d_work, size_t work_bytes,
                              bk_stream_t stream);

/*
 * bk_morton_order (host only): perm[k] = index of the k-th location in
 * Z-order (Sec. IV-D orders locations so that a tile holds nearby points).
 * Coordinates are quantised to 16 bits over [0, 1] (clamped), x on the even
 * bits and y on the odd bits, ties keep their input order.
 * locs: HOST, 2n doubles (SoA).  perm: HOST, n int64.
 */
bk_status bk_morton_order(const double* locs, int64_t n, int64_t* perm);

/*
 * Batched persistent form.  A maximum-likelihood sweep regenerates many
 * covariance matrices of uneven n with per-instance (sigma^2, beta, nu)
 * every likelihood evaluation (Sec. III-A; the paper accelerates exactly this
 * step of the MLE loop).  bk_matern_batched builds all of them in ONE
 * persistent launch: CTAs take lower-triangle tiles of any instance from a
 * device counter.  The plan (created once per list of sizes) owns the work
 * list and that counter; the call itself allocates nothing and does not
 * synchronise, so it can be captured in a CUDA graph.  Calls that use the
 * same plan must not overlap on the GPU (they share the counter).
 */
typedef struct {
  const double* locs; /* device, 2n doubles (SoA) */
  int64_t n;          /* must equal the plan's size for this instance */
  double sigma2, beta, nu;
  void* out;          /* device, ld * n elements of the batch dtype, column-major */
  int64_t ld;         /* >= n */
} bk_matern_desc;

typedef struct bk_plan bk_plan;

/* sizes: HOST array of `count` instance sizes.  dtype: output dtype of every
   instance; opts (may be NULL) selects the form (default: compute = dtype).
   Allocates the plan's device work list; picks a launch shape from the
   autotune cache when one exists for this GPU, dtype, form and size bucket. */
bk_status bk_batched_plan_create(bk_plan** plan, const int64_t* sizes, int32_t count,
                                 bk_dtype dtype, const bk_opts* opts);
bk_status bk_batched_plan_destroy(bk_plan* plan);
/* Reports the work list size and the launch shape (any output may be NULL). */
bk_status bk_batched_plan_info(const bk_plan* plan, int64_t* total_tiles, int* warps,
                               int* ctas_per_sm, int* chunk, int* tuned);
/* Times launch shapes (warps per CTA, CTAs per SM, tiles per grab) on the
   first `sample_tiles` tiles (<= 0: all) of the caller's batch, keeps the
   fastest in the plan and appends it to the cache file ($BK_AUTOTUNE_CACHE,
   else $XDG_CACHE_HOME or ~/.cache /libbesselk/autotune.txt).  Writes into the
   instances' outputs and synchronises `stream`. */
bk_status bk_batched_autotune(bk_plan* plan, const bk_matern_desc* d_descs, int64_t sample_tiles,
                              bk_stream_t stream);
/* d_descs: DEVICE array of `count` descriptors (caller-owned).  A descriptor
   that does not match the plan (n, ld < n, NULL pointers, beta or nu <= 0,
   sigma2 < 0) is skipped in-kernel and counted in BK_CTR_FAIL when the
   plan's opts supplied counters. */
bk_status bk_matern_batched(const bk_matern_desc* d_descs, int32_t count, bk_dtype dtype,
                            const bk_plan* plan, bk_stream_t stream);

/*
 * Learned window (not in the paper; the window search of Sec. IV-B is the
 * part it replaces).  A 2 -> 64 -> 64 -> 64 -> 4 tanh network maps
 * (ln x, nu) to (t*, t* - t0, t1 - t*, ln N) of the eps = 2^-23 window.  It is
 * trained on the GPU by this library's kernels (bk_learned_train) on labels
 * from a bounds search, and used through bk_opts.window = BK_WIN_LEARNED with
 * compute = BK_F32: the network is tabulated on a 512 x 256 grid over
 * ln x in [ln 1e-3, ln 140] and nu in [0.05, 20] after every training or
 * load, kernels interpolate the table, widen the window by a relative and an
 * absolute margin and check it (the integrand at both ends must be below
 * eps times its value at the predicted peak, checked with an upper bound of
 * g).  An end that fails is moved by one Newton step of the bounds search
 * from the prediction (BK_CTR_REPAIR); points outside the grid, or whose
 * slope does not allow that step, use the full window search
 * (BK_CTR_FALLBACK).
 */
typedef struct bk_learned bk_learned;

/* Allocates a network with Glorot-uniform weights drawn from `seed`
   (synchronises the device). */
bk_status bk_learned_create(bk_learned** model, uint64_t seed);
bk_status bk_learned_destroy(bk_learned* model);
/* Adam steps (learning rate decayed by a cosine from lr to lr/20 over the
   call) on mini-batches of `batch` samples (a multiple of 128) drawn with
   replacement by a counter-based hash of (seed, step).  Data (device,
   caller-owned): x[n], nu[n] and labels[n][6] = (t*, t0, t1, g(t*), N, any),
   as written by the oracle's label script.  The target mean and standard
   deviation are taken from this data on the first call.  d_loss (device,
   optional): receives the mean squared error of each step.  Rebuilds the
   table at the end.  Enqueued on `stream`. */
bk_status bk_learned_train(bk_learned* model, const double* d_x, const double* d_nu,
                           const double* d_labels, int64_t n, int32_t steps, int32_t batch,
                           float lr, uint64_t seed, float* d_loss, bk_stream_t stream);
/* The kernel of each training step (bk_learned_train, bk_learned_grad).
   BK_TRAIN_TENSOR (the default): the products of the two 64 x 64 hidden
   layers in the forward and backward passes and their weight gradients run
   as tcgen05 MMAs on the tensor cores, TF32 operands (10 significand bits)
   with FP32 accumulation, from shared memory into tensor memory; the other
   layers, tanh and the bias gradients on the FP32 pipes.  A step whose wait
   for its MMAs gives up (a bounded wait) leaves its gradient incomplete and
   sets an error that the next bk_learned_params(get) returns as BK_ERR_CUDA.
   BK_TRAIN_SIMT: the whole step in FP32 on the FP32 pipes.  Errors:
   BK_ERR_INVALID_ARG for another value or a NULL model. */
enum { BK_TRAIN_TENSOR = 0, BK_TRAIN_SIMT = 1 };
bk_status bk_learned_set_train_path(bk_learned* model, int path);
/* Full-batch gradient of the training loss over samples 0 .. n-1 (n a
   multiple of 128) into d_grad[8772] (device), and the loss into *d_loss. */
bk_status bk_learned_grad(bk_learned* model, const double* d_x, const double* d_nu,
                          const double* d_labels, int64_t n, float* d_grad, float* d_loss,
                          bk_stream_t stream);
/* Per-point network outputs: d_out[4 i ..] = (t*, t0, t1, N) for (x[i], nu[i]). */
bk_status bk_learned_infer(const bk_learned* model, const double* d_x, const double* d_nu,
                           float* d_out, int64_t n, bk_stream_t stream);
/* Host copies of the 8772 parameters (get and/or set; set rebuilds the table)
   and of the 8 target statistics (mean[4], std[4]); synchronising. */
bk_status bk_learned_params(bk_learned* model, float* h_get, const float* h_set);
bk_status bk_learned_stats(bk_learned* model, float* h_get8, const float* h_set8);
/* Relative and absolute window margins (defaults 0.05 and 0.02). */
bk_status bk_learned_set_margins(bk_learned* model, float rel, float abs_margin);
/* Checkpoint with parameters, Adam state, step count and target statistics,
   guarded by a checksum; load resumes training where save left it. */
bk_status bk_learned_save(const bk_learned* model, const char* path);
bk_status bk_learned_load(bk_learned* model, const char* path);

/*
 * bk_matern_batched_static: the work of bk_matern_batched without a plan and
 * without allocating anything.  The paper has no counterpart; this entry
 * point exists for callers that cannot call cudaMalloc where they build their
 * matrices: code inside a framework that owns all device memory through its
 * own pool allocator (an extra cudaMalloc may fail or stall other streams),
 * and real-time or embedded services that forbid allocation after start-up.
 * Its scratch (work list and tile counter) is a fixed array compiled into the
 * library, held by every GPU that loads the library until the process exits;
 * it fits at most 4096 instances (count > 4096 is BK_ERR_INVALID_ARG).
 * Every call looks up that array's device address on the current device
 * (cudaGetSymbolAddress; the first call on a device also loads the library's
 * device code there), so make the first call on each device before any
 * stream capture.  All calls share the one array and each call rewrites it
 * (work list, counter zeroed) before use: calls that can overlap on the GPU
 * (other streams, other host threads) race with each other and must be
 * ordered by the caller.  Descriptors as for bk_matern_batched; dtype picks
 * the output type and the form (compute = dtype).  There are no counters on
 * this path: an invalid descriptor (n < 0, ld < n, NULL pointers, beta or
 * nu <= 0, sigma2 < 0) is skipped without a report and its output is left
 * untouched.  The FP64 form here computes e^{-2 nu h} once per entry (a plan
 * keeps per-instance tables of it), so it is somewhat slower than
 * bk_matern_batched with a plan.  Launch shape fixed (8 warps, 2 CTAs per
 * SM).  Enqueues two kernels on `stream` and does not synchronise.
 */
bk_status bk_matern_batched_static(const bk_matern_desc* d_descs, int32_t count, bk_dtype dtype,
                                   bk_stream_t stream);

/* Gaussian log-likelihood of observations z under the covariance matrix a
 * (the step that consumes the generated matrix in the maximum-likelihood
 * loop the paper accelerates, Sec. II; not part of the paper's method):
 *   l = -1/2 (z^T a^{-1} z + log det a + n log 2 pi),
 * by an in-place blocked Cholesky a = L L^T in FP64 (64 x 64 tiles),
 * log det a = 2 sum log L_ii and the forward substitution L y = z
 * (z^T a^{-1} z = y^T y).
 *   a:   n x n column-major FP64 (device), ld >= n; only the lower triangle
 *        is read, and it is overwritten by L (the upper triangle is untouched)
 *   z:   n FP64 observations (device, read only)
 *   y:   n FP64 workspace (device); receives L^{-1} z
 *   out: 3 FP64 (device): [l, log det a, z^T a^{-1} z]
 * A matrix that is not positive definite (a pivot <= 0) gives NaN in out and
 * adds 1 to BK_CTR_FAIL when opts carries counters (other options are
 * ignored).  n = 0 writes zeros.  n <= 65535 * 64.  Asynchronous on
 * `stream` (about 5 launches per 64 rows); allocates nothing. */
bk_status bk_gaussian_loglik(double* a, int64_t n, int64_t ld, const double* z, double* y,
                             double* out, const bk_opts* opts, bk_stream_t stream);

/*
 * bk_probe_pipe: throughput probe for the roofline denominators (not part of
 * the paper's method).  Launches grid x block threads; each runs `iters`
 * trips of 8 independent operations on one pipe: kind 0 = FP64 FMA,
 * 1 = FP32 FMA, 2 = ex2.approx.f32 on the MUFU unit, 3 = FP64 -> FP32
 * conversion, 4 = FP32 -> FP64 conversion (each chained through integer
 * operations).  Operations per launch = grid * block * iters * 8.  sink:
 * device, grid * block doubles (written).
 */
bk_status bk_probe_pipe(int kind, int64_t iters, int grid, int block, double* sink,
                        bk_stream_t stream);

/*
 * bk_math_probe: evaluates one of the plain form's device math helpers on n
 * inputs, as the kernels compute it (a test hook for those helpers, not part
 * of the paper's method).  fn:
 *   0  e^a by the final normalisations' exponential (any a; |a| >= 708 takes
 *      the range-checked path)
 *   1  log a for finite a > 0 (subnormals included)
 *   2  2^{u/4096} by the centred node loop's exponential, |u| < 2^22
 *   3  2^{-D/4096} by the uncentred node loop's exponential of a node
 *      exponent in fixed point (fix40_node, exp2s_fix), 0.25 <= D < 2^22
 *   4  round(v) and v - round(v) for 0 <= v < 2^22 (halves round up), taken
 *      on the integer pipe: out[2i] = round(v), out[2i + 1] = the remainder
 *   5  2 cosh v for v >= 0 (the series tiers and the exponential path)
 *   6  sqrt a for a > 0
 *   7  e^a by the accurate set-up exponential, |a| < 708
 *   8  e^a by the Matern entries' final exponential on the integer pipe,
 *      exp_units_full(a 4096/ln 2) (any a; |a| >= 707.4 takes the
 *      range-checked path)
 *   9  log a from the Matern entries' log parts (nd and log1p(d) on the
 *      integer pipe), assembled as nd ln2/4096 + log1p(d), finite a > 0
 *  10  sqrt a by the Matern entries' integer-pipe square root, a > 0
 *  11  2^{-U/4096} by the same exponential for U = round(a 2^40) 2^-40,
 *      -4.09e6 < a < 4.09e6 (signed: the node loop's D_j - G_j)
 *  12  1 + w by the node loop's fixed-point geometric factor (w in units of
 *      2^-63, truncated, then rounded to a double), 0 <= w <= 1
 *  13  r truncated to units of 2^-64 (clamped below 2^64), as a double,
 *      0 <= r <= 1
 * in: device, n doubles; out: device, n doubles (2n for fn 4).  Inputs
 * outside a function's stated domain give unspecified values (no fault).
 * Errors: BK_ERR_INVALID_ARG for an unknown fn, n < 0 or null pointers with
 * n > 0.
 */
bk_status bk_math_probe(int fn, const double* in, double* out, int64_t n, bk_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* BESSELK_BK_H */
