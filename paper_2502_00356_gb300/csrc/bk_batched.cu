// Batched persistent Matern writer (a maximum-likelihood parameter sweep
// issues many covariance matrices of uneven n with per-instance
// (sigma^2, beta, nu); Sec. III-A motivates regenerating them every
// likelihood evaluation).  One launch covers every lower-triangle tile of
// every instance: CTAs take tiles from a device counter, so instances of any
// size share the machine without a launch per matrix.  The plan owns the
// work list (tile prefix sums per instance) and the counter; the hot call is
// one memset + one launch, both capturable in a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cerrno>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <sys/stat.h>
#include <vector>

#include "bk_internal.h"
#include "bk_forms.cuh"
#include "bk_tiles.cuh"

namespace bk {

// Work item w (a global tile number) -> instance k with prefix[k] <= w < prefix[k+1].
__device__ __forceinline__ int find_instance(const int64_t* __restrict__ prefix, int count,
                                             int64_t w) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(prefix + mid) <= w) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <typename OutT>
struct BatchSmem {
  SymTileSmem<OutT> tile;
  const double* locs;
  OutT* out;
  int64_t n, ld, item;
  MaternParams mp;
  const double* wnu;  // the instance's table of e^{-2 nu h}, or null
};

// Persistent kernel: each CTA repeatedly takes `chunk` consecutive tiles from
// *next (scratch, zeroed before the launch) until `limit` tiles are taken.
template <class Form, typename OutT, int WARPS>
__global__ void __launch_bounds__(WARPS * 32, Form::kMinBlocks * 8 / WARPS) matern_batched_kernel(
    const Form form, const bk_matern_desc* __restrict__ descs, int count, const int64_t* __restrict__ prefix,
    const int64_t* __restrict__ sizes, int64_t limit, unsigned long long* __restrict__ next,
    int chunk, unsigned long long* __restrict__ ctr, const double* __restrict__ wnu_tabs) {
  __shared__ BatchSmem<OutT> sm;
  __shared__ double s_tab[Form::kStageTable ? kExpTabSize : 1];
  const Form f = bind_table(form, s_tab);
  Tally tl{0u, 0u, 0u, 0u, 0u, 0u, 0u};
  unsigned evals = 0;
  int cur = -1;
  while (true) {
    __syncthreads();  // shared data of the previous round is no longer read
    if (threadIdx.x == 0) sm.item = (int64_t)atomicAdd(next, (unsigned long long)chunk);
    __syncthreads();
    const int64_t base = sm.item;
    if (base >= limit) break;
    const int64_t end = min(base + (int64_t)chunk, limit);
    for (int64_t w = base; w < end; ++w) {
      const int k = find_instance(prefix, count, w);
      if (k != cur) {
        __syncthreads();
        if (threadIdx.x == 0) {
          bk_matern_desc d = descs[k];
          // a descriptor that does not match the plan is skipped (n = 0) and counted
          const bool ok = d.n == __ldg(sizes + k) && d.ld >= d.n && d.locs != nullptr &&
                          d.out != nullptr && d.beta > 0.0 && d.nu > 0.0 && d.sigma2 >= 0.0;
          if (!ok) {
            d.n = 0;
            if (ctr != nullptr) atomicAdd(ctr + BK_CTR_FAIL, 1ull);
          }
          sm.locs = d.locs;
          sm.out = (OutT*)d.out;
          sm.n = d.n;
          sm.ld = d.ld;
          sm.mp = matern_params(d.sigma2, d.beta, d.nu);  // a1, once per instance run
          sm.wnu = (wnu_tabs != nullptr) ? wnu_tabs + (int64_t)k * kCoshTabSize : nullptr;
        }
        __syncthreads();
        cur = k;
      }
      int64_t I, J;
      tri_tile(w - __ldg(prefix + k), I, J);
      __syncthreads();
      if constexpr (Form::kDecayTable) {
        Form fk = f;
        fk.wnu = sm.wnu;
        sym_tile<Form, OutT, WARPS>(fk, sm.tile, sm.locs, sm.n, I, J, sm.mp, sm.out, sm.ld, tl,
                                    evals);
      } else {
        sym_tile<Form, OutT, WARPS>(f, sm.tile, sm.locs, sm.n, I, J, sm.mp, sm.out, sm.ld, tl,
                                    evals);
      }
    }
  }
  flush_tally(ctr, tl, evals);
}

// Fills each instance's table of e^{-2 nu h} on kCoshTab's steps from its
// descriptor's nu (instances with a bad descriptor are skipped by the tile
// kernel whatever their table holds).
__global__ void __launch_bounds__(256) batched_decay_kernel(const bk_matern_desc* __restrict__ descs,
                                                              int count, double* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)count * kCoshTabSize) return;
  const int k = (int)(i / kCoshTabSize), j = (int)(i % kCoshTabSize);
  const double nu = descs[k].nu;
  out[i] = decay_entry(nu > 0.0 ? nu : 0.0, j, kExp2Tab);
}

}  // namespace bk

// ---------------------------------------------------------------------------
// Plan and launch (host)

struct bk_plan {
  int device;
  int32_t count;
  bk_dtype dtype;
  bk_opts opts;
  int64_t total_tiles;
  int64_t* d_prefix;               // count + 1 tile offsets (device)
  int64_t* d_sizes;                // count instance sizes (device)
  unsigned long long* d_next;      // tile counter (device scratch)
  double* d_wnu;                   // count x kCoshTabSize: e^{-2 nu h} per instance, or null
  int warps, ctas_per_sm, chunk;   // launch shape
  int tuned;                       // 1 when the shape came from the autotuner or its cache
  double tuned_ms;
  std::string key;
};

namespace bk {
namespace {

template <class Form>
Form make_form(const bk_plan*) { return Form{}; }
template <>
FormF64 make_form<FormF64>(const bk_plan* p) {
  return FormF64{nullptr, p->opts.search_f64 != 0, 0.0};
}
template <>
FormF64Series make_form<FormF64Series>(const bk_plan* p) {
  return FormF64Series{nullptr, p->opts.search_f64 != 0, p->opts.series_below};
}
template <>
FormF64Fixed make_form<FormF64Fixed>(const bk_plan* p) {
  return FormF64Fixed{nullptr, p->opts.fixed_t1, p->opts.fixed_bins, p->opts.series_below};
}
template <>
FormF32Learned make_form<FormF32Learned>(const bk_plan* p) {
  return FormF32Learned{learned_view(p->opts.learned)};
}

template <class Form, typename OutT, int WARPS>
cudaError_t launch_batched_t(const bk_plan* p, const bk_matern_desc* d, int64_t limit,
                             int ctas_per_sm, int chunk, cudaStream_t s) {
  const int grid = current_sm_count() * ctas_per_sm;
  matern_batched_kernel<Form, OutT, WARPS><<<grid, WARPS * 32, 0, s>>>(
      make_form<Form>(p), d, p->count, p->d_prefix, p->d_sizes, limit, p->d_next, chunk, p->opts.d_counters,
      Form::kDecayTable ? p->d_wnu : nullptr);
  return cudaGetLastError();
}

template <class Form, typename OutT>
cudaError_t launch_batched_w(const bk_plan* p, const bk_matern_desc* d, int64_t limit, int warps,
                             int ctas_per_sm, int chunk, cudaStream_t s) {
  if (warps == 4) return launch_batched_t<Form, OutT, 4>(p, d, limit, ctas_per_sm, chunk, s);
  return launch_batched_t<Form, OutT, 8>(p, d, limit, ctas_per_sm, chunk, s);
}

cudaError_t launch_batched(const bk_plan* p, const bk_matern_desc* d, int64_t limit, int warps,
                           int ctas_per_sm, int chunk, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(p->d_next, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  if (p->d_wnu != nullptr) {
    const int64_t cells = (int64_t)p->count * kCoshTabSize;
    batched_decay_kernel<<<(unsigned)((cells + 255) / 256), 256, 0, s>>>(d, p->count, p->d_wnu);
  }
  const bool f64 = (p->opts.compute == BK_F64);
  const bool learned = (p->opts.window == BK_WIN_LEARNED);
  if (p->opts.window == BK_WIN_FIXED)
    return (p->dtype == BK_F64)
               ? launch_batched_w<FormF64Fixed, double>(p, d, limit, warps, ctas_per_sm, chunk, s)
               : launch_batched_w<FormF64Fixed, float>(p, d, limit, warps, ctas_per_sm, chunk, s);
  if (f64 && p->opts.series_below > 0.0)
    return (p->dtype == BK_F64)
               ? launch_batched_w<FormF64Series, double>(p, d, limit, warps, ctas_per_sm, chunk, s)
               : launch_batched_w<FormF64Series, float>(p, d, limit, warps, ctas_per_sm, chunk, s);
  if (p->dtype == BK_F64) {
    if (learned)
      return launch_batched_w<FormF32Learned, double>(p, d, limit, warps, ctas_per_sm, chunk, s);
    return f64 ? launch_batched_w<FormF64, double>(p, d, limit, warps, ctas_per_sm, chunk, s)
               : launch_batched_w<FormF32, double>(p, d, limit, warps, ctas_per_sm, chunk, s);
  }
  if (learned)
    return launch_batched_w<FormF32Learned, float>(p, d, limit, warps, ctas_per_sm, chunk, s);
  return f64 ? launch_batched_w<FormF64, float>(p, d, limit, warps, ctas_per_sm, chunk, s)
             : launch_batched_w<FormF32, float>(p, d, limit, warps, ctas_per_sm, chunk, s);
}

int max_ctas_per_sm(const bk_plan* p, int warps) {
  int blocks = 0;
  const void* fn = nullptr;
  const bool f64 = (p->opts.compute == BK_F64);
  if (p->opts.window == BK_WIN_FIXED) {
    if (p->dtype == BK_F64)
      fn = (warps == 4) ? (const void*)matern_batched_kernel<FormF64Fixed, double, 4>
                        : (const void*)matern_batched_kernel<FormF64Fixed, double, 8>;
    else
      fn = (warps == 4) ? (const void*)matern_batched_kernel<FormF64Fixed, float, 4>
                        : (const void*)matern_batched_kernel<FormF64Fixed, float, 8>;
  } else if (f64 && p->opts.series_below > 0.0) {
    if (p->dtype == BK_F64)
      fn = (warps == 4) ? (const void*)matern_batched_kernel<FormF64Series, double, 4>
                        : (const void*)matern_batched_kernel<FormF64Series, double, 8>;
    else
      fn = (warps == 4) ? (const void*)matern_batched_kernel<FormF64Series, float, 4>
                        : (const void*)matern_batched_kernel<FormF64Series, float, 8>;
  } else if (p->opts.window == BK_WIN_LEARNED) {
    if (p->dtype == BK_F64)
      fn = (warps == 4) ? (const void*)matern_batched_kernel<FormF32Learned, double, 4>
                        : (const void*)matern_batched_kernel<FormF32Learned, double, 8>;
    else
      fn = (warps == 4) ? (const void*)matern_batched_kernel<FormF32Learned, float, 4>
                        : (const void*)matern_batched_kernel<FormF32Learned, float, 8>;
  } else if (p->dtype == BK_F64) {
    if (warps == 4) fn = f64 ? (const void*)matern_batched_kernel<FormF64, double, 4>
                             : (const void*)matern_batched_kernel<FormF32, double, 4>;
    else fn = f64 ? (const void*)matern_batched_kernel<FormF64, double, 8>
                  : (const void*)matern_batched_kernel<FormF32, double, 8>;
  } else {
    if (warps == 4) fn = f64 ? (const void*)matern_batched_kernel<FormF64, float, 4>
                             : (const void*)matern_batched_kernel<FormF32, float, 4>;
    else fn = f64 ? (const void*)matern_batched_kernel<FormF64, float, 8>
                  : (const void*)matern_batched_kernel<FormF32, float, 8>;
  }
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fn, warps * 32, 0) != cudaSuccess)
    return 1;
  return std::max(1, blocks);
}

// ---- autotune cache: one line per key: "<key> <warps> <ctas_per_sm> <chunk> <ms>"
std::mutex g_cache_mutex;

std::string cache_path() {
  const char* env = std::getenv("BK_AUTOTUNE_CACHE");
  if (env != nullptr) return std::string(env);
  const char* xdg = std::getenv("XDG_CACHE_HOME");
  const char* home = std::getenv("HOME");
  std::string dir;
  if (xdg != nullptr && *xdg) dir = std::string(xdg) + "/libbesselk";
  else if (home != nullptr && *home) dir = std::string(home) + "/.cache/libbesselk";
  else return std::string();
  return dir + "/autotune.txt";
}

bool cache_lookup(const std::string& key, int& warps, int& cps, int& chunk, double& ms) {
  std::lock_guard<std::mutex> lk(g_cache_mutex);
  const std::string path = cache_path();
  if (path.empty()) return false;
  FILE* f = std::fopen(path.c_str(), "r");
  if (f == nullptr) return false;
  char kbuf[256];
  int w, c, ch;
  double m;
  bool found = false;
  while (std::fscanf(f, "%255s %d %d %d %lf", kbuf, &w, &c, &ch, &m) == 5) {
    if (key == kbuf) {  // the last entry for a key wins
      warps = w;
      cps = c;
      chunk = ch;
      ms = m;
      found = true;
    }
  }
  std::fclose(f);
  return found;
}

void cache_store(const std::string& key, int warps, int cps, int chunk, double ms) {
  std::lock_guard<std::mutex> lk(g_cache_mutex);
  const std::string path = cache_path();
  if (path.empty()) return;
  const size_t slash = path.find_last_of('/');
  if (slash != std::string::npos) {  // create the directory chain (best effort)
    std::string dir = path.substr(0, slash);
    for (size_t pos = 1; pos <= dir.size(); ++pos)
      if (pos == dir.size() || dir[pos] == '/') mkdir(dir.substr(0, pos).c_str(), 0755);
  }
  FILE* f = std::fopen(path.c_str(), "a");
  if (f == nullptr) return;
  std::fprintf(f, "%s %d %d %d %.6f\n", key.c_str(), warps, cps, chunk, ms);
  std::fclose(f);
}

std::string make_key(const bk_plan* p) {
  cudaDeviceProp prop;
  std::string name = "gpu";
  if (cudaGetDeviceProperties(&prop, p->device) == cudaSuccess) name = prop.name;
  for (char& c : name)
    if (c == ' ') c = '_';
  int bucket = 0;
  while ((1LL << bucket) < p->total_tiles) ++bucket;
  char buf[256];
  std::snprintf(buf, sizeof(buf), "%s|out%d|compute%d|win%d|tiles2^%d", name.c_str(),
                (int)p->dtype, (int)p->opts.compute, (int)p->opts.window, bucket);
  return std::string(buf);
}

}  // namespace
}  // namespace bk

using namespace bk;

extern "C" {

bk_status bk_batched_plan_create(bk_plan** plan, const int64_t* sizes, int32_t count,
                                 bk_dtype dtype, const bk_opts* opts) {
  if (plan == nullptr) return set_error(BK_ERR_INVALID_ARG, "plan is NULL");
  *plan = nullptr;
  if (count < 1) return set_error(BK_ERR_INVALID_ARG, "count must be >= 1");
  if (sizes == nullptr) return set_error(BK_ERR_INVALID_ARG, "sizes is NULL");
  if (dtype != BK_F64 && dtype != BK_F32)
    return set_error(BK_ERR_INVALID_ARG, "dtype: unknown value %d", (int)dtype);
  bk_opts o;
  bk_opts_default(&o);
  if (opts != nullptr) o = *opts; else o.compute = dtype;
  const bk_status st = check_opts(&o);
  if (st != BK_OK) return st;
  std::vector<int64_t> prefix((size_t)count + 1, 0);
  for (int32_t k = 0; k < count; ++k) {
    if (sizes[k] < 0) return set_error(BK_ERR_INVALID_ARG, "sizes[%d] < 0", (int)k);
    const int64_t nb = (sizes[k] + kTile - 1) / kTile;
    prefix[(size_t)k + 1] = prefix[(size_t)k] + nb * (nb + 1) / 2;
  }
  bk_plan* p = new bk_plan();
  p->count = count;
  p->dtype = dtype;
  p->opts = o;
  p->total_tiles = prefix.back();
  p->d_prefix = nullptr;
  p->d_sizes = nullptr;
  p->d_next = nullptr;
  p->d_wnu = nullptr;
  p->warps = 8;
  p->chunk = 1;
  p->tuned = 0;
  p->tuned_ms = 0.0;
  cudaError_t e = cudaGetDevice(&p->device);
  if (e == cudaSuccess) e = cudaMalloc((void**)&p->d_prefix, prefix.size() * sizeof(int64_t));
  if (e == cudaSuccess) e = cudaMalloc((void**)&p->d_sizes, (size_t)count * sizeof(int64_t));
  if (e == cudaSuccess) e = cudaMalloc((void**)&p->d_next, sizeof(unsigned long long));
  if (e == cudaSuccess)
    e = cudaMemcpy(p->d_prefix, prefix.data(), prefix.size() * sizeof(int64_t),
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(p->d_sizes, sizes, (size_t)count * sizeof(int64_t), cudaMemcpyHostToDevice);
  // per-instance tables of e^{-2 nu h} for the searched-window FP64 forms
  // (without them, or for more than 4,096 instances, the kernel computes the
  // values itself)
  if (e == cudaSuccess && o.compute == BK_F64 && o.window != BK_WIN_FIXED &&
      o.window != BK_WIN_LEARNED && count <= 4096) {
    if (cudaMalloc((void**)&p->d_wnu, (size_t)count * kCoshTabSize * sizeof(double)) != cudaSuccess) {
      (void)cudaGetLastError();
      p->d_wnu = nullptr;
    }
  }
  if (e != cudaSuccess) {
    cudaFree(p->d_prefix);
    cudaFree(p->d_sizes);
    cudaFree(p->d_next);
    delete p;
    return (e == cudaErrorMemoryAllocation) ? set_error(BK_ERR_NOMEM, "plan: out of device memory")
                                            : check_cuda(e, "bk_batched_plan_create");
  }
  p->ctas_per_sm = std::min(2, max_ctas_per_sm(p, p->warps));
  p->key = make_key(p);
  int w, c, ch;
  double ms;
  if (cache_lookup(p->key, w, c, ch, ms) && (w == 4 || w == 8) && c >= 1 && ch >= 1 &&
      c <= max_ctas_per_sm(p, w)) {
    p->warps = w;
    p->ctas_per_sm = c;
    p->chunk = ch;
    p->tuned = 1;
    p->tuned_ms = ms;
  }
  *plan = p;
  return BK_OK;
}

bk_status bk_batched_plan_destroy(bk_plan* plan) {
  if (plan == nullptr) return BK_OK;
  cudaFree(plan->d_prefix);
  cudaFree(plan->d_sizes);
  cudaFree(plan->d_next);
  cudaFree(plan->d_wnu);
  delete plan;
  return BK_OK;
}

bk_status bk_batched_plan_info(const bk_plan* plan, int64_t* total_tiles, int* warps,
                               int* ctas_per_sm, int* chunk, int* tuned) {
  if (plan == nullptr) return set_error(BK_ERR_INVALID_ARG, "plan is NULL");
  if (total_tiles) *total_tiles = plan->total_tiles;
  if (warps) *warps = plan->warps;
  if (ctas_per_sm) *ctas_per_sm = plan->ctas_per_sm;
  if (chunk) *chunk = plan->chunk;
  if (tuned) *tuned = plan->tuned;
  return BK_OK;
}

bk_status bk_matern_batched(const bk_matern_desc* d_descs, int32_t count, bk_dtype dtype,
                            const bk_plan* plan, bk_stream_t stream) {
  if (plan == nullptr) return set_error(BK_ERR_INVALID_ARG, "plan is NULL");
  if (count != plan->count)
    return set_error(BK_ERR_INVALID_ARG, "count %d does not match the plan (%d)", (int)count,
                     (int)plan->count);
  if (dtype != plan->dtype) return set_error(BK_ERR_INVALID_ARG, "dtype does not match the plan");
  if (d_descs == nullptr) return set_error(BK_ERR_INVALID_ARG, "d_descs is NULL");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != plan->device)
    return set_error(BK_ERR_INVALID_ARG, "the plan belongs to device %d", plan->device);
  if (plan->total_tiles == 0) return BK_OK;
  return check_cuda(launch_batched(plan, d_descs, plan->total_tiles, plan->warps,
                                   plan->ctas_per_sm, plan->chunk, (cudaStream_t)stream),
                    "bk_matern_batched launch");
}

bk_status bk_batched_autotune(bk_plan* plan, const bk_matern_desc* d_descs, int64_t sample_tiles,
                              bk_stream_t stream) {
  if (plan == nullptr || d_descs == nullptr)
    return set_error(BK_ERR_INVALID_ARG, "plan and d_descs must be non-NULL");
  if (plan->total_tiles == 0) return BK_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t limit = (sample_tiles > 0) ? std::min(sample_tiles, plan->total_tiles)
                                           : plan->total_tiles;
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess)
    return check_cuda(cudaGetLastError(), "bk_batched_autotune events");
  float best = 1e30f;
  int bw = plan->warps, bc = plan->ctas_per_sm, bch = plan->chunk;
  const int warps_c[2] = {4, 8};
  const int chunk_c[2] = {1, 4};
  bk_status st = BK_OK;
  for (int wi = 0; wi < 2 && st == BK_OK; ++wi) {
    // CTAs per SM: 1, 2, 4, ... below the occupancy limit, and the limit itself
    const int maxc = std::min(max_ctas_per_sm(plan, warps_c[wi]), 8);
    for (int c = 1; c <= maxc && st == BK_OK; c = (c * 2 > maxc && c < maxc) ? maxc : c * 2) {
      for (int ci = 0; ci < 2 && st == BK_OK; ++ci) {
        float ms = 0.0f;
        for (int rep = 0; rep < 2; ++rep) {  // the first run warms the shape up
          cudaEventRecord(a, s);
          cudaError_t e = launch_batched(plan, d_descs, limit, warps_c[wi], c, chunk_c[ci], s);
          cudaEventRecord(b, s);
          if (e == cudaSuccess) e = cudaEventSynchronize(b);
          if (e != cudaSuccess) {
            st = check_cuda(e, "bk_batched_autotune");
            break;
          }
          cudaEventElapsedTime(&ms, a, b);
        }
        if (st == BK_OK && ms < best) {
          best = ms;
          bw = warps_c[wi];
          bc = c;
          bch = chunk_c[ci];
        }
      }
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (st != BK_OK) return st;
  plan->warps = bw;
  plan->ctas_per_sm = bc;
  plan->chunk = bch;
  plan->tuned = 1;
  plan->tuned_ms = best;
  cache_store(plan->key, bw, bc, bch, best);
  return BK_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free batched entry point (bk_matern_batched_static).
//
// bk_batched_plan_create calls cudaMalloc for the work list and the tile
// counter.  Some callers cannot allocate device memory where they build
// their matrices: code running inside a framework that owns all device
// memory through its own pool (a cudaMalloc there can fail, or stall other
// streams while the driver maps memory), and real-time or embedded services
// that forbid allocation after start-up.  For them the same batched work runs
// with its scratch in the fixed array below, which is part of the loaded
// library image: every GPU that loads the library holds it until the process
// exits.  It fits kStaticMaxInstances instances.

namespace bk {
namespace {

constexpr int kStaticMaxInstances = 4096;
// Word layout of the scratch (8-byte words; each part starts on 256 bytes):
// [0] tile counter, [kStaticPrefixOff ...] count + 1 tile offsets,
// [kStaticSizesOff ...] count instance sizes.
constexpr int kStaticPrefixOff = 32;
constexpr int kStaticSizesOff = ((kStaticPrefixOff + kStaticMaxInstances + 1 + 31) / 32) * 32;
constexpr int kStaticWords = kStaticSizesOff + kStaticMaxInstances;

static __device__ __align__(256) unsigned long long g_static_scratch[kStaticWords];

// One block: reads each descriptor's n, writes the sizes and the tile prefix
// sums, and zeroes the tile counter (the scratch keeps the previous call's
// contents, so everything is rewritten here every call).
__global__ void __launch_bounds__(1024) static_batch_prep_kernel(
    const bk_matern_desc* __restrict__ descs, int count, unsigned long long* __restrict__ scratch) {
  int64_t* prefix = (int64_t*)(scratch + kStaticPrefixOff);
  int64_t* sizes = (int64_t*)(scratch + kStaticSizesOff);
  __shared__ int64_t part[1024];
  const int per = (count + (int)blockDim.x - 1) / (int)blockDim.x;
  const int k0 = (int)threadIdx.x * per, k1 = min(count, k0 + per);
  int64_t local = 0;
  for (int k = k0; k < k1; ++k) {
    const int64_t n = descs[k].n;
    sizes[k] = n;
    const int64_t nb = (n > 0) ? (n + kTile - 1) / kTile : 0;
    local += nb * (nb + 1) / 2;
  }
  part[threadIdx.x] = local;
  __syncthreads();
  for (int off = 1; off < (int)blockDim.x; off <<= 1) {  // inclusive scan of the partial sums
    const int64_t v = ((int)threadIdx.x >= off) ? part[threadIdx.x - off] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int64_t run = (threadIdx.x == 0) ? 0 : part[threadIdx.x - 1];
  for (int k = k0; k < k1; ++k) {
    prefix[k] = run;
    const int64_t n = sizes[k];
    const int64_t nb = (n > 0) ? (n + kTile - 1) / kTile : 0;
    run += nb * (nb + 1) / 2;
  }
  if (threadIdx.x == blockDim.x - 1) prefix[count] = part[blockDim.x - 1];
  if (threadIdx.x == 0) scratch[0] = 0ull;
}

// The persistent kernel of bk_matern_batched, with its work list, tile total
// and counter taken from the static scratch (filled by the preparation
// kernel earlier on the same stream).
template <class Form, typename OutT, int WARPS>
__global__ void __launch_bounds__(WARPS * 32, Form::kMinBlocks * 8 / WARPS) matern_batched_static_kernel(
    const bk_matern_desc* __restrict__ descs, int count, unsigned long long* __restrict__ scratch) {
  const int64_t* prefix = (const int64_t*)(scratch + kStaticPrefixOff);
  const int64_t limit = prefix[count];
  __shared__ BatchSmem<OutT> sm;
  __shared__ double s_tab[Form::kStageTable ? kExpTabSize : 1];
  const Form f = bind_table(Form{}, s_tab);
  Tally tl{0u, 0u, 0u, 0u, 0u, 0u, 0u};
  unsigned evals = 0;
  int cur = -1;
  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) sm.item = (int64_t)atomicAdd(scratch, 1ull);
    __syncthreads();
    const int64_t w = sm.item;
    if (w >= limit) break;
    const int k = find_instance(prefix, count, w);
    if (k != cur) {
      __syncthreads();
      if (threadIdx.x == 0) {
        bk_matern_desc d = descs[k];
        // sizes[k] was copied from this descriptor by the preparation kernel,
        // so only the descriptor's own fields need checking here.  There are
        // no counters on this path: a skipped descriptor leaves its output
        // untouched and is not reported.
        const bool ok = d.n >= 0 && d.ld >= d.n && d.locs != nullptr && d.out != nullptr &&
                        d.beta > 0.0 && d.nu > 0.0 && d.sigma2 >= 0.0;
        if (!ok) d.n = 0;  // an invalid descriptor is skipped
        sm.locs = d.locs;
        sm.out = (OutT*)d.out;
        sm.n = d.n;
        sm.ld = d.ld;
        sm.mp = matern_params(d.sigma2, d.beta, d.nu);
      }
      __syncthreads();
      cur = k;
    }
    int64_t I, J;
    tri_tile(w - prefix[k], I, J);
    __syncthreads();
    sym_tile<Form, OutT, WARPS>(f, sm.tile, sm.locs, sm.n, I, J, sm.mp, sm.out, sm.ld, tl,
                                evals);
  }
}

// Device address of the scratch on the current device.  The array's name in
// host code is only a host-side handle, so the address is looked up with
// cudaGetSymbolAddress on every call (a host-side lookup once the library's
// device code is loaded on the device; the first call on a device also loads
// it there).  Not caching it keeps the address right after the context is
// torn down and created again (cudaDeviceReset), when the array may move.
bk_status static_scratch_address(unsigned long long** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
  if (e != cudaSuccess) return check_cuda(e, "bk_matern_batched_static: cudaGetSymbolAddress");
  *out = (unsigned long long*)p;
  return BK_OK;
}

}  // namespace
}  // namespace bk

extern "C" bk_status bk_matern_batched_static(const bk_matern_desc* d_descs, int32_t count,
                                              bk_dtype dtype, bk_stream_t stream) {
  using namespace bk;
  if (count < 1 || count > kStaticMaxInstances)
    return set_error(BK_ERR_INVALID_ARG,
                     "bk_matern_batched_static: count must be in [1, %d] (got %d); use a plan "
                     "(bk_batched_plan_create) for larger batches",
                     kStaticMaxInstances, (int)count);
  if (d_descs == nullptr) return set_error(BK_ERR_INVALID_ARG, "d_descs is NULL");
  if (dtype != BK_F64 && dtype != BK_F32)
    return set_error(BK_ERR_INVALID_ARG, "dtype: unknown value %d", (int)dtype);
  unsigned long long* scratch = nullptr;
  bk_status st = static_scratch_address(&scratch);
  if (st != BK_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  static_batch_prep_kernel<<<1, 1024, 0, s>>>(d_descs, count, scratch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return check_cuda(e, "bk_matern_batched_static: preparation launch");
  const int grid = current_sm_count() * 2;
  if (dtype == BK_F64)
    matern_batched_static_kernel<FormF64, double, 8><<<grid, 256, 0, s>>>(d_descs, count, scratch);
  else
    matern_batched_static_kernel<FormF32, float, 8><<<grid, 256, 0, s>>>(d_descs, count, scratch);
  return check_cuda(cudaGetLastError(), "bk_matern_batched_static launch");
}
