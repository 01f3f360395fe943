// Matern matrices delivered to host memory (bk_matern_tile_host).
//
// Two ways:
//  * Host memory that the device can address (cudaHostGetDevicePointer gives
//    its device address: page-locked memory from cudaHostAlloc, cudaMallocHost
//    or cudaHostRegister, and on GB300, whose GPU reaches the CPU's page tables
//    through ATS, ordinary pageable memory too): the tile writer stores the
//    matrix straight into it over the GPU-CPU link (NVLink-C2C), as it would
//    into device memory.  No staging copy and no second pass over the data;
//    only the locations are copied in.
//  * Otherwise, or when the caller asks for it (BK_HOST_STAGED): the matrix is generated in a device workspace in
//    panels of block-columns (block-column order), and each finished panel's
//    columns are copied out while later panels are generated.  After the
//    tiles of block-columns 0 .. J - 1 every entry of columns below 32 J is
//    final (tile (I, J) writes block (I, J) and, transposed, block (J, I)), so
//    panel p's columns can leave as soon as its tiles are done.  All panel
//    kernels are enqueued first: copies into pageable memory block the calling
//    thread, and the kernels keep the GPU busy meanwhile.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "bk_internal.h"

namespace bk {
namespace {

constexpr int kMaxPanels = 16;
constexpr int kBlock = 32;
constexpr size_t kAlign = 256;

size_t round_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// Workspace layout: locations (16 n bytes), the e^{-2 nu h} table of the
// plain form, then the n x n matrix with leading dimension n.
struct Layout {
  size_t locs, table, matrix, total;
};
Layout layout(int64_t n, bk_dtype dtype) {
  Layout L;
  L.locs = 0;
  L.table = round_up((size_t)n * 2 * sizeof(double));
  L.matrix = L.table + round_up((size_t)BK_COSH_TABLE_LEN * sizeof(double));
  const size_t elem = dtype == BK_F64 ? sizeof(double) : sizeof(float);
  L.total = L.matrix + (size_t)n * (size_t)n * elem;
  return L;
}

// The copy stream and events of one device (created on first use, kept until
// the process exits; no device memory).
struct DeviceCopier {
  cudaStream_t stream = nullptr;
  cudaEvent_t ev[kMaxPanels + 1] = {};
};
std::mutex g_copier_mutex;
DeviceCopier g_copiers[64];

bk_status copier_for_current_device(DeviceCopier** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return check_cuda(e, "bk_matern_tile_host: cudaGetDevice");
  if (dev < 0 || dev >= 64)
    return set_error(BK_ERR_UNSUPPORTED, "bk_matern_tile_host: device %d out of range", dev);
  DeviceCopier& c = g_copiers[dev];
  if (c.stream == nullptr) {
    e = cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return check_cuda(e, "bk_matern_tile_host: cudaStreamCreate");
    for (int k = 0; k <= kMaxPanels; ++k) {
      e = cudaEventCreateWithFlags(&c.ev[k], cudaEventDisableTiming);
      if (e != cudaSuccess) return check_cuda(e, "bk_matern_tile_host: cudaEventCreate");
    }
  }
  *out = &c;
  return BK_OK;
}

// Block-column boundaries of `panels` panels with about equal tile counts:
// the first block-column whose block-column-order offset reaches p/panels of
// the triangle.
std::vector<int64_t> panel_bounds(int64_t nb, int panels) {
  std::vector<int64_t> b(panels + 1, nb);
  b[0] = 0;
  const double total = (double)nb * (double)(nb + 1) / 2.0;
  int64_t J = 0;
  for (int p = 1; p < panels; ++p) {
    const double want = total * p / panels;
    while (J < nb && (double)(J * nb - J * (J - 1) / 2) < want) ++J;
    b[p] = std::max(J, b[p - 1]);
  }
  return b;
}

}  // namespace
}  // namespace bk

using namespace bk;

extern "C" {

size_t bk_matern_tile_host_workspace(int64_t n, bk_dtype dtype, int staged) {
  if (n < 0 || (dtype != BK_F64 && dtype != BK_F32)) return 0;
  const Layout L = layout(n, dtype);
  return staged ? L.total : L.matrix;
}

bk_status bk_matern_tile_host(const double* h_locs, int64_t n, double sigma2, double beta,
                              double nu, void* h_out, int64_t ld, bk_dtype dtype,
                              const bk_opts* opts, int mode, void* d_work, size_t work_bytes,
                              bk_stream_t stream) {
  if (mode != BK_HOST_AUTO && mode != BK_HOST_STAGED)
    return set_error(BK_ERR_INVALID_ARG, "mode: unknown value %d", mode);
  if (dtype != BK_F64 && dtype != BK_F32)
    return set_error(BK_ERR_INVALID_ARG, "dtype: unknown value %d", (int)dtype);
  if (n < 0) return set_error(BK_ERR_INVALID_ARG, "n must be >= 0 (got %lld)", (long long)n);
  if (!(sigma2 >= 0.0) || !(sigma2 <= 1.7e308) || !(beta > 0.0) || !(beta <= 1.7e308) ||
      !(nu > 0.0) || !(nu <= 1.7e308))
    return set_error(BK_ERR_INVALID_ARG,
                     "sigma2 must be finite and >= 0, beta and nu finite and > 0");
  if (n == 0) return BK_OK;
  if (h_locs == nullptr || h_out == nullptr || d_work == nullptr)
    return set_error(BK_ERR_INVALID_ARG, "h_locs, h_out and d_work must be non-NULL");
  if (ld < n)
    return set_error(BK_ERR_INVALID_ARG, "ld (%lld) < n (%lld)", (long long)ld, (long long)n);
  if (n > INT64_MAX / ld) return set_error(BK_ERR_INVALID_ARG, "ld * n overflows int64");
  if (((uintptr_t)d_work % kAlign) != 0)
    return set_error(BK_ERR_INVALID_ARG, "d_work must be 256-byte aligned");
  const Layout L = layout(n, dtype);
  if (work_bytes < L.matrix)
    return set_error(BK_ERR_NOMEM, "bk_matern_tile_host: workspace of %zu bytes, %zu needed",
                     work_bytes, L.matrix);
  bk_opts o;
  bk_opts_default(&o);
  if (opts != nullptr) o = *opts; else o.compute = dtype;
  bk_status st = check_opts(&o);
  if (st != BK_OK) return st;

  // The device address of h_out, when the device can write it directly
  // (BK_HOST_AUTO).
  void* d_out = nullptr;
  if (mode == BK_HOST_AUTO && cudaHostGetDevicePointer(&d_out, h_out, 0) != cudaSuccess) {
    (void)cudaGetLastError();  // not addressable from the device: the staged way
    d_out = nullptr;
  }
  if (d_out == nullptr && work_bytes < L.total)
    return set_error(BK_ERR_NOMEM,
                     "bk_matern_tile_host: h_out is not device-mapped, so the matrix is staged "
                     "in the workspace: %zu bytes, %zu needed", work_bytes, L.total);

  char* ws = (char*)d_work;
  double* d_locs = (double*)(ws + L.locs);
  if (o.compute == BK_F64 && o.d_cosh_table == nullptr) o.d_cosh_table = (double*)(ws + L.table);
  const size_t elem = dtype == BK_F64 ? sizeof(double) : sizeof(float);
  cudaStream_t s = (cudaStream_t)stream;

  auto launch = [&](void* out, int64_t ldo, const SymRange& r) {
    return (o.window == BK_WIN_LEARNED)
               ? launch_matern_sym_learned(o.learned, d_locs, n, sigma2, beta, nu, out, ldo, dtype,
                                           o.d_counters, s, r)
           : (o.compute == BK_F64)
               ? launch_matern_sym_f64(d_locs, n, sigma2, beta, nu, out, ldo, dtype, o, s, r)
               : launch_matern_sym_f32(d_locs, n, sigma2, beta, nu, out, ldo, dtype,
                                       o.d_counters, s, r);
  };

  cudaError_t e = cudaMemcpyAsync(d_locs, h_locs, (size_t)n * 2 * sizeof(double),
                                  cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return check_cuda(e, "bk_matern_tile_host: locations to the device");
  if (d_out != nullptr) return check_cuda(launch(d_out, ld, SymRange{}), "bk_matern_tile_host launch");

  // Staged: all panel kernels first (each followed by its event), then the
  // copies of each panel's columns on the copy stream.
  std::lock_guard<std::mutex> lk(g_copier_mutex);
  DeviceCopier* cp = nullptr;
  if ((st = copier_for_current_device(&cp)) != BK_OK) return st;
  void* d_mat = ws + L.matrix;
  const int64_t nb = (n + kBlock - 1) / kBlock;
  const int panels = (int)std::min<int64_t>(kMaxPanels, nb);
  const std::vector<int64_t> bounds = panel_bounds(nb, panels);
  for (int p = 0; p < panels; ++p) {
    SymRange r;
    r.j0 = bounds[p];
    r.j1 = bounds[p + 1];
    r.fill_table = (p == 0);
    if (r.j1 > r.j0 && (e = launch(d_mat, n, r)) != cudaSuccess)
      return check_cuda(e, "bk_matern_tile_host: panel launch");
    if ((e = cudaEventRecord(cp->ev[p], s)) != cudaSuccess)
      return check_cuda(e, "bk_matern_tile_host: panel event");
  }
  for (int p = 0; p < panels; ++p) {
    const int64_t c0 = bounds[p] * kBlock, c1 = std::min<int64_t>(bounds[p + 1] * kBlock, n);
    if (c1 <= c0) continue;
    if ((e = cudaStreamWaitEvent(cp->stream, cp->ev[p], 0)) != cudaSuccess)
      return check_cuda(e, "bk_matern_tile_host: panel wait");
    e = cudaMemcpy2DAsync((char*)h_out + (size_t)(c0 * ld) * elem, (size_t)ld * elem,
                          (const char*)d_mat + (size_t)(c0 * n) * elem, (size_t)n * elem,
                          (size_t)n * elem, (size_t)(c1 - c0), cudaMemcpyDeviceToHost,
                          cp->stream);
    if (e != cudaSuccess) return check_cuda(e, "bk_matern_tile_host: panel copy");
  }
  // `stream` continues once every copy has landed in h_out.
  if ((e = cudaEventRecord(cp->ev[kMaxPanels], cp->stream)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(s, cp->ev[kMaxPanels], 0)) != cudaSuccess)
    return check_cuda(e, "bk_matern_tile_host: completion event");
  return BK_OK;
}

}  // extern "C"
