// Pipe-rate probes for the roofline denominators of this ALU-bound library:
// FP64 FMA, FP32 FMA and the MUFU ex2 unit.  Each thread runs `iters` trips
// of 8 independent dependency chains (enough instruction-level parallelism
// to keep a pipe busy) and writes one value to `sink` so nothing is removed.
#include <cuda_runtime.h>

#include <cstdint>

#include "bk_internal.h"
#include "bk_math64.cuh"

namespace bk {
namespace {

__global__ void probe_dfma(int64_t iters, double* sink) {
  double a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = 1.0 + 1e-3 * (threadIdx.x + k);
  const double m = 0.9999999, c = 1e-7;
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fma(a[k], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  sink[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void probe_ffma(int64_t iters, double* sink) {
  float a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = 1.0f + 1e-3f * (threadIdx.x + k);
  const float m = 0.9999f, c = 1e-4f;
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fmaf(a[k], m, c);
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  sink[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__device__ __forceinline__ float ex2_neg(float v) {  // 2^-v on the MUFU unit
  float r;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(-v));
  return r;
}

__global__ void probe_ex2(int64_t iters, double* sink) {
  float a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = 0.5f + 1e-3f * (threadIdx.x + k);
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = ex2_neg(a[k]);  // stays in [0.5, 1)
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  sink[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// FP64 -> FP32 conversions: per trip one conversion of a double in [1, 2),
// whose float result is turned back into a double in [1, 2) by integer
// operations only (so the compiler cannot fold a round trip).
__global__ void probe_cvt64(int64_t iters, double* sink) {
  double a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = 1.0 + 1e-3 * (threadIdx.x + k);
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int b = __float_as_int((float)a[k]);
      a[k] = __hiloint2double(0x3ff00000 | ((b + 1) & 0x000fffff), b);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  sink[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// FP32 -> FP64 conversions: per trip one conversion of a float in [1, 2),
// whose double result is turned back into a float in [1, 2) by integer
// operations only.
__global__ void probe_cvt32(int64_t iters, double* sink) {
  float a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = 1.0f + 1e-3f * (threadIdx.x + k);
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int h = __double2hiint((double)a[k]);
      a[k] = __int_as_float(0x3f800000 | ((h + 1) & 0x007fffff));
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  sink[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// The plain form's math helpers on an array of inputs (bk_math_probe), with
// the exponential table read from global memory.
__global__ void math_probe_kernel(int fn, const double* __restrict__ in, double* __restrict__ out,
                                  int64_t n) {
  const double* tab = kExp2Tab;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double v = in[i];
    switch (fn) {
      case 0: out[i] = exp_tab_full(v, tab); break;
      case 1: out[i] = log_tab(v, tab); break;
      case 2: out[i] = exp2s_int<false>(v, tab); break;
      case 3: out[i] = exp2s_fix(fix40_node(v), tab); break;
      case 4: {
        int M;
        double r;
        round_rem(v, M, r);
        out[2 * i] = (double)M;
        out[2 * i + 1] = r;
        break;
      }
      case 5: out[i] = two_cosh_warp(v, tab); break;
      case 6: out[i] = sqrt_pos(v); break;
      case 7: out[i] = exp_acc(v, tab); break;
      case 8: out[i] = exp_units_full(v * kExpScale, tab); break;
      case 10: out[i] = sqrt_int(v); break;
      case 11: out[i] = exp2s_fix(__double2ll_rn(v * 0x1p40), tab); break;
      case 12: out[i] = one_plus_w(fix63_unit(v)); break;
      case 13: out[i] = (double)fix64_unit(v) * 0x1p-64; break;
      default: {
        double nd;
        const double l1p = log_tab_parts(v, tab, nd);
        out[i] = fma(nd, kExpC1, l1p);
        break;
      }
    }
  }
}

}  // namespace
}  // namespace bk

extern "C" bk_status bk_probe_pipe(int kind, int64_t iters, int grid, int block, double* sink,
                                   bk_stream_t stream) {
  using namespace bk;
  if (iters < 0 || grid < 1 || block < 1 || block > 1024 || sink == nullptr)
    return set_error(BK_ERR_INVALID_ARG, "bk_probe_pipe: bad launch arguments");
  cudaStream_t s = (cudaStream_t)stream;
  switch (kind) {
    case 0: probe_dfma<<<grid, block, 0, s>>>(iters, sink); break;
    case 1: probe_ffma<<<grid, block, 0, s>>>(iters, sink); break;
    case 2: probe_ex2<<<grid, block, 0, s>>>(iters, sink); break;
    case 3: probe_cvt64<<<grid, block, 0, s>>>(iters, sink); break;
    case 4: probe_cvt32<<<grid, block, 0, s>>>(iters, sink); break;
    default: return set_error(BK_ERR_INVALID_ARG, "bk_probe_pipe: unknown kind %d", kind);
  }
  return check_cuda(cudaGetLastError(), "bk_probe_pipe launch");
}

extern "C" bk_status bk_math_probe(int fn, const double* in, double* out, int64_t n,
                                   bk_stream_t stream) {
  using namespace bk;
  if (fn < 0 || fn > 13) return set_error(BK_ERR_INVALID_ARG, "bk_math_probe: unknown fn %d", fn);
  if (n < 0 || (n > 0 && (in == nullptr || out == nullptr)))
    return set_error(BK_ERR_INVALID_ARG, "bk_math_probe: bad arguments");
  if (n == 0) return BK_OK;
  const int64_t blocks = (n + 255) / 256;
  const int grid = (int)(blocks < 152 * 8 ? blocks : 152 * 8);
  math_probe_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(fn, in, out, n);
  return check_cuda(cudaGetLastError(), "bk_math_probe launch");
}
