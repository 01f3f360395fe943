// The Gaussian log-likelihood that consumes the generated covariance matrix
// (the step after matrix generation in the maximum-likelihood loop the paper
// accelerates, Sec. II):
//   l = -1/2 (z^T Sigma^{-1} z + log det Sigma + n log 2 pi),
// by an in-place blocked Cholesky Sigma = L L^T in FP64 (right-looking,
// 64 x 64 tiles: factor the diagonal tile, solve the tiles below it,
// update the trailing lower triangle), log det Sigma = 2 sum log L_ii, and
// the forward substitution L y = z interleaved with the factorisation
// (z^T Sigma^{-1} z = y^T y).  Every step is one of the kernels below; the
// host only sequences the launches on the caller's stream.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "bk_internal.h"
#include "bk_tiles.cuh"

namespace bk {
namespace {

constexpr int kNB = 64;  // tile edge

// Rows (or columns) of the tile that starts at o.
__device__ __forceinline__ int tile_len(int64_t n, int64_t o) {
  return (int)(n - o < kNB ? n - o : kNB);
}

// The diagonal tile (k, k): unblocked right-looking Cholesky in shared
// memory.  A non-positive pivot becomes NaN, which propagates to every later
// result (the log-likelihood then reads NaN), and is counted.
__global__ void __launch_bounds__(256) chol_diag_kernel(double* __restrict__ a, int64_t ld,
                                                        int64_t n, int64_t k,
                                                        unsigned long long* __restrict__ ctr) {
  __shared__ double S[kNB][kNB + 1];
  __shared__ double s_inv;
  const int64_t o = k * kNB;
  const int b = tile_len(n, o);
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int r = e % b, c = e / b;
    if (r >= c) S[r][c] = a[(o + r) + (o + c) * ld];
  }
  for (int j = 0; j < b; ++j) {
    __syncthreads();
    if (threadIdx.x == 0) {
      const double d = S[j][j];
      double p = sqrt(d);
      if (!(d > 0.0)) {
        p = __longlong_as_double(0x7ff8000000000000LL);
        if (ctr != nullptr) atomicAdd(ctr + BK_CTR_FAIL, 1ull);
      }
      S[j][j] = p;
      s_inv = 1.0 / p;
    }
    __syncthreads();
    const double inv = s_inv;
    for (int i = j + 1 + threadIdx.x; i < b; i += blockDim.x) S[i][j] *= inv;
    __syncthreads();
    // trailing update of the tile: S[i][c] -= S[i][j] S[c][j], j < c <= i
    const int m = b - j - 1;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int r = j + 1 + e % m, c = j + 1 + e / m;
      if (r >= c) S[r][c] = fma(-S[r][j], S[c][j], S[r][c]);
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int r = e % b, c = e / b;
    if (r >= c) a[(o + r) + (o + c) * ld] = S[r][c];
  }
}

// The tiles (i, k), i > k: L_ik = A_ik L_kk^{-T}, one tile per block, one
// row of the tile per thread (forward substitution along the row).
__global__ void __launch_bounds__(kNB) chol_trsm_kernel(double* __restrict__ a, int64_t ld,
                                                        int64_t n, int64_t k) {
  __shared__ double Lk[kNB][kNB + 1];
  __shared__ double X[kNB][kNB + 1];
  const int64_t o = k * kNB;
  const int64_t ro = o + (int64_t)(blockIdx.x + 1) * kNB;  // first row of the tile
  const int b = tile_len(n, o);             // == kNB for all but the last step
  const int rows = tile_len(n, ro);
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int r = e % b, c = e / b;
    Lk[r][c] = (r >= c) ? a[(o + r) + (o + c) * ld] : 0.0;
  }
  for (int e = threadIdx.x; e < rows * b; e += blockDim.x) {
    const int r = e % rows, c = e / rows;
    X[r][c] = a[(ro + r) + (o + c) * ld];
  }
  __syncthreads();
  const int r = threadIdx.x;
  if (r < rows) {
    for (int c = 0; c < b; ++c) {
      double s = X[r][c];
      for (int l = 0; l < c; ++l) s = fma(-X[r][l], Lk[c][l], s);
      X[r][c] = s / Lk[c][c];
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < rows * b; e += blockDim.x) {
    const int rr = e % rows, c = e / rows;
    a[(ro + rr) + (o + c) * ld] = X[rr][c];
  }
}

// The trailing update A_ij -= L_ik L_jk^T for k < j <= i (lower-triangle
// tiles of the remaining matrix, one per block): a 64 x 64 x 64 FP64
// product, 256 threads with a 4 x 4 register tile each, the two panels
// staged through shared memory in halves of 32 columns.  Diagonal tiles
// write only their lower triangle.
__global__ void __launch_bounds__(256) chol_update_kernel(double* __restrict__ a, int64_t ld,
                                                          int64_t n, int64_t k) {
  __shared__ double Pi[kNB][33];
  __shared__ double Pj[kNB][33];
  int64_t ti, tj;
  tri_tile((int64_t)blockIdx.x, ti, tj);  // (ti, tj) with ti >= tj, relative to k + 1
  const int64_t o = k * kNB;
  const int64_t io = (k + 1 + ti) * kNB, jo = (k + 1 + tj) * kNB;
  const int ri = tile_len(n, io), rj = tile_len(n, jo);
  const int tr = threadIdx.x % 16, tc = threadIdx.x / 16;  // 16 x 16 threads, 4 x 4 each
  double acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = 0.0;
  for (int half = 0; half < 2; ++half) {
    const int64_t co = o + half * 32;
    __syncthreads();
    for (int e = threadIdx.x; e < kNB * 32; e += blockDim.x) {
      const int r = e % kNB, c = e / kNB;
      Pi[r][c] = (r < ri) ? a[(io + r) + (co + c) * ld] : 0.0;
      Pj[r][c] = (r < rj) ? a[(jo + r) + (co + c) * ld] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int c = 0; c < 32; ++c) {
      double x[4], y[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) x[u] = Pi[tr + 16 * u][c];
#pragma unroll
      for (int v = 0; v < 4; ++v) y[v] = Pj[tc + 16 * v][c];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(x[u], y[v], acc[u][v]);
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int r = tr + 16 * u, c = tc + 16 * v;
      if (r < ri && c < rj && (ti != tj || r >= c)) {
        double* p = a + (io + r) + (jo + c) * ld;
        *p -= acc[u][v];
      }
    }
  }
}

// Forward substitution of the diagonal tile: y_k <- L_kk^{-1} y_k (y holds
// z minus the contributions of the earlier tiles); one block, sequential in
// the tile's columns with the column's updates spread over the threads.
__global__ void __launch_bounds__(kNB) trsv_diag_kernel(const double* __restrict__ a, int64_t ld,
                                                        int64_t n, int64_t k,
                                                        double* __restrict__ y) {
  __shared__ double v[kNB];
  const int64_t o = k * kNB;
  const int b = tile_len(n, o);
  if ((int)threadIdx.x < b) v[threadIdx.x] = y[o + threadIdx.x];
  __syncthreads();
  for (int c = 0; c < b; ++c) {
    if (threadIdx.x == 0) v[c] /= a[(o + c) + (o + c) * ld];
    __syncthreads();
    const int r = threadIdx.x;
    if (r > c && r < b) v[r] = fma(-a[(o + r) + (o + c) * ld], v[c], v[r]);
    __syncthreads();
  }
  if ((int)threadIdx.x < b) y[o + threadIdx.x] = v[threadIdx.x];
}

// y_r -= sum_c L_rc y_c over the tile's columns, for every row below it.
__global__ void __launch_bounds__(256) gemv_update_kernel(const double* __restrict__ a,
                                                          int64_t ld, int64_t n, int64_t k,
                                                          double* __restrict__ y) {
  const int64_t o = k * kNB;
  const int b = tile_len(n, o);
  const int64_t r = o + b + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  double s = 0.0;
  for (int c = 0; c < b; ++c) s = fma(a[r + (o + c) * ld], y[o + c], s);
  y[r] -= s;
}

// out = [l, log det Sigma, y^T y]: one block reduces sum log L_ii and y^T y.
__global__ void __launch_bounds__(256) loglik_finish_kernel(const double* __restrict__ a,
                                                            int64_t ld, int64_t n,
                                                            const double* __restrict__ y,
                                                            double* __restrict__ out) {
  __shared__ double s_ld[256], s_q[256];
  double ldet = 0.0, q = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    ldet += log(a[i + i * ld]);
    q = fma(y[i], y[i], q);
  }
  s_ld[threadIdx.x] = ldet;
  s_q[threadIdx.x] = q;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      s_ld[threadIdx.x] += s_ld[threadIdx.x + w];
      s_q[threadIdx.x] += s_q[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double logdet = 2.0 * s_ld[0];
    out[1] = logdet;
    out[2] = s_q[0];
    out[0] = -0.5 * (s_q[0] + logdet + (double)n * 1.8378770664093454836);  // log 2 pi
  }
}

}  // namespace

cudaError_t launch_loglik(double* a, int64_t n, int64_t ld, const double* z, double* y,
                          double* out, unsigned long long* ctr, cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(y, z, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return e;
  const int64_t nt = (n + kNB - 1) / kNB;
  for (int64_t k = 0; k < nt; ++k) {
    chol_diag_kernel<<<1, 256, 0, s>>>(a, ld, n, k, ctr);
    const int64_t below = nt - k - 1;
    if (below > 0) {
      chol_trsm_kernel<<<(unsigned)below, kNB, 0, s>>>(a, ld, n, k);
      chol_update_kernel<<<(unsigned)(below * (below + 1) / 2), 256, 0, s>>>(a, ld, n, k);
    }
    trsv_diag_kernel<<<1, kNB, 0, s>>>(a, ld, n, k, y);
    const int64_t rest = n - std::min<int64_t>(n, (k + 1) * kNB);
    if (rest > 0) gemv_update_kernel<<<(unsigned)((rest + 255) / 256), 256, 0, s>>>(a, ld, n, k, y);
  }
  loglik_finish_kernel<<<1, 256, 0, s>>>(a, ld, n, y, out);
  return cudaGetLastError();
}

}  // namespace bk
