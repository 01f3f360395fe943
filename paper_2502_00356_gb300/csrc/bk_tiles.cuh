// Kernels shared by the arithmetic forms: the bk_eval kernel, the fused
// symmetric Matern tile writer and the m x n block writer, templated on a
// Form passed by value that supplies one K_nu evaluation and one Matern entry:
//   double eval(double x, double nu, Tally&, unsigned& evals, double& log_k) const;
//   double matern(const Loc& a, const Loc& b, const MaternParams&, Tally&, unsigned& evals) const;
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "bk.h"
#include "bk_internal.h"
#include "bk_math64.cuh"
#include "bk_forms.cuh"
#include "bk_matern_common.cuh"

namespace bk {


// Adds this warp's tallies to the caller's counters (one atomic per warp and
// counter).  Every lane of the warp must call it.
__device__ __forceinline__ void flush_tally(unsigned long long* ctr, const Tally& tl,
                                            unsigned evals) {
  if (ctr == nullptr) return;
  unsigned long long v[8] = {tl.fail,       tl.nodes,    tl.iters,   evals,
                             tl.peak_iters, tl.fallback, tl.repairs, tl.series};
  const int idx[8] = {BK_CTR_FAIL,       BK_CTR_NODES,    BK_CTR_ITERS,  BK_CTR_EVALS,
                      BK_CTR_PEAK_ITERS, BK_CTR_FALLBACK, BK_CTR_REPAIR, BK_CTR_SERIES};
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    unsigned long long a = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if ((threadIdx.x & 31) == 0 && a) atomicAdd(ctr + idx[k], a);
  }
}


// Adds the block's tallies to the caller's counters: warp sums, then one
// shared-memory total and one global atomic per counter and block.  Every
// thread of the block must call it.
__device__ __forceinline__ void flush_tally_block(unsigned long long* ctr, const Tally& tl,
                                                  unsigned evals) {
  if (ctr == nullptr) return;
  __shared__ unsigned long long s_acc[8];
  if (threadIdx.x < 8) s_acc[threadIdx.x] = 0ull;
  __syncthreads();
  unsigned long long v[8] = {tl.fail,       tl.nodes,    tl.iters,   evals,
                             tl.peak_iters, tl.fallback, tl.repairs, tl.series};
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    unsigned long long a = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if ((threadIdx.x & 31) == 0 && a) atomicAdd(&s_acc[k], a);
  }
  __syncthreads();
  const int idx[8] = {BK_CTR_FAIL,       BK_CTR_NODES,    BK_CTR_ITERS,  BK_CTR_EVALS,
                      BK_CTR_PEAK_ITERS, BK_CTR_FALLBACK, BK_CTR_REPAIR, BK_CTR_SERIES};
  if (threadIdx.x < 8 && s_acc[threadIdx.x]) atomicAdd(ctr + idx[threadIdx.x], s_acc[threadIdx.x]);
}

// Binds a form to its exponential table: the block's shared copy (filled
// here, block-wide) or the global one.
template <class Form>
__device__ __forceinline__ Form bind_table(const Form& form, double* s_tab) {
  Form f = form;
  if constexpr (Form::kStageTable) {
    exp_table_init(s_tab);
    f.tab = s_tab;
  } else {
    f.tab = kExp2Tab;
  }
  return f;
}

constexpr int kSortChunk = 1024;  // pairs per counting sort (8 rounds of 128)

// Orders the pairs [lo, lo + cnt), cnt <= kSortChunk, by bucket_of(x, nu) in
// 0 .. 63 (the form's cost bucket) with a counting sort in shared memory:
// s_perm receives their local indices in ascending bucket order (in any
// order inside a bucket).  Warps that then take consecutive runs of 32 see
// similar node counts and search paths, where random pairs leave most lanes
// idle while the slowest finishes.  Each pair's arithmetic is unchanged and
// results go back to their own positions.  Every thread of the 128-thread
// block calls it; x and nu are read again from L1 in the rounds that follow.
template <class BucketOf>
__device__ __forceinline__ void sort_chunk(const double* __restrict__ x,
                                           const double* __restrict__ nu, int64_t lo, int cnt,
                                           unsigned short* s_perm, unsigned* s_cnt,
                                           BucketOf bucket_of) {
  constexpr int kR = kSortChunk / 128;
  const int t = threadIdx.x;
  __syncthreads();  // the previous chunk's order is no longer read
  if (t < 64) s_cnt[t] = 0u;
  __syncthreads();
  unsigned short rank[kR];
  unsigned char bk[kR];
#pragma unroll
  for (int r = 0; r < kR; ++r) {
    const int k = r * 128 + t;
    bk[r] = 0;
    rank[r] = 0;
    if (k < cnt) {
      bk[r] = (unsigned char)bucket_of(x[lo + k], nu[lo + k]);
      rank[r] = (unsigned short)atomicAdd(&s_cnt[bk[r]], 1u);
    }
  }
  __syncthreads();
  if (t < 32) {  // exclusive prefix sum of the 64 counts, two per lane
    const unsigned c0 = s_cnt[2 * t], c1 = s_cnt[2 * t + 1];
    unsigned v = c0 + c1;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned u = __shfl_up_sync(0xffffffffu, v, d);
      if (t >= d) v += u;
    }
    const unsigned ex = v - (c0 + c1);
    s_cnt[2 * t] = ex;
    s_cnt[2 * t + 1] = ex + c0;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kR; ++r) {
    const int k = r * 128 + t;
    if (k < cnt) s_perm[s_cnt[bk[r]] + rank[r]] = (unsigned short)k;
  }
  __syncthreads();
}

// The sorted position thread t takes in round r of a sorted chunk: warp w
// takes run 4r + w in even rounds and run 4r + 3 - w in odd ones, so that
// the four warps get equal shares of cheap and costly runs.
__device__ __forceinline__ int sorted_slot(int r) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  return (4 * r + ((r & 1) ? 3 - w : w)) * 32 + l;
}

// Block b's pairs [lo, hi) when the grid (one wave of resident blocks) takes
// the n pairs in equal contiguous chunks of whole 128-pair rounds (+9 % on
// 10^7 FP64 evaluations over a grid-stride loop).
__device__ __forceinline__ void block_range(int64_t n, int64_t& lo, int64_t& hi) {
  const int64_t chunk = ((n + gridDim.x - 1) / gridDim.x + 127) / 128 * 128;
  lo = (int64_t)blockIdx.x * chunk;
  hi = lo + chunk < n ? lo + chunk : n;
}

// Bare evaluations of the FP64 forms, 128 per block and round, in chunks
// sorted by the form's cost bucket (sort_chunk).
template <class Form, typename OutT>
__global__ void __launch_bounds__(128, 6) eval_kernel(const Form form, const double* __restrict__ x,
                                                   const double* __restrict__ nu,
                                                   OutT* __restrict__ out,
                                                   OutT* __restrict__ log_out, int64_t n,
                                                   unsigned long long* __restrict__ ctr) {
  constexpr int kB = 128;
  __shared__ double s_tab[Form::kStageTable ? kExpTabSize : 1];
  __shared__ unsigned short s_perm[kSortChunk];
  __shared__ unsigned s_cnt[64];
  const Form f = bind_table(form, s_tab);
  Tally tl{0u, 0u, 0u, 0u, 0u, 0u, 0u};
  unsigned evals = 0;
  const bool want_log = (log_out != nullptr);
  int64_t lo, hi;
  block_range(n, lo, hi);
  for (int64_t base = lo; base < hi; base += kSortChunk) {
    const int cnt = (int)(hi - base < kSortChunk ? hi - base : kSortChunk);
    sort_chunk(x, nu, base, cnt, s_perm, s_cnt,
               [&](double xi, double vi) { return f.sort_bucket(xi, vi); });
    const int rounds = (cnt + kB - 1) / kB;
    for (int r = 0; r < rounds; ++r) {
      const int p = sorted_slot(r);
      if (p < cnt) {
        const int64_t i = base + s_perm[p];
        OutT k, lk;
        f.template eval_out<OutT>(x[i], nu[i], tl, evals, k, lk, want_log);
        out[i] = k;
        if (log_out != nullptr) log_out[i] = lk;
      }
    }
  }
  flush_tally(ctr, tl, evals);
}

// Bare evaluations of the FP32 forms with the quadrature split over L lanes
// (eval_out_f32_coop), 128 pairs per block and round in input order, eight
// blocks per SM.  Sorting chunks of 1,024 pairs by eval_cost_bucket first
// (as eval_kernel does) raised the learned form's active lanes from 23.2 to
// 28.2 of 32 and cut its warp instructions by 6 %, but the warps of a sorted
// chunk run the same phases together and issued 77 % of cycles instead of
// 83 %: 2.55e10 against 2.59e10 evaluations/s on 10^8 pairs (measured), so
// the pairs stay in input order here.
template <class Form, typename OutT, int L>
__global__ void __launch_bounds__(128, 8) eval_coop_kernel(const Form form,
                                                        const double* __restrict__ x,
                                                        const double* __restrict__ nu,
                                                        OutT* __restrict__ out,
                                                        OutT* __restrict__ log_out, int64_t n,
                                                        unsigned long long* __restrict__ ctr) {
  constexpr int kB = 128;
  __shared__ double s_tab[Form::kStageTable ? kExpTabSize : 1];
  const Form f = bind_table(form, s_tab);
  Tally tl{0u, 0u, 0u, 0u, 0u, 0u, 0u};
  unsigned evals = 0;
  const bool want_log = (log_out != nullptr);
  for (int64_t base = (int64_t)blockIdx.x * kB; base < n; base += (int64_t)gridDim.x * kB) {
    const int64_t i = base + threadIdx.x;
    const bool valid = i < n;
    OutT k, lk;
    eval_out_f32_coop<L>(f, valid, valid ? x[i] : 1.0, valid ? nu[i] : 1.0, tl, evals, k, lk,
                         want_log);
    if (valid) {
      out[i] = k;
      if (log_out != nullptr) log_out[i] = lk;
    }
  }
  flush_tally(ctr, tl, evals);
}

// K, dK/dx and dK/dnu of the plain form, 128 pairs per block and round, in
// chunks sorted by the cost bucket (sort_chunk).  Domain: x = 0 gives (+inf,
// -inf, NaN), x = +inf gives (0, 0, 0), x < 0 or NaN and non-finite nu give
// NaN; dK/dnu is odd in nu (K_{-nu} = K_nu).  Null outputs are skipped.
template <class Form>
__global__ void __launch_bounds__(128, 4) eval_grad_kernel(const Form form, const double* __restrict__ x,
                                                        const double* __restrict__ nu,
                                                        double* __restrict__ k,
                                                        double* __restrict__ dkdx,
                                                        double* __restrict__ dkdnu, int64_t n,
                                                        unsigned long long* __restrict__ ctr) {
  constexpr int kB = 128;
  __shared__ double s_tab[Form::kStageTable ? kExpTabSize : 1];
  __shared__ unsigned short s_perm[kSortChunk];
  __shared__ unsigned s_cnt[64];
  const Form f = bind_table(form, s_tab);
  Tally tl{0u, 0u, 0u, 0u, 0u, 0u, 0u};
  unsigned evals = 0;
  const double qnan = __longlong_as_double(0x7ff8000000000000LL);
  int64_t lo, hi;
  block_range(n, lo, hi);
  for (int64_t base = lo; base < hi; base += kSortChunk) {
    const int cnt = (int)(hi - base < kSortChunk ? hi - base : kSortChunk);
    sort_chunk(x, nu, base, cnt, s_perm, s_cnt,
               [](double xi, double vi) { return eval_cost_bucket(xi, vi); });
    const int rounds = (cnt + kB - 1) / kB;
    for (int r = 0; r < rounds; ++r) {
      const int p = sorted_slot(r);
      if (p >= cnt) continue;
      const int64_t i = base + s_perm[p];
      const double xi = x[i], vi = nu[i], av = fabs(vi);
      double kk = qnan, dx = qnan, dn = qnan;
      if (xi > 0.0 && xi < kInf && av < kInf) {
        f.eval_grad(xi, av, tl, evals, kk, dx, dn);
        if (vi < 0.0) dn = -dn;
      } else if (xi == 0.0 && av < kInf) {
        kk = kInf;
        dx = -kInf;
      } else if (xi == kInf && av < kInf) {
        kk = dx = dn = 0.0;
      }
      if (k != nullptr) k[i] = kk;
      if (dkdx != nullptr) dkdx[i] = dx;
      if (dkdnu != nullptr) dkdnu[i] = dn;
    }
  }
  flush_tally(ctr, tl, evals);
}

constexpr int kTile = 32;     // tile edge (rows and columns)
constexpr int kWarps = 8;     // 256 threads: warp w computes columns w, w+8, w+16, w+24
constexpr int kThreads = kWarps * 32;

// One 32 x 32 tile (I, J), I >= J, of a symmetric matrix: lane i of warp w
// computes M(r0 + i, c0 + c) for c = w, w + WARPS, ...: a warp covers one
// column against 32 consecutive (Morton-near) rows, so its lanes see similar
// distances.  The tile is staged in shared memory and stored twice with
// coalesced 32-element column segments: as block (I, J) and, transposed, as
// block (J, I).  Diagonal tiles are computed whole (both halves).  Callers
// synchronise the block before the shared arrays are reused.
template <typename OutT>
struct SymTileSmem {
  Loc r[kTile], c[kTile];
  OutT tile[kTile][kTile + 1];
};

__device__ __forceinline__ void stage_loc(Loc& L, const double* __restrict__ locs, int64_t n,
                                          int64_t i) {
  L.x = (i < n) ? locs[i] : 0.0;
  L.y = (i < n) ? locs[n + i] : 0.0;
  split_f(L.x, L.xh, L.xl);
  split_f(L.y, L.yh, L.yl);
}

template <class Form, typename OutT, int WARPS>
__device__ __forceinline__ void sym_tile(const Form& form, SymTileSmem<OutT>& sm,
                                         const double* __restrict__ locs,
                                         int64_t n, int64_t I, int64_t J, const MaternParams& mp,
                                         OutT* __restrict__ out, int64_t ld, Tally& tl,
                                         unsigned& evals) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t r0 = I * kTile, c0 = J * kTile;
  if (warp == 0) stage_loc(sm.r[lane], locs, n, r0 + lane);
  else if (warp == 1) stage_loc(sm.c[lane], locs, n, c0 + lane);
  __syncthreads();
#pragma unroll 1
  for (int c = warp; c < kTile; c += WARPS) {
    OutT v = (OutT)0;
    const bool in = r0 + lane < n && c0 + c < n;
    if constexpr (Form::kFloatEval) {
      v = matern_out_f32_coop<Form, OutT>(form, in, sm.r[lane], sm.c[c], mp, tl, evals);
    } else {
      if (in) v = form.template matern_out<OutT>(sm.r[lane], sm.c[c], mp, tl, evals);
    }
    sm.tile[lane][c] = v;
  }
  __syncthreads();
  if constexpr (sizeof(OutT) == sizeof(float)) {
    // FP32 output, interior tile, 16-byte aligned columns: 16-byte stores,
    // 256 per block half (item t: column t / 8, rows 4 (t % 8) .. 4 (t % 8)
    // + 3; a warp writes four whole 128-byte column segments).
    if (r0 + kTile <= n && c0 + kTile <= n && (ld & 3) == 0 &&
        ((uintptr_t)out & 15) == 0) {
#pragma unroll
      for (int t = threadIdx.x; t < kTile * kTile / 4; t += WARPS * 32) {
        const int c = t >> 3, q = (t & 7) * 4;
        float4 v;
        v.x = sm.tile[q][c];
        v.y = sm.tile[q + 1][c];
        v.z = sm.tile[q + 2][c];
        v.w = sm.tile[q + 3][c];
        *reinterpret_cast<float4*>(out + (r0 + q) + (c0 + c) * ld) = v;
        if (I != J) {  // block (J, I): entry (c0 + i, r0 + c) = tile[c][i]
          v.x = sm.tile[c][q];
          v.y = sm.tile[c][q + 1];
          v.z = sm.tile[c][q + 2];
          v.w = sm.tile[c][q + 3];
          *reinterpret_cast<float4*>(out + (c0 + q) + (r0 + c) * ld) = v;
        }
      }
      return;
    }
  }
#pragma unroll
  for (int c = warp; c < kTile; c += WARPS) {
    const int64_t i = r0 + lane, j = c0 + c;
    if (i < n && j < n) out[i + j * ld] = sm.tile[lane][c];
  }
  if (I != J) {
#pragma unroll
    for (int c = warp; c < kTile; c += WARPS) {
      const int64_t i = c0 + lane, j = r0 + c;  // entry (c0+lane, r0+c) = M(r0+c, c0+lane)
      if (i < n && j < n) out[i + j * ld] = sm.tile[c][lane];
    }
  }
}

// Lower-triangle tile number t = I (I + 1)/2 + J  ->  (I, J).
__device__ __forceinline__ void tri_tile(int64_t t, int64_t& I, int64_t& J) {
  I = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while (I * (I + 1) / 2 > t) --I;
  while ((I + 1) * (I + 2) / 2 <= t) ++I;
  J = t - I * (I + 1) / 2;
}

// Lower-triangle tiles in block-column order: with nb block rows, tile
// number T = off(J) + (I - J), off(J) = J nb - J (J - 1)/2, for I >= J.
// After the tiles of block-columns 0 .. J - 1 every entry in a row or a
// column below 32 J is final, which is what lets a caller copy finished
// panels while the next ones are computed.
__device__ __forceinline__ int64_t col_tile_offset(int64_t J, int64_t nb) {
  return J * nb - J * (J - 1) / 2;
}
__device__ __forceinline__ void col_tile(int64_t T, int64_t nb, int64_t& I, int64_t& J) {
  const double b = 2.0 * (double)nb + 1.0;
  J = (int64_t)(0.5 * (b - sqrt(fmax(b * b - 8.0 * (double)T, 0.0))));
  if (J < 0) J = 0;
  while (J > 0 && col_tile_offset(J, nb) > T) --J;
  while (col_tile_offset(J + 1, nb) <= T) ++J;
  I = J + (T - col_tile_offset(J, nb));
}

// Full symmetric matrix: block b computes the lower-triangle tiles
// [b, b + 1, ..., b + Form::kTilesPerBlock - 1] (then strides by the grid,
// which only matters beyond 2^31 blocks).  Many short blocks let the
// hardware block scheduler balance the uneven tile costs across the SMs.
// col_base < 0: the whole triangle in row order (tri_tile); else tile tix is
// number col_base + tix of the block-column order (col_tile), for writing a
// range of block-columns.
template <class Form, typename OutT>
__global__ void __launch_bounds__(kThreads, Form::kMinBlocks) matern_sym_kernel(
    const Form form, const double* __restrict__ locs, int64_t n, const MaternParams mp,
    OutT* __restrict__ out, int64_t ld, int64_t ntiles, unsigned long long* __restrict__ ctr,
    int64_t col_base) {
  __shared__ SymTileSmem<OutT> sm;
  __shared__ double s_tab[Form::kStageTable ? kExpTabSize : 1];
  const Form f = bind_table(form, s_tab);
  Tally tl{0u, 0u, 0u, 0u, 0u, 0u, 0u};
  unsigned evals = 0;
  constexpr int kPer = Form::kTilesPerBlock;
  for (int64_t base = (int64_t)blockIdx.x * kPer; base < ntiles; base += (int64_t)gridDim.x * kPer) {
    const int64_t end = min(base + kPer, ntiles);
    for (int64_t tix = base; tix < end; ++tix) {
      int64_t I, J;
      if (col_base < 0) tri_tile(tix, I, J);
      else col_tile(col_base + tix, (n + kTile - 1) / kTile, I, J);
      __syncthreads();  // the previous tile's shared data is no longer read
      sym_tile<Form, OutT, kWarps>(f, sm, locs, n, I, J, mp, out, ld, tl, evals);
    }
  }
  flush_tally_block(ctr, tl, evals);
}

// General m x n block (Algorithm 3's single tile between two location sets),
// tiles assigned to blocks as in matern_sym_kernel.
template <class Form, typename OutT>
__global__ void __launch_bounds__(kThreads, Form::kMinBlocks) matern_block_kernel(
    const Form form, const double* __restrict__ locs1, int64_t m, const double* __restrict__ locs2, int64_t n,
    const MaternParams mp, OutT* __restrict__ out, int64_t ld, int64_t tiles_m,
    int64_t ntiles, unsigned long long* __restrict__ ctr) {
  __shared__ Loc s_r[kTile], s_c[kTile];
  __shared__ double s_tab[Form::kStageTable ? kExpTabSize : 1];
  const Form f = bind_table(form, s_tab);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  Tally tl{0u, 0u, 0u, 0u, 0u, 0u, 0u};
  unsigned evals = 0;
  constexpr int kPer = Form::kTilesPerBlock;
  for (int64_t base = (int64_t)blockIdx.x * kPer; base < ntiles; base += (int64_t)gridDim.x * kPer) {
    const int64_t end = min(base + kPer, ntiles);
    for (int64_t tix = base; tix < end; ++tix) {
      const int64_t r0 = (tix % tiles_m) * kTile, c0 = (tix / tiles_m) * kTile;
      __syncthreads();
      if (warp == 0) stage_loc(s_r[lane], locs1, m, r0 + lane);
      else if (warp == 1) stage_loc(s_c[lane], locs2, n, c0 + lane);
      __syncthreads();
#pragma unroll 1
      for (int k = 0; k < kTile / kWarps; ++k) {
        const int c = warp + kWarps * k;
        const int64_t i = r0 + lane, j = c0 + c;
        if (i < m && j < n) out[i + j * ld] = f.template matern_out<OutT>(s_r[lane], s_c[c], mp, tl, evals);
      }
    }
  }
  flush_tally_block(ctr, tl, evals);
}

// Blocks for tile kernels: ceil(ntiles / per_block), capped at 2^31 - 1.
inline int tile_grid(int64_t ntiles, int per_block) {
  const int64_t g = (ntiles + per_block - 1) / per_block;
  return (int)(g < 1 ? 1 : (g > 2147483647 ? 2147483647 : g));
}

// Blocks for a grid-stride launch: min(work, SMs x per_sm).
int grid_for(int64_t work_items, int per_sm);

// The grid of one wave of per_sm blocks per SM for n pairs in rounds of 128,
// with no block left without a round (block_range).
inline int one_wave_grid(int64_t n, int per_sm) {
  const int64_t slots = (int64_t)current_sm_count() * per_sm;
  const int64_t rounds = (n + 127) / 128;
  const int64_t per = (rounds + slots - 1) / slots;  // rounds per block
  return (int)((rounds + per - 1) / per);
}

template <class Form, typename OutT>
cudaError_t launch_eval_coop(const Form& form, int lanes, int grid, const double* x,
                             const double* nu, OutT* out, OutT* log_out, int64_t n,
                             unsigned long long* ctr, cudaStream_t s) {
  switch (lanes) {
    case 2: eval_coop_kernel<Form, OutT, 2><<<grid, 128, 0, s>>>(form, x, nu, out, log_out, n, ctr); break;
    case 4: eval_coop_kernel<Form, OutT, 4><<<grid, 128, 0, s>>>(form, x, nu, out, log_out, n, ctr); break;
    case 8: eval_coop_kernel<Form, OutT, 8><<<grid, 128, 0, s>>>(form, x, nu, out, log_out, n, ctr); break;
    default: eval_coop_kernel<Form, OutT, 1><<<grid, 128, 0, s>>>(form, x, nu, out, log_out, n, ctr); break;
  }
  return cudaGetLastError();
}

// lanes: for the FP32 forms, the lanes per evaluation in the node loop (1, 2,
// 4, 8; eval_coop_kernel); the FP64 forms take one lane per evaluation.
template <class Form>
cudaError_t launch_eval_form(const Form& form, const double* x, const double* nu, void* out, void* log_out,
                             bk_dtype out_t, int64_t n, unsigned long long* ctr, cudaStream_t s,
                             int lanes = 1) {
  if (n == 0) return cudaSuccess;
  if constexpr (Form::kFloatEval) {
    const int grid = grid_for((n + 127) / 128, 16);
    if (out_t == BK_F64)
      return launch_eval_coop(form, lanes, grid, x, nu, (double*)out, (double*)log_out, n, ctr, s);
    return launch_eval_coop(form, lanes, grid, x, nu, (float*)out, (float*)log_out, n, ctr, s);
  } else {
    // one wave of the resident slots (6 blocks per SM), each block taking an
    // equal contiguous chunk of whole rounds (block_range)
    const int grid = one_wave_grid(n, 6);
    if (out_t == BK_F64)
      eval_kernel<Form, double><<<grid, 128, 0, s>>>(form, x, nu, (double*)out, (double*)log_out,
                                                     n, ctr);
    else
      eval_kernel<Form, float><<<grid, 128, 0, s>>>(form, x, nu, (float*)out, (float*)log_out, n,
                                                    ctr);
    return cudaGetLastError();
  }
}

template <class Form>
cudaError_t launch_matern_sym_form(const Form& form, const double* locs, int64_t n, double sigma2, double beta,
                                   double nu, void* out, int64_t ld, bk_dtype out_t,
                                   unsigned long long* ctr, cudaStream_t s,
                                   const SymRange& range = SymRange{}) {
  if (n == 0) return cudaSuccess;
  const int64_t nb = (n + kTile - 1) / kTile;
  int64_t ntiles = nb * (nb + 1) / 2, col_base = -1;
  if (range.j1 >= 0) {  // block-columns [j0, j1) in block-column order
    const int64_t j0 = range.j0 < 0 ? 0 : range.j0, j1 = range.j1 < nb ? range.j1 : nb;
    if (j1 <= j0) return cudaSuccess;
    col_base = j0 * nb - j0 * (j0 - 1) / 2;
    ntiles = (j1 * nb - j1 * (j1 - 1) / 2) - col_base;
  }
  const int grid = tile_grid(ntiles, Form::kTilesPerBlock);
  const MaternParams mp = matern_params_host(sigma2, beta, nu);
  if (out_t == BK_F64)
    matern_sym_kernel<Form, double><<<grid, kThreads, 0, s>>>(form, locs, n, mp, (double*)out, ld,
                                                              ntiles, ctr, col_base);
  else
    matern_sym_kernel<Form, float><<<grid, kThreads, 0, s>>>(form, locs, n, mp, (float*)out, ld,
                                                             ntiles, ctr, col_base);
  return cudaGetLastError();
}

template <class Form>
cudaError_t launch_matern_block_form(const Form& form, const double* locs1, int64_t m, const double* locs2,
                                     int64_t n, double sigma2, double beta, double nu, void* out,
                                     int64_t ld, bk_dtype out_t, unsigned long long* ctr,
                                     cudaStream_t s) {
  if (m == 0 || n == 0) return cudaSuccess;
  const int64_t tm = (m + kTile - 1) / kTile, tn = (n + kTile - 1) / kTile;
  const int64_t ntiles = tm * tn;
  const int grid = tile_grid(ntiles, Form::kTilesPerBlock);
  const MaternParams mp = matern_params_host(sigma2, beta, nu);
  if (out_t == BK_F64)
    matern_block_kernel<Form, double><<<grid, kThreads, 0, s>>>(
        form, locs1, m, locs2, n, mp, (double*)out, ld, tm, ntiles, ctr);
  else
    matern_block_kernel<Form, float><<<grid, kThreads, 0, s>>>(
        form, locs1, m, locs2, n, mp, (float*)out, ld, tm, ntiles, ctr);
  return cudaGetLastError();
}

}  // namespace bk
