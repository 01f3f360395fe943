// The two arithmetic forms of one K_nu evaluation and one Matern entry, as
// policies for the kernels of bk_tiles.cuh:
//  * FormF64, the plain form: FP64 search and quadrature (bk_math64.cuh);
//  * FormF32, the precision form: FP32 search and quadrature on the FMA and
//    MUFU pipes (bk_math32.cuh), FP64 distance and log-domain normalisation.
#pragma once

#include "bk.h"
#include "bk_math32.cuh"
#include "bk_math64.cuh"
#include "bk_matern_common.cuh"
#include "bk_series.cuh"

namespace bk {

// A pair's sorting key for the bare evaluations: an estimate of its node
// count, monotone in the two things that set it, the window's width (which
// grows like ln(1 + 74/x) past the peak, 74 = 2 log(1/eps)) and the
// strip-bound step (which shrinks like 1/(30 + 3 nu)); in FP32 on truncated
// copies.  Positive floats order like their bit patterns.  Any key is valid:
// it only groups pairs of similar cost into warps.
__device__ __forceinline__ unsigned eval_cost_key(double x, double nu) {
  const float xf = f32_trunc(x), nf = fabsf(f32_trunc(nu));
  float r, l2;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(xf));
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l2) : "f"(fmaf(74.0f, r, 1.0f)));
  const float est = (l2 + 1.5f) * fmaf(3.0f, nf, 30.0f);
  return (est > 0.0f && est < 3.0e38f) ? __float_as_uint(est) : 0xfffffffeu;
}

// The bare evaluations' cost bucket (0 .. 63) for sort_chunk: the node-count
// estimate of eval_cost_key (about 72 .. 1,600 for x in [1e-3, 140] and
// nu <= 20) on a log scale of 12 buckets per octave, in 1 .. 62; pairs
// outside the domain take 63.
__device__ __forceinline__ int eval_cost_bucket(double x, double nu) {
  const unsigned key = eval_cost_key(x, nu);
  if (key >= 0xfffffffeu) return 63;
  float l2;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l2) : "f"(__uint_as_float(key)));
  const int b = __float2int_rd(l2 * 12.0f) - 70;
  return b < 1 ? 1 : (b > 62 ? 62 : b);
}

// The element-wise domain rules of the C-ABI around a form's evaluation.
template <class Form>
__device__ __forceinline__ double eval_domain(const Form& form, double x, double nu, Tally& tl,
                                              unsigned& evals, double& log_k, bool want_log) {
  nu = fabs(nu);
  if (x > 0.0 && x < kInf && nu < kInf) return form.eval(x, nu, tl, evals, log_k, want_log);
  if (x == 0.0 && nu == nu) {
    log_k = kInf;
    return kInf;
  }
  if (x == kInf && nu < kInf) {
    log_k = -kInf;
    return 0.0;
  }
  log_k = __longlong_as_double(0x7ff8000000000000LL);
  return log_k;
}

// FP32 start values for the plain form's FP64 search: the FP32 search run
// on the same eps (2^-52) inside x in [1e-4, 1e4], nu <= 40, where its sinh
// and cosh stay accurate; none outside (the FP64 search then starts from
// its own bounds).  Its iterations are FP32 work and are not tallied: the
// plain form's counters count FP64 Newton iterations.
__device__ __forceinline__ const Start32* plain_starts_f(float xf, float nu, Start32& st) {
  if (!(xf >= 1e-4f && xf <= 1e4f && nu <= 40.0f)) return nullptr;
  Tally fp32_work{0u, 0u, 0u, 0u, 0u, 0u, 0u};
  const Window32 w = window_f32(xf, nu, (float)kLogInvEps64, fp32_work);
  st = Start32{w.ts, w.t0, w.t1, w.cs};
  return &st;
}
__device__ __forceinline__ const Start32* plain_starts(double x, float nu, Start32& st) {
  return plain_starts_f(f32_trunc(x), nu, st);
}

// Every form carries `tab`, the 2^{j/4096} table of exp2s.  All forms read
// the global table through L1, where its 32 KB stay resident: a per-block
// shared-memory copy (kStageTable, bind_table) cost more than it saved,
// since a block computes one tile, or one short chunk of pairs (measured:
// +0.3 % on the FP64 tile writer, +3 % on 10^5 bare evaluations without it).  kTilesPerBlock is the
// number of 32 x 32 tiles one block of the tile kernels computes, and
// kMinBlocks the resident 256-thread blocks per SM the tile kernels are
// compiled for (it caps their registers: 3 -> 85, 4 -> 64).
// kSeries: whether the form has the small-x series branch at all (a separate
// instantiation, so that the default form carries no call site for it).
template <bool kSeries>
struct FormF64T {
  static constexpr bool kStageTable = false;
  static constexpr int kTilesPerBlock = 1;
  static constexpr int kMinBlocks = 3;
  static constexpr bool kFloatEval = false;
  const double* tab;
  bool search_f64;      // FP64 Newton search for every point (no FP32 roots)
  double series_below;  // x below which Temme's series replaces the integral (0: never)
  const double* wnu = nullptr;  // e^{-2 nu h} on kCoshTab's steps for the launch's nu, or null
  static constexpr bool kDecayTable = true;

  // The bare evaluations' cost bucket (sort_chunk): an estimate of the node
  // count from the arguments alone (eval_cost_bucket), and 0 for the series.
  // The exact count from the FP32 window costs a second window search per
  // pair, more than the better ordering saves (measured).
  __device__ __forceinline__ int sort_bucket(double x, double nu) const {
    if (kSeries && x < series_below) return 0;
    return eval_cost_bucket(x, nu);
  }

  // log K from Temme's series (Sec. IV-A), tallied.
  __device__ __forceinline__ double series(double x, double nu, Tally& tl) const {
    unsigned terms;
    const double lk = series_log_k(x, nu, terms);
    ++tl.series;
    tl.nodes += terms;
    return lk;
  }

  __device__ __forceinline__ double eval(double x, double nu, Tally& tl, unsigned& evals,
                                         double& log_k, bool want_log) const {
    ++evals;
    if (kSeries && x < series_below) {
      log_k = series(x, nu, tl);
      return exp_tab_full(log_k, tab);
    }
    Start32 st;
    const Start32* sp = search_f64 ? nullptr : plain_starts(x, f32_trunc(nu), st);
    double hS;
    const double sc =
        scale_f64((0.5 * kExpScale) * x, nu, kPlainLog2OverTol, kPlainMaxNodes, tab, hS, tl, sp);
    if (!want_log && (__double2hiint(sc) | __double2loint(sc)) == 0) return hS;  // t0 = 0
    const bool big = !bits_le(sc, 700.0);
    const double lh = (want_log || big) ? log_tab(hS, tab) : 0.0;
    if (want_log) log_k = sc + lh;
    return big ? exp_tab_full(sc + lh, tab) : exp_tab_full(sc, tab) * hS;
  }

  // K, dK/dx and dK/dnu for finite x > 0, nu >= 0 on one set of nodes
  // (scale3_f64): FP32 roots for the orders nu and nu + 1 as the window.
  __device__ __forceinline__ void eval_grad(double x, double nu, Tally& tl, unsigned& evals,
                                            double& k, double& dkdx, double& dkdnu) const {
    ++evals;
    Start32 st, st1;
    const Start32* sp = search_f64 ? nullptr : plain_starts(x, f32_trunc(nu), st);
    const Start32* sp1 = (sp != nullptr) ? plain_starts(x, f32_trunc(nu + 1.0), st1) : nullptr;
    if (sp1 == nullptr) sp = nullptr;
    double hS, hSx, hSn;
    const double sc = scale3_f64(x, nu, tab, sp, sp1, hS, hSx, hSn, tl);
    if (sc > 700.0) {  // e^sc alone would overflow where the products need not
      k = exp_tab_full(sc + log_tab(hS, tab), tab);
      dkdx = -exp_tab_full(sc + log_tab(hSx, tab), tab);
      dkdnu = (hSn > 0.0) ? exp_tab_full(sc + log_tab(hSn, tab), tab) : 0.0;
      return;
    }
    const double e = exp_tab_full(sc, tab);
    k = e * hS;
    dkdx = -e * hSx;
    dkdnu = e * hSn;
  }

  // a2 + a3..a7 for one entry: distance, x = r / beta, log K_nu(x),
  // M = exp(log prefactor + nu log x + log K).  sigma^2 where r == 0
  // (Algorithm 3 tests the computed distance for exact zero).  x is carried
  // as xh = x K/2 (K = 4096/ln 2), the node loop's half-scaled argument, from
  // one product and the integer-pipe root: xh = sqrt(r^2 xh_c2) with the
  // matrix's constant xh_c2 = (K/2 / beta)^2.
  __device__ __forceinline__ double matern(const Loc& a, const Loc& b, const MaternParams& mp,
                                           Tally& tl, unsigned& evals) const {
    const double dx = b.x - a.x, dy = b.y - a.y;
    const double r2 = fma(dx, dx, dy * dy);
    if (!bits_pos(r2)) return mp.sigma2;  // r == 0 (r2 >= 0)
    const double xh = sqrt_int(r2 * mp.xh_c2);
    ++evals;
    if constexpr (kSeries) {
      const double z = xh * kTwoOverK;
      if (z < series_below)
        return exp_tab_full(fma(mp.nu, log_tab(z, tab), mp.log_pref) + series(z, mp.nu, tl), tab);
    }
    Start32 st;
    const Start32* sp =
        search_f64 ? nullptr : plain_starts_f(f32_trunc(xh) * (float)kTwoOverK, mp.nu_hi, st);
    double hS;
    const double sc = scale_f64(xh, mp.nu, kPlainLog2OverTol, kPlainMaxNodes, tab, hS, tl, sp, wnu);
    // exp(a1 + nu log x + sc) hS with the exponent formed in the table's
    // units: log x = log(xh 2^-12) + ln(2 ln 2), log(xh 2^-12) = nd ln2/4096 +
    // log1p(d) from the integer pipe, so u = K (a1 + nu ln(2 ln 2)) + nu nd +
    // nu K log1p(d) + K sc (the constant per matrix): two FMAs, and a third
    // only for windows that do not start at t = 0 (sc != 0)
    double nd;
    const double l1p = log_tab_parts(xh, tab, nd, -12);
    double u = fma(mp.nu_k, l1p, fma(mp.nu, nd, mp.log_pref_kh));
    if ((__double2hiint(sc) | __double2loint(sc)) != 0) u = fma(sc, kExpScale, u);
    return exp_units_full(u, tab) * hS;
  }

  template <typename OutT>
  __device__ __forceinline__ OutT matern_out(const Loc& a, const Loc& b, const MaternParams& mp,
                                             Tally& tl, unsigned& evals) const {
    return to_out<OutT>(matern(a, b, mp, tl, evals));
  }

  template <typename OutT>
  __device__ __forceinline__ void eval_out(double x, double nu, Tally& tl, unsigned& evals,
                                           OutT& k, OutT& log_k, bool want_log) const {
    double lk = 0.0;
    k = to_out<OutT>(eval_domain(*this, x, nu, tl, evals, lk, want_log));
    log_k = to_out<OutT>(lk);
  }
};

using FormF64 = FormF64T<false>;        // the plain form
using FormF64Series = FormF64T<true>;   // the plain form with Temme's series below a threshold

// The paper's refined algorithm (Algorithm 2) in FP64: Temme's series below
// series_below (0.1 in the paper), else the fixed window [0, t1] with `bins`
// bins (9 and 40 in the paper; Sec. IV-C), no per-point search.
struct FormF64Fixed {
  static constexpr bool kStageTable = false;
  static constexpr int kTilesPerBlock = 1;
  static constexpr int kMinBlocks = 3;
  static constexpr bool kFloatEval = false;
  static constexpr bool kDecayTable = false;
  const double* tab;
  double t1;
  int bins;
  double series_below;

  // The bare evaluations' cost bucket: the series or the fixed b + 1 nodes.
  __device__ __forceinline__ int sort_bucket(double x, double) const {
    return x < series_below ? 0 : 1;
  }

  __device__ __forceinline__ double log_k_of(double x, double nu, Tally& tl, double& hS,
                                             bool& by_series) const {
    by_series = x < series_below;
    if (by_series) {
      unsigned terms;
      const double lk = series_log_k(x, nu, terms);
      ++tl.series;
      tl.nodes += terms;
      hS = 1.0;
      return lk;
    }
    return fixed_scale_f64(x, nu, t1, bins, tab, hS, tl);
  }

  __device__ __forceinline__ double eval(double x, double nu, Tally& tl, unsigned& evals,
                                         double& log_k, bool want_log) const {
    ++evals;
    double hS;
    bool by_series;
    const double sc = log_k_of(x, nu, tl, hS, by_series);
    if (by_series) {
      log_k = sc;
      return exp_tab_full(sc, tab);
    }
    const double lh = (want_log || sc > 700.0) ? log_tab(hS, tab) : 0.0;
    if (want_log) log_k = sc + lh;
    return (sc > 700.0) ? exp_tab_full(sc + lh, tab) : exp_tab_full(sc, tab) * hS;
  }

  __device__ __forceinline__ double matern(const Loc& a, const Loc& b, const MaternParams& mp,
                                           Tally& tl, unsigned& evals) const {
    const double dx = b.x - a.x, dy = b.y - a.y;
    const double r = sqrt(fma(dx, dx, dy * dy));
    if (r == 0.0) return mp.sigma2;
    const double z = r * mp.inv_beta;
    ++evals;
    double hS;
    bool by_series;
    const double sc = log_k_of(z, mp.nu, tl, hS, by_series);
    return exp_tab_full(fma(mp.nu, log_tab(z, tab), mp.log_pref) + sc, tab) * hS;
  }

  template <typename OutT>
  __device__ __forceinline__ OutT matern_out(const Loc& a, const Loc& b, const MaternParams& mp,
                                             Tally& tl, unsigned& evals) const {
    return to_out<OutT>(matern(a, b, mp, tl, evals));
  }

  template <typename OutT>
  __device__ __forceinline__ void eval_out(double x, double nu, Tally& tl, unsigned& evals,
                                           OutT& k, OutT& log_k, bool want_log) const {
    double lk = 0.0;
    k = to_out<OutT>(eval_domain(*this, x, nu, tl, evals, lk, want_log));
    log_k = to_out<OutT>(lk);
  }
};

// The end of one FP32-form Matern entry after the quadrature (a7): the log
// of the entry, (log prefactor - ln 2) + nu (log x + s) - x cosh s (s the
// quadrature's shift point), summed as a double-float and exponentiated in
// FP32 times h S, written as OutT without FP64 instructions.  Near r -> 0
// the terms nu log x and nu s - x cosh s grow (to ~nu ln(2 nu/x)) and
// cancel; the double-float sum (~44 bits, log x to 1e-9 absolute) keeps the
// entry's relative error at the 1e-8 level there.  FP64 only for FP64 output
// beyond the float range.
template <typename OutT>
__device__ __forceinline__ OutT matern_f32_finish(DF z, const Quad32& q,
                                                  const MaternParams& mp) {
  if (!bits_pos(mp.sigma2)) return (OutT)0;  // sigma^2 = 0 (log c = -inf)
  {
    // (log c - ln 2) + nu (log x + s) - x cosh s
    const DF nu = DF{mp.nu_hi, mp.nu_lo};
    DF a = df_add(DF{mp.log_pref_m_ln2_hi, mp.log_pref_m_ln2_lo},
                  df_mul(nu, df_add_f(df_log(z), q.ts)));
    a = df_add(a, df_neg(df_mul(z, q.ch)));
    if constexpr (sizeof(OutT) == sizeof(float)) {
      return df_exp_times(a, q.hS);
    } else {
      if (a.hi >= -85.0f && a.hi <= 85.0f) return widen_f(df_exp_times(a, q.hS));
    }
  }
  const double z64 = (double)z.hi + (double)z.lo;
  const double lz = log_pos(z64);
  return to_out<OutT>(exp_fast(fma(mp.nu, lz, mp.log_pref) + log_scale_from(z64, mp.nu, q)) *
                      (double)q.hS);
}

// a2 for the FP32 forms: x = r / beta as a double-float from the staged
// double-float coordinates (hi is what the FP32 integrand uses).
__device__ __forceinline__ DF matern_x_df(const Loc& a, const Loc& b, const MaternParams& mp) {
  const DF r = df_hypot_diff(a.xh, a.xl, a.yh, a.yl, b.xh, b.xl, b.yh, b.yl);
  if (r.hi == 0.0f) return r;
  return df_mul(r, DF{mp.inv_beta_f, mp.inv_beta_lo});
}

// The FP32 forms' bare evaluation: inside x in [1e-4, 1e4], nu in
// [2^-70, 40] the arguments are split into double-floats by integer
// operations and the result is assembled as for the Matern entries, with no
// FP64 instruction on the way (FP64 output widens the FP32 value exactly);
// elsewhere, and for FP64 output beyond the float range, the form's FP64
// normalisation (eval) and the domain rules of the C-ABI apply.  The node
// loops of the warp's 32 evaluations run on groups of L lanes
// (coop_trapezoid_f32).  The learned form's check (a finite
// positive sum, no node more than e^2 above the predicted peak) is taken after
// the first pass; evaluations that fail it, or whose predicted window was
// unusable, take the searched window in a second pass (only when some lane
// of the warp needs one).  Every lane of the warp must call it; `valid` is
// false for lanes without a pair.
template <int L, class Form, typename OutT>
__device__ __forceinline__ void eval_out_f32_coop(const Form& f, bool valid, double x, double nu,
                                                  Tally& tl, unsigned& evals, OutT& k,
                                                  OutT& log_k, bool want_log) {
  // x > 0 finite and |nu| finite: 64-bit tests of the bits, which the
  // compiler may turn into FP64 comparisons; this kernel is bound by
  // instruction issue, not by the FP64 pipe, so one FP64 compare is cheaper
  // here than several integer instructions (measured 1.5 %)
  const long long xb = __double_as_longlong(x);
  const long long vb = __double_as_longlong(nu) & 0x7fffffffffffffffLL;
  bool okx = false, okn = false;
  DF xd{0.0f, 0.0f}, nd{0.0f, 0.0f};
  if (valid && xb > 0 && xb < 0x7ff0000000000000LL && vb < 0x7ff0000000000000LL) {
    xd = df_from_bits(x, okx);
    nd = df_from_bits(__longlong_as_double(vb), okn);
  }
  const bool fast = okx && okn && xd.hi >= 1e-4f && xd.hi <= 1e4f && nd.hi <= 40.0f;
  auto x64_of = [&] { return x; };
  Window32 w;
  Quad32 q;
  q.hS = 0.0f;
  q.amax = 0.0f;
  Job32 jb = no_job32();
  bool need_search = false;
  if (fast) {
    ++evals;
    if (f.first_window(xd.hi, x64_of, nd.hi, w, tl)) jb = job_f32(xd.hi, nd.hi, nd.lo, w, q, tl);
    else need_search = true;
  }
  float hS, amax;
  coop_trapezoid_f32<L, Form::kChecked>(jb, hS, amax);
  if (jb.N >= 0) {
    q.hS = hS;
    q.amax = amax;
  }
  if constexpr (Form::kChecked) {
    if (fast && !(isfinite(q.hS) && q.hS > 0.0f && q.amax <= 2.0f)) need_search = true;
    if (__any_sync(0xffffffffu, need_search)) {
      Job32 jb2 = no_job32();
      if (need_search) {
        ++tl.fallback;
        w = search_window_f32(xd.hi, x64_of, nd.hi, f.tab, tl);
        jb2 = job_f32(xd.hi, nd.hi, nd.lo, w, q, tl);
      }
      coop_trapezoid_f32<L, Form::kChecked>(jb2, hS, amax);
      if (jb2.N >= 0) {
        q.hS = hS;
        q.amax = amax;
      }
    }
  }
  if (!valid) return;
  if (fast) {
    const DF a = df_log_scale(xd, nd, q);
    if constexpr (sizeof(OutT) == sizeof(float)) {
      k = df_exp_times(a, q.hS);
      if (want_log) log_k = a.hi + (a.lo + kLn2f * mufu_lg2(q.hS));
      return;
    } else {
      if (a.hi >= -85.0f && a.hi <= 85.0f) {
        k = widen_f(df_exp_times(a, q.hS));
        if (want_log) log_k = widen_f(a.hi) + widen_f(a.lo + kLn2f * mufu_lg2(q.hS));
        return;
      }
      --evals;  // counted again by the FP64 path below
    }
  }
  double lk = 0.0;
  const double kd = eval_domain<Form>(f, x, nu, tl, evals, lk, want_log);
  k = to_out<OutT>(kd);
  log_k = to_out<OutT>(lk);
}

// One Matern entry of the FP32 forms with the structure of eval_out_f32_coop
// (one lane per entry): the window and job of every lane, the node loop, then
// the learned form's check, and the searched window for the entries that
// fail it in a second pass taken only when some lane of the warp needs one.
// Every lane of the warp must call it; `valid` is false outside the matrix
// (the result is then 0 and unused).
template <class Form, typename OutT>
__device__ __forceinline__ OutT matern_out_f32_coop(const Form& f, bool valid, const Loc& a,
                                                    const Loc& b, const MaternParams& mp,
                                                    Tally& tl, unsigned& evals) {
  DF z{0.0f, 0.0f};
  if (valid) z = matern_x_df(a, b, mp);
  const bool work = valid && z.hi != 0.0f;  // r == 0 gives sigma^2 (Algorithm 3)
  auto x64_of = [&] { return (double)z.hi + (double)z.lo; };
  Window32 w;
  Quad32 q;
  q.hS = 0.0f;
  q.amax = 0.0f;
  Job32 jb = no_job32();
  bool need_search = false;
  if (work) {
    ++evals;
    if (f.first_window(z.hi, x64_of, mp.nu_hi, w, tl))
      jb = job_f32(z.hi, mp.nu_hi, mp.nu_lo, w, q, tl);
    else
      need_search = true;
  }
  float hS, amax;
  coop_trapezoid_f32<1, Form::kChecked>(jb, hS, amax);
  if (jb.N >= 0) {
    q.hS = hS;
    q.amax = amax;
  }
  if constexpr (Form::kChecked) {
    if (work && !(isfinite(q.hS) && q.hS > 0.0f && q.amax <= 2.0f)) need_search = true;
    if (__any_sync(0xffffffffu, need_search)) {
      Job32 jb2 = no_job32();
      if (need_search) {
        ++tl.fallback;
        w = search_window_f32(z.hi, x64_of, mp.nu_hi, f.tab, tl);
        jb2 = job_f32(z.hi, mp.nu_hi, mp.nu_lo, w, q, tl);
      }
      coop_trapezoid_f32<1, Form::kChecked>(jb2, hS, amax);
      if (jb2.N >= 0) {
        q.hS = hS;
        q.amax = amax;
      }
    }
  }
  if (!work) {
    if (!valid) return (OutT)0;
    return sizeof(OutT) == sizeof(float) ? (OutT)mp.sigma2_f : (OutT)mp.sigma2;
  }
  return matern_f32_finish<OutT>(z, q, mp);
}

// The FP32 precision form (search window).
struct FormF32 {
  static constexpr bool kStageTable = false;
  static constexpr int kTilesPerBlock = 4;
  static constexpr int kMinBlocks = 4;
  static constexpr bool kFloatEval = true;
  static constexpr bool kDecayTable = false;
  static constexpr bool kChecked = false;  // the searched window needs no check
  const double* tab;

  template <class X64>
  __device__ __forceinline__ Quad32 quad(float x, X64 x64_of, float nu, float nu_lo, Window32& w,
                                         Tally& tl) const {
    w = search_window_f32(x, x64_of, nu, tab, tl);
    return quad_f32(x, nu, nu_lo, w, tl);
  }

  // The window tried first by the lane-split evaluation (eval_out_f32_coop).
  template <class X64>
  __device__ __forceinline__ bool first_window(float x, X64 x64_of, float nu, Window32& w,
                                               Tally& tl) const {
    w = search_window_f32(x, x64_of, nu, tab, tl);
    return true;
  }

  // FP64 normalisation (outside the float path of eval_out_f32_coop).
  __device__ __forceinline__ double eval(double x, double nu, Tally& tl, unsigned& evals,
                                         double& log_k, bool) const {
    ++evals;
    const float xf = (float)x, nf = (float)nu, nl = (float)(nu - (double)nf);
    Window32 w;
    const Quad32 q = quad(xf, [&] { return x; }, nf, nl, w, tl);
    const double sc = log_scale_from(x, nu, q);
    log_k = sc + (double)(kLn2f * mufu_lg2(q.hS));
    return exp_fast(sc) * (double)q.hS;
  }


  // a2 as a double-float; a3..a6 in FP32 on x.hi; a7 by matern_f32_finish.
  template <typename OutT>
  __device__ __forceinline__ OutT matern_out(const Loc& a, const Loc& b, const MaternParams& mp,
                                             Tally& tl, unsigned& evals) const {
    const DF z = matern_x_df(a, b, mp);
    if (z.hi == 0.0f) return sizeof(OutT) == sizeof(float) ? (OutT)mp.sigma2_f : (OutT)mp.sigma2;
    ++evals;
    Window32 w;
    const Quad32 q = quad(z.hi, [&] { return (double)z.hi + (double)z.lo; }, mp.nu_hi, mp.nu_lo,
                          w, tl);
    return matern_f32_finish<OutT>(z, q, mp);
  }
};

// Device view (table and margins) of a window network with weights.
LearnedView learned_view(const bk_learned* m);

// FP32 form with the learned window (a10): the window comes from the
// tabulated network, checked (and where needed repaired) in-kernel, else from
// the search (counted as a fallback).  A badly placed predicted peak (a node
// value more than e^2 above the value at the predicted peak, or a non-finite
// sum) also falls back.
struct FormF32Learned {
  static constexpr bool kStageTable = false;
  static constexpr int kTilesPerBlock = 4;
  static constexpr int kMinBlocks = 4;
  static constexpr bool kFloatEval = true;
  static constexpr bool kDecayTable = false;
  static constexpr bool kChecked = true;  // quadratures of predicted windows are checked
  LearnedView lv;
  const double* tab;

  template <class X64>
  __device__ __forceinline__ bool first_window(float x, X64, float nu, Window32& w,
                                               Tally& tl) const {
    return learned_window_f32(lv, x, nu, w, tl.repairs);
  }

  template <class X64>
  __device__ __forceinline__ Quad32 quad(float x, X64 x64_of, float nu, float nu_lo, Window32& w,
                                         Tally& tl) const {
    if (learned_window_f32(lv, x, nu, w, tl.repairs)) {
      const Quad32 q = quad_f32(x, nu, nu_lo, w, tl);
      // A predicted peak more than 2 below the true one (some node exceeds it
      // by that much) would cost FP32 accuracy in the scaled nodes.
      if (isfinite(q.hS) && q.hS > 0.0f && q.amax <= 2.0f) return q;
    }
    ++tl.fallback;
    w = search_window_f32(x, x64_of, nu, tab, tl);
    return quad_f32(x, nu, nu_lo, w, tl);
  }

  __device__ __forceinline__ double eval(double x, double nu, Tally& tl, unsigned& evals,
                                         double& log_k, bool) const {
    ++evals;
    const float xf = (float)x, nf = (float)nu, nl = (float)(nu - (double)nf);
    Window32 w;
    const Quad32 q = quad(xf, [&] { return x; }, nf, nl, w, tl);
    const double sc = log_scale_from(x, nu, q);
    log_k = sc + (double)(kLn2f * mufu_lg2(q.hS));
    return exp_fast(sc) * (double)q.hS;
  }


  template <typename OutT>
  __device__ __forceinline__ OutT matern_out(const Loc& a, const Loc& b, const MaternParams& mp,
                                             Tally& tl, unsigned& evals) const {
    const DF z = matern_x_df(a, b, mp);
    if (z.hi == 0.0f) return sizeof(OutT) == sizeof(float) ? (OutT)mp.sigma2_f : (OutT)mp.sigma2;
    ++evals;
    Window32 w;
    const Quad32 q = quad(z.hi, [&] { return (double)z.hi + (double)z.lo; }, mp.nu_hi, mp.nu_lo,
                          w, tl);
    return matern_f32_finish<OutT>(z, q, mp);
  }
};

}  // namespace bk
