// FP64 device arithmetic for the plain form: exp and log written here (no
// math-library internals), the peak/window search and the self-checked
// trapezoid of Sec. IV-B.
#pragma once

#include <cstdint>

namespace bk {

// ---------------------------------------------------------------------------
// Constants.  ln2 is split Cody-Waite style: kLn2Hi is ln 2 rounded to 32
// significant bits (so k * kLn2Hi is exact for |k| < 2^21) and kLn2Lo is the
// remainder; both were derived from a 50-digit value of ln 2.
constexpr double kLog2e = 0x1.71547652b82fep+0;   // 1 / ln 2
constexpr double kLn2 = 0x1.62e42fefa39efp-1;     // ln 2
constexpr double kLn2Hi = 0x1.62e42fee00000p-1;
constexpr double kLn2Lo = 0x1.a39ef35793c76p-33;
constexpr double kRoundMagic = 6755399441055744.0;  // 1.5 * 2^52: adding it rounds to an integer
constexpr double kSqrt2 = 1.4142135623730951;
// -log(2^-52): the paper's machine epsilon (Sec. IV-C) in the window rule.
constexpr double kLogInvEps64 = 36.04365338911715;

// ---------------------------------------------------------------------------
// Bit-level helpers that keep work off the FP64 pipe: on this GPU FP64
// compares and FP64 <-> FP32 conversions issue to the FP64 unit at its
// 2-per-clock rate, like FMAs, while integer operations do not.

// v > 0 for v not NaN (NaN with a clear sign bit counts as positive).
//
// These tests (and the other bit-pattern tests of this file) are written on
// the 32-bit words: a 64-bit comparison of a double's bits with a constant
// can be folded by the compiler into an FP64 comparison (a masked
// "> 0x7ff0000000000000" test into isnan, say), which takes an FP64-pipe slot
// (measured: one such test per node cost 17 % of the FP64 tile writer's time).
__device__ __forceinline__ bool bits_pos(double v) {
  const int hi = __double2hiint(v);
  return hi > 0 || (hi == 0 && __double2loint(v) != 0);
}
// a <= b for a, b >= 0 (false when a is NaN).
__device__ __forceinline__ bool bits_le(double a, double b) {
  const int ha = __double2hiint(a), hb = __double2hiint(b);
  return ha < hb || (ha == hb && (unsigned)__double2loint(a) <= (unsigned)__double2loint(b));
}
// v truncated to a float (23 stored significand bits) by integer operations
// only (no conversion on the FP64 pipe): magnitudes below 2^-126 give a
// signed zero, above the float range a signed infinity, NaN a NaN.
__device__ __forceinline__ float f32_trunc(double v) {
  const long long b = __double_as_longlong(v);
  const unsigned hi = (unsigned)((unsigned long long)b >> 32);
  const int e = (int)((hi >> 20) & 0x7ff) - 1023;
  const unsigned sign = hi & 0x80000000u;
  const unsigned mant = (unsigned)((b >> 29) & 0x7fffff);
  const unsigned big = sign | 0x7f800000u | ((e == 1024 && (b & 0xfffffffffffffLL) != 0) ? 0x400000u : 0u);
  const unsigned r = (e < -126) ? sign : (e > 127) ? big : (sign | ((unsigned)(e + 127) << 23) | mant);
  return __uint_as_float(r);
}
// A float as a double by integer operations only (exact for every input:
// subnormals are normalised, infinities and NaN payloads kept), so that no
// conversion is issued on the FP64 pipe.
__device__ __forceinline__ double widen_f(float f) {
  const unsigned u = (unsigned)__float_as_int(f);
  const unsigned sign = u & 0x80000000u, ex = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  unsigned hi, lo;
  if (ex == 0xffu) {  // infinity, NaN
    hi = sign | 0x7ff00000u | (m >> 3);
    lo = m << 29;
  } else if (ex != 0u) {
    hi = sign | ((ex + 896u) << 20) | (m >> 3);
    lo = m << 29;
  } else if (m == 0u) {
    hi = sign;
    lo = 0u;
  } else {  // m 2^-149 with its leading bit at p
    const int p = 31 - __clz((int)m);
    const unsigned long long mm = ((unsigned long long)m << (52 - p)) & 0xfffffffffffffULL;
    hi = sign | ((unsigned)(p - 149 + 1023) << 20) | (unsigned)(mm >> 32);
    lo = (unsigned)mm;
  }
  return __hiloint2double((int)hi, (int)lo);
}

// sqrt a for a > 0: an FP32 reciprocal square root of a's leading bits as
// the seed (relative error ~2^-22), then two Newton-Heron steps in FP64,
// s <- s + (a - s^2) h with h = 1/(2 s0) from the seed: the error squares
// to ~2^-44 and then falls below the final rounding (within an ulp).  4 FP64
// operations; a outside [2^-120, 2^120] takes the library square root.
__device__ __forceinline__ double sqrt_pos(double a) {
  const float af = f32_trunc(a);
  if (!(af >= 0x1p-120f && af <= 0x1p120f)) return sqrt(a);
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(af));
  const double s0 = widen_f(af * y), h = widen_f(0.5f * y);
  const double s1 = fma(fma(-s0, s0, a), h, s0);
  return fma(fma(-s1, s1, a), h, s1);
}

// sqrt a for normal a > 0 without FP64 arithmetic, within an ulp (others:
// the library root).  a = A 2^(E - 52) with E even and A in [2^52, 2^54), so
// that sqrt a = S 2^(E/2 - 52) with S = sqrt(N), N = A 2^52, S in [2^52,
// 2^53).  An FP32 seed (rsqrt.approx and one Newton step on a's leading 24
// bits) gives S0 = m 2^k within about 2^-22.5; the first correction
// (N - S0^2) / (2 S0) uses the exact 64-bit residual A - m^2 2^(2k - 52) and
// is taken in FP32 (S1 within about 2^9); the second uses N - S1^2 computed
// exactly as a 128-bit difference (below 2^63 in magnitude), its leading bits
// in FP32.  The bounds were checked by an exact emulation with the hardware
// approximations perturbed by their full error (72,000 cases).
__device__ __forceinline__ double sqrt_int(double a) {
  const long long b = __double_as_longlong(a);
  const int ea = (int)((b >> 52) & 0x7ff) - 1023;
  if (ea == -1023 || ea == 1024) return sqrt(a);  // zero, subnormal, inf, NaN
  const int odd = ea & 1;
  const int E = ea - odd;  // even
  const unsigned long long A = ((unsigned long long)(b & 0xfffffffffffffLL) | (1ULL << 52)) << odd;
  const float af = __uint2float_rn((unsigned)(A >> 30)) * 0x1p-22f;  // exact, in [1, 4)
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(af));
  y = y * fmaf(-0.5f * af, y * y, 1.5f);
  const unsigned sb = __float_as_uint(af * y);  // sqrt(A 2^-52), about [1, 2)
  const int es = (int)((sb >> 23) & 0xff) - 127;
  const unsigned m24 = (sb & 0x7fffffu) | 0x800000u;
  const int k = 29 + es;  // S0 = m24 2^k
  const unsigned long long mm = (unsigned long long)m24 * m24;
  const int sh2 = 2 * k - 52;  // 6 + 2 es
  const long long R0 = (long long)A - (long long)(sh2 >= 0 ? (mm << sh2) : (mm >> -sh2));
  float inv;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(inv) : "f"(__uint2float_rn(m24)));
  // c0 = R0 2^52 / (2 m24 2^k) = R0 inv 2^(51 - k), |R0| < 2^33, |c0| < 2^31
  const float c0f = __int2float_rn((int)(R0 >> 3)) * inv * __int_as_float((51 - k + 3 + 127) << 23);
  const unsigned long long S1 =
      ((unsigned long long)m24 << k) + (unsigned long long)((long long)__float2int_rn(c0f * 0x1p-4f) * 16);
  // N - S1^2 as a 128-bit difference
  const unsigned long long Nlo = A << 52, Nhi = A >> 12;
  const unsigned long long Plo = S1 * S1, Phi = __umul64hi(S1, S1);
  const unsigned long long Rlo = Nlo - Plo;
  const unsigned long long Rhi = Nhi - Phi - (Nlo < Plo ? 1ULL : 0ULL);
  const long long t = (long long)((Rhi << 32) | (Rlo >> 32));  // (N - S1^2) 2^-32
  float rs;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rs) : "f"(__uint2float_rn((unsigned)(S1 >> 29))));
  // c1 = (N - S1^2) / (2 S1) = t 2^32 rs 2^-29 / 2
  const float c1f = __int2float_rn((int)(t >> 3)) * rs * 32.0f;
  const long long S2 = (long long)S1 + __float2int_rn(c1f);
  return __longlong_as_double(((long long)(E / 2 + 1023) << 52) + (S2 - (1LL << 52)));
}

__device__ __forceinline__ double pow2i(int k) {  // 2^k for k in [-1022, 1023]
  return __hiloint2double((k + 1023) << 20, 0);
}

// e^r for |r| <= ln2/2 by its Taylor polynomial of degree 12 (truncation below
// 0.3466^13 / 13! < 2e-16 relative), Horner form.
__device__ __forceinline__ double exp_taylor12(double r) {
  double p = 1.0 / 479001600.0;
  p = fma(p, r, 1.0 / 39916800.0);
  p = fma(p, r, 1.0 / 3628800.0);
  p = fma(p, r, 1.0 / 362880.0);
  p = fma(p, r, 1.0 / 40320.0);
  p = fma(p, r, 1.0 / 5040.0);
  p = fma(p, r, 1.0 / 720.0);
  p = fma(p, r, 1.0 / 120.0);
  p = fma(p, r, 1.0 / 24.0);
  p = fma(p, r, 1.0 / 6.0);
  p = fma(p, r, 0.5);
  p = fma(p, r, 1.0);
  p = fma(p, r, 1.0);
  return p;
}


// e^a over the whole double range (NaN -> NaN, overflow -> inf, deep underflow -> 0).
__device__ __forceinline__ double exp_full(double a) {
  if (a != a) return a;
  if (a > 709.782712893384) return __longlong_as_double(0x7ff0000000000000LL);
  if (a < -745.2) return 0.0;
  double kd = fma(a, kLog2e, kRoundMagic);
  const int k = __double2loint(kd);
  kd -= kRoundMagic;
  double r = fma(-kd, kLn2Hi, a);
  r = fma(-kd, kLn2Lo, r);
  const int k1 = k >> 1;  // split 2^k so both halves are normal numbers
  return (exp_taylor12(r) * pow2i(k1)) * pow2i(k - k1);
}

// log(a) for finite a > 0: a = 2^e m with m in [sqrt(1/2), sqrt(2)), then
// log m = 2 atanh(s), s = (m - 1)/(m + 1), |s| <= 0.1716, from the series
// atanh(s) = s sum_j s^{2j}/(2j+1) up to j = 9 (truncation < 3e-17 relative).
constexpr int kLogOps = 24;  // approximate FP64 op count incl. the division
__device__ __forceinline__ double log_pos(double a) {
  int hi = __double2hiint(a);
  int lo = __double2loint(a);
  int e = 0;
  if (hi < 0x00100000) {  // subnormal: scale into the normal range
    a *= 0x1p54;
    e = -54;
    hi = __double2hiint(a);
    lo = __double2loint(a);
  }
  e += (hi >> 20) - 1023;
  double m = __hiloint2double((hi & 0x000fffff) | 0x3ff00000, lo);  // [1, 2)
  if (m > kSqrt2) {
    m *= 0.5;
    e += 1;
  }
  const double s = (m - 1.0) / (m + 1.0);
  const double s2 = s * s;
  double q = 1.0 / 19.0;
  q = fma(q, s2, 1.0 / 17.0);
  q = fma(q, s2, 1.0 / 15.0);
  q = fma(q, s2, 1.0 / 13.0);
  q = fma(q, s2, 1.0 / 11.0);
  q = fma(q, s2, 1.0 / 9.0);
  q = fma(q, s2, 1.0 / 7.0);
  q = fma(q, s2, 1.0 / 5.0);
  q = fma(q, s2, 1.0 / 3.0);
  q = fma(q, s2, 1.0);
  const double lm = 2.0 * s * q;
  const double ed = (double)e;
  return fma(ed, kLn2Hi, fma(ed, kLn2Lo, lm));
}

// ---------------------------------------------------------------------------
// Table-driven exponential for the hot loops (Tang's method with a 4096-entry
// table).  The kernels work in scaled units u = a K, K = 4096/ln 2, so that
// e^a = 2^{u/4096}: u = 4096 k + j + rho (round to nearest, |rho| <= 1/2),
// e^a = 2^k 2^{j/4096} e^{y}, y = rho ln2/4096, |y| <= c = 8.46e-5, and e^y from
// the quadratic 1 + y (1 + c^2/8) + y^2/2: the Taylor quadratic with the
// cubic term's best linear replacement on [-c, c] (y^3 ~ (3c^2/4) y, the
// Chebyshev projection), relative error below 2.6e-14.  2^{j/4096} comes from
// kExp2Tab (32 KB, read through L1); 2^k is added to the entry's exponent
// field.  Valid for u in [-1022 * 4096,
// 1023 * 4096] (a in [-708, 709]); below that the result is clamped to about
// 2^-1022, not garbage.
static __device__ const double kExp2Tab[4096] = {
#include "bk_exp2_table.inc"
};
constexpr int kExpTabBits = 12;
constexpr int kExpTabSize = 1 << kExpTabBits;
constexpr double kExpScale = 0x1.71547652b82fep+12;  // 4096 / ln 2
constexpr double kExpC1 = 0x1.62e42fefa39efp-13;     // ln2 / 4096
constexpr double kExpK1 = 0x1.62e42ff4f7b0ap-13;     // (ln2/4096)(1 + c^2/8)
constexpr double kExpK2 = 0x1.ebfbdff82c58fp-27;     // (ln2/4096)^2 / 2
constexpr double kExpC3 = 0x1.c6b08d704a0c0p-41;     // (ln2/4096)^3 / 6
constexpr double kExpC1Hi = 0x1.62e42ff000000p-13;   // ln2/4096 to 29 bits
constexpr double kExpC1Lo = -0x1.718432a1b0e26p-47;  // ln2/4096 - kExpC1Hi

// Copies the table into a shared-memory array of kExpTabSize doubles (all
// threads of the block take part) and synchronises the block.
__device__ __forceinline__ void exp_table_init(double* tab) {
  for (int i = threadIdx.x; i < kExpTabSize; i += blockDim.x) tab[i] = kExp2Tab[i];
  __syncthreads();
}

// 2^{u/4096} for u in scaled units.  FP64 ops: 1 add + 2 sub (rounding and
// rho, exact), 2 fma (polynomial), 1 mul.
constexpr int kExp2sOps = 6;
__device__ __forceinline__ double exp2s(double u, const double* __restrict__ tab) {
  const double v = u + kRoundMagic;
  const int n = __double2loint(v);
  const double rho = u - (v - kRoundMagic);
  const double p = fma(fma(kExpK2, rho, kExpK1), rho, 1.0);
  const double tj = tab[n & (kExpTabSize - 1)];
  const int k = max(n >> kExpTabBits, -1022);
  return p * __hiloint2double(__double2hiint(tj) + (k << 20), __double2loint(tj));
}

// For 0 <= v < 2^22: M = round(v) and rho = v - M (|rho| <= 1/2), both
// exact and on the integer pipe.  With sh the position of v's binary point
// in its 53-bit significand sig, M = (sig + 2^(sh-1)) >> sh and
// rho 2^sh = ((sig + 2^(sh-1)) mod 2^sh) - 2^(sh-1), an integer below 2^53 in
// magnitude, normalised into a double by its leading-bit position.  v < 1/4
// (and 0) gives M = 0, rho = v.  Out of range (v >= 2^22) gives
// M = 4,000,000 and rho = v, so that exp2s_cubic stays finite for finite
// arguments; NaN gives rho = NaN.
__device__ __forceinline__ void round_rem(double v, int& M, double& rho) {
  const long long b = __double_as_longlong(v);
  const int e = (int)((b >> 52) & 0x7ff) - 1023;
  const long long sig = (b & 0xfffffffffffffLL) | 0x10000000000000LL;
  const int sh = 52 - min(max(e, -2), 21);  // 31 .. 54
  const long long half = 1LL << (sh - 1);
  const long long t = sig + half;
  M = (int)(t >> sh);
  const long long R = (t & ((half << 1) - 1)) - half;  // rho 2^sh
  const unsigned long long A = (unsigned long long)(R < 0 ? -R : R);
  const int L = 63 - __clzll((long long)A);  // leading bit (L <= 53)
  const unsigned long long frac = (L <= 52) ? ((A << (52 - L)) & 0xfffffffffffffULL) : 0ULL;
  const unsigned long long rb = ((unsigned long long)(R < 0) << 63) |
                                ((unsigned long long)(L - sh + 1023) << 52) | frac;
  rho = (A == 0ULL) ? 0.0 : __longlong_as_double((long long)rb);
  rho = (e < -2) ? v : rho;
  if (e > 21) {
    M = 4000000;
    rho = v;
  }
}

// Constants of the node loop's exponential (exp2s_fix): K1 = (ln2/4096)(1 +
// c^2/8) in units of 2^-75 and K2 = (ln2/4096)^2/2 in units of 2^-57.
constexpr unsigned long long kExpK1Q75 = (unsigned long long)(kExpK1 * 0x1p75);  // exact
constexpr unsigned long long kExpK2Q57 = (unsigned long long)(kExpK2 * 0x1p57 + 0.5);
static_assert(kExpK1Q75 < (1ULL << 63) && kExpK2Q57 < (1ULL << 32), "fixed-point constants");
// ---------------------------------------------------------------------------
// 64-bit fixed point for the uncentred node loop (node_sum_cosh), whose node
// exponent U_j = D_j - G_j (D_j = K x cosh t_j from the FP64 recurrence, G_j
// = K nu (t_j - t_start) a multiple of a fixed step) is formed on the integer
// pipe in units of 2^-40: |U| < 2^23 fits 64 bits with 40 fractional bits.

// D in [0.25, 2^22) (a node loop's K x cosh t_j) in units of 2^-40: the
// significand shifted by the exponent, truncated (below 2^-40 absolute, the
// error of a relative 1.7e-16 in 2^{-D/4096}; exact for D >= 2^12).
__device__ __forceinline__ long long fix40_node(double D) {
  const int e = (int)((unsigned)__double2hiint(D) >> 20) - 1023;  // -2 .. 21
  const unsigned long long sig =
      (((unsigned long long)__double_as_longlong(D) & 0xfffffffffffffULL) | 0x10000000000000ULL)
      << 11;                                                     // D 2^{63 - e}
  return (long long)(sig >> (23 - e));
}

// w in [0, 1] in units of 2^-63 (w = 1 gives 2^63), truncated; values above 1
// are clamped to 1.
__device__ __forceinline__ unsigned long long fix63_unit(double w) {
  const int e = (int)((unsigned)__double2hiint(w) >> 20) - 1023;
  const unsigned long long sig =
      (((unsigned long long)__double_as_longlong(w) & 0xfffffffffffffULL) | 0x10000000000000ULL)
      << 11;  // w 2^{63 - e}
  if (e >= 0) return 1ULL << 63;
  return (e < -63) ? 0ULL : sig >> (-e);
}

// r in [0, 1] in units of 2^-64, truncated and clamped below 2^64 (r = 1
// gives 2^64 - 1).
__device__ __forceinline__ unsigned long long fix64_unit(double r) {
  const int e = (int)((unsigned)__double2hiint(r) >> 20) - 1023;
  const unsigned long long sig =
      (((unsigned long long)__double_as_longlong(r) & 0xfffffffffffffULL) | 0x10000000000000ULL)
      << 11;  // r 2^{63 - e}
  if (e >= 0) return ~0ULL;
  return (e < -64) ? 0ULL : sig >> (-1 - e);
}

// 1 + w for w = Wq 2^-63 in [0, 1], rounded to nearest (ties up) by adding
// the 52-bit fraction to the bits of 1.0 (w = 1 carries into the exponent
// field and gives 2.0): integer operations only.
__device__ __forceinline__ double one_plus_w(unsigned long long Wq) {
  return __longlong_as_double(0x3ff0000000000000LL + (long long)((Wq + 1024ULL) >> 11));
}

// 2^{-U/4096} times 2^kAdj for U = U40 2^-40 in (-2^23, 2^23) with the
// result in [2^-1000, 2^1000] (the node loop's range), computed on the
// integer pipe without FP64 arithmetic.  m = round(U) (ties up) is U40 + 2^39
// shifted right by 40 (arithmetically); the remainder rho = U - m in [-1/2,
// 1/2) comes from the low 40 bits of U40 + 2^39, moved to the top of a 64-bit
// word, the top bit flipped (subtracting 1/2) and shifted back by one (rho
// 2^63).  p = 2^{-rho/4096} = 1 - K1 rho + K2 rho^2 (the minimax quadratic,
// relative error below 2.6e-14) is evaluated in 64-bit fixed point: K1 |rho|
// as the high half of a 64 x 64-bit product, K2 rho^2 from the leading 32
// bits of rho (its error below 2^-58), delta = p - 1 in units of 2^-62.  The
// result p T, T = 2^{-m/4096} = 2^k t_j with t_j = 2^{j/4096} from the table,
// is t_j's 53-bit significand M plus delta M (the high half of a 64 x 64-bit
// product, truncated: below 2^-52 relative), renormalised into [2^52, 2^53)
// and given the exponent k.  On GB300 an FP64 operation occupies the FP64
// pipe 32 times as long as an integer instruction occupies its own, so these
// ~30 integer instructions cost less than the 3 FP64 operations of an FP64
// polynomial and product.  The table index and exponent come from -m.  No
// range tests: the callers keep U inside the range.  kAdj = -1 halves the
// result (the trapezoid's end weights).
template <int kAdj = 0>
__device__ __forceinline__ double exp2s_fix(long long U40, const double* __restrict__ tab) {
  const long long t = U40 + (1LL << 39);
  const int m = (int)(t >> 40);  // round(U)
  const long long rq =
      (long long)(((unsigned long long)t << 24) ^ 0x8000000000000000ULL) >> 1;  // rho 2^63
  const unsigned long long ar = (unsigned long long)(rq < 0 ? -rq : rq);         // <= 2^62
  const long long t1 = (long long)(__umul64hi(ar, kExpK1Q75) >> 12);  // K1 |rho| 2^62
  const unsigned int rh = (unsigned int)(ar >> 31);                   // |rho| 2^32
  const unsigned long long r2 = ((unsigned long long)rh * rh) >> 32;  // rho^2 2^32
  const long long t2 = (long long)((r2 * kExpK2Q57) >> 27);           // K2 rho^2 2^62
  const long long d = (rq < 0 ? t1 : -t1) + t2;                       // (p - 1) 2^62
  const int n = -m;
  const long long tb = __double_as_longlong(tab[n & (kExpTabSize - 1)]);  // t_j in [1, 2)
  const long long M = (tb & 0xfffffffffffffLL) | 0x10000000000000LL;      // t_j 2^52
  const unsigned long long ad = (unsigned long long)(d < 0 ? -d : d);      // < 2^49
  const long long X = (long long)__umul64hi(ad << 2, (unsigned long long)M);  // |delta| M
  long long Mp = M + (d < 0 ? -X : X);  // p t_j 2^52, within 2^40 of [2^52, 2^53)
  int k = (n >> kExpTabBits) + kAdj;
  if (Mp >= 0x20000000000000LL) {
    Mp = (Mp + 1) >> 1;
    ++k;
  } else if (Mp < 0x10000000000000LL) {
    Mp <<= 1;
    --k;
  }
  return __longlong_as_double(((long long)(k + 1023) << 52) | (Mp & 0xfffffffffffffLL));
}

// e^a for a in [-708, 709] (callers clamp); one scaling multiply on top of exp2s.
constexpr int kExpTabOps = 1 + kExp2sOps;
__device__ __forceinline__ double exp_tab(double a, const double* __restrict__ tab) {
  return exp2s(a * kExpScale, tab);
}

// e^a for |a| < 708 with an exact reduction: kd = round(a K),
// r = a - kd ln2/4096 with ln2/4096 split in two (kd times the 29-bit head is
// exact for |kd| < 2^23), e^r from its Taylor polynomial of degree 3
// (|r| <= 8.5e-5, truncation < 3e-18 relative), times the table entry
// 2^{(kd mod 4096)/4096} and 2^{floor(kd/4096)}: the accurate exponential of
// the set-up values of the node recurrences (e^{t0}, e^{h}, e^{-2 nu h}, ...),
// whose relative errors the recurrences multiply by up to the node count.
// FP64 ops: 1 fma + 1 sub (rounding), 2 fma (reduction), 3 fma
// (polynomial), 1 mul.
__device__ __forceinline__ double exp_acc(double a, const double* __restrict__ tab) {
  const double v = fma(a, kExpScale, kRoundMagic);
  const int n = __double2loint(v);
  const double kd = v - kRoundMagic;
  double r = fma(-kd, kExpC1Hi, a);
  r = fma(-kd, kExpC1Lo, r);
  const double p = fma(fma(fma(r, 1.0 / 6.0, 0.5), r, 1.0), r, 1.0);
  const double tj = tab[n & (kExpTabSize - 1)];
  const int k = max(n >> kExpTabBits, -1022);
  return p * __hiloint2double(__double2hiint(tj) + (k << 20), __double2loint(tj));
}

// 2^{u/4096} for |u| < 2^22 with e^r from its Taylor cubic (|r| <= 8.5e-5,
// truncation < 3e-18 relative): the rounding and remainder of u on the
// integer pipe (round_rem, signs restored by integer operations), then 4 FP64
// operations.
__device__ __forceinline__ double exp2s_cubic(double u, const double* __restrict__ tab) {
  const long long ub = __double_as_longlong(u);
  int M;
  double r;
  round_rem(__longlong_as_double(ub & 0x7fffffffffffffffLL), M, r);
  const int n = (ub < 0) ? -M : M;
  const double rho =
      __longlong_as_double(__double_as_longlong(r) ^ (ub & (long long)0x8000000000000000ULL));
  const double p = fma(fma(fma(kExpC3, rho, kExpK2), rho, kExpC1), rho, 1.0);
  const double tj = tab[n & (kExpTabSize - 1)];
  const int k = max(n >> kExpTabBits, -1022);
  return p * __hiloint2double(__double2hiint(tj) + (k << 20), __double2loint(tj));
}

// 2^{u/4096} on the integer pipe.  The nearest integer n of u and the
// remainder rho = u - n (|rho| <= 1/2) are taken exactly from u's
// significand (on |u|, the signs restored by integer
// operations); p = 2^{rho/4096} in 64-bit fixed point (C1 rho from a 64 x
// 64-bit high product, the square and cube from the leading 32 bits of rho,
// their errors below 2^-58); and p t_j 2^k, t_j = 2^{j/4096}, from t_j's
// significand as in exp2s_fix (truncation below 2^-52 relative).  No
// FP64 arithmetic.  kCubic: the Taylor cubic (truncation below 3e-18
// relative; the final exponential, |u| < 4.18e6); else the minimax quadratic
// (2.6e-14; the FP64 node loops, whose node exponents satisfy |u| < 3e5)
// with these ranges: accurate for u in [-1022 * 4096, 1023 * 4096], the
// exponent clamped at -1022 below, |u| >= 2^22 giving a finite value near
// 2^{+-976}, NaN NaN.
constexpr unsigned long long kExpC1Q75 = (unsigned long long)(kExpC1 * 0x1p75);  // exact
constexpr unsigned long long kExpC3Q72 = (unsigned long long)(kExpC3 * 0x1p72 + 0.5);
static_assert(kExpC1Q75 < (1ULL << 63) && kExpC3Q72 < (1ULL << 32), "fixed-point constants");
template <bool kCubic = true>
__device__ __forceinline__ double exp2s_int(double u, const double* __restrict__ tab) {
  const long long b = __double_as_longlong(u);
  const bool neg = (int)(b >> 32) < 0;
  const int e = (int)((b >> 52) & 0x7ff) - 1023;
  const long long sig = (b & 0xfffffffffffffLL) | 0x10000000000000LL;
  const int sh = 52 - min(max(e, -2), 21);  // 31 .. 54
  const long long half = 1LL << (sh - 1);
  const long long t = sig + half;
  int m = (int)(t >> sh);                              // round(|u|)
  const long long R = (t & ((half << 1) - 1)) - half;  // (|u| - m) 2^sh
  long long rq = R << (63 - sh);                       // (|u| - m) 2^63
  if (e < -2) rq = (e >= -11) ? (sig << (e + 11)) : ((e > -74) ? (sig >> (-11 - e)) : 0LL);
  const bool negr = neg != (rq < 0);  // the sign of rho = u - n
  const unsigned long long ar = (unsigned long long)(rq < 0 ? -rq : rq);
  const long long c1 = (long long)(__umul64hi(ar, kCubic ? kExpC1Q75 : kExpK1Q75) >> 12);
  const unsigned long long rh = ar >> 31;         // |rho| 2^32
  const unsigned long long r2 = (rh * rh) >> 32;  // rho^2 2^32
  const long long c2 = (long long)((r2 * kExpK2Q57) >> 27);  // K2 rho^2 2^62
  long long c3 = 0;
  if constexpr (kCubic) c3 = (long long)((((r2 * rh) >> 32) * kExpC3Q72) >> 42);  // C3 |rho|^3
  long long d = (negr ? -(c1 + c3) : (c1 + c3)) + c2;  // (p - 1) 2^62
  const bool out = !kCubic && e > 21;  // |u| >= 2^22 (and NaN): clamp
  if (out) {
    m = 4000000;
    d = 0;
  }
  const int n = neg ? -m : m;
  const long long tb = __double_as_longlong(tab[n & (kExpTabSize - 1)]);  // t_j in [1, 2)
  const long long M = (tb & 0xfffffffffffffLL) | 0x10000000000000LL;
  const unsigned long long ad = (unsigned long long)(d < 0 ? -d : d);      // < 2^49
  const long long X = (long long)__umul64hi(ad << 2, (unsigned long long)M);
  long long Mp = M + (d < 0 ? -X : X);
  int k = kCubic ? (n >> kExpTabBits) : max(n >> kExpTabBits, -1022);
  if (Mp >= 0x20000000000000LL) {
    Mp = (Mp + 1) >> 1;
    ++k;
  } else if (Mp < 0x10000000000000LL && k > -1022) {
    Mp <<= 1;
    --k;
  }
  const double r = __longlong_as_double(((long long)(k + 1023) << 52) | (Mp & 0xfffffffffffffLL));
  if constexpr (!kCubic) {
    const bool nan = out && e == 1024 && ((((unsigned)(b >> 32)) & 0xfffffu) | (unsigned)b) != 0u;
    return nan ? u : r;
  }
  return r;
}

// e^a over the whole double range for the final normalisations: u = a K
// rounded to a double, then exp2s_cubic.  The roundings of u and of K cost
// at most 1.3e-16 |a| relative, the order of the rounding a itself carries
// from the sums that formed it: 5 FP64 operations.  |a| >= 708 goes to exp_full
// (NaN -> NaN, overflow -> inf, deep underflow -> 0).
__device__ __forceinline__ double exp_tab_full(double a, const double* __restrict__ tab) {
  if (!((__double2hiint(a) & 0x7fffffff) < 0x40862000))  // |a| < 708 (708 = 0x40862000 00000000)
    return exp_full(a);
  return exp2s_cubic(a * kExpScale, tab);
}

// e^{u / K}, K = 4096 / ln 2, for an exponent the caller formed directly in
// the table's units (u = a K with the scaling folded into its constants):
// exp2s_int for |u| < 4.18e6 (|a| < 707.4; no FP64 operation), exp_full of
// u ln2/4096 beyond (overflow, deep underflow, NaN).
__device__ __forceinline__ double exp_units_full(double u, const double* __restrict__ tab) {
  if (!((__double2hiint(u) & 0x7fffffff) < 0x414fe410))  // |u| < 4.18e6 (= 0x414fe410 00000000)
    return exp_full(u * kExpC1);
  return exp2s_int(u, tab);
}

// log a for finite a > 0 with the same table: a = 2^e m, m in [1, 2); j =
// round(4096 log2 m) from the FP32 hardware log of m's leading bits, so that
// m 2^{-j/4096} = 1 + d with |d| <= 8.5e-5; log a = (4096 e + j) ln2/4096 +
// log1p(d), log1p from its series to d^3 (truncation < 2e-17 absolute).
// FP64 ops: 1 fma (d), 3 (series), 1 fma (assembly).
__device__ __forceinline__ double log_tab(double a, const double* __restrict__ tab) {
  int hi = __double2hiint(a);
  int lo = __double2loint(a);
  int e = 0;
  if (hi < 0x00100000) {  // subnormal: scale into the normal range
    a *= 0x1p54;
    e = -54;
    hi = __double2hiint(a);
    lo = __double2loint(a);
  }
  e += (hi >> 20) - 1023;
  const int mh = hi & 0x000fffff;
  const double m = __hiloint2double(mh | 0x3ff00000, lo);  // [1, 2)
  const float mf = __int_as_float(0x3f800000 | (mh << 3) | ((unsigned)lo >> 29));
  float l2;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l2) : "f"(mf));
  const int j = __float2int_rn(l2 * (float)kExpTabSize);  // 0..4096
  // 2^{-j/4096} = 2^{(4096 - j)/4096} / 2 (j > 0), 1 (j = 0)
  const double tj = tab[(kExpTabSize - j) & (kExpTabSize - 1)];
  const double tinv =
      __hiloint2double(__double2hiint(tj) - (j > 0 ? (1 << 20) : 0), __double2loint(tj));
  const double d = fma(m, tinv, -1.0);
  const double l1p = fma(d * d, fma(d, 1.0 / 3.0, -0.5), d);
  // 4096 e + j as a double without an FP64-pipe conversion (|.| < 2^23 is
  // exact in a float); one FMA with ln2/4096 rounded (error below |log a|
  // 2^-53, the order of the result's own rounding)
  const double nd = widen_f(__int2float_rn(e * kExpTabSize + j));
  return fma(nd, kExpC1, l1p);
}

// log a for finite a > 0 split as log a = nd ln2/4096 + l1p, with nd =
// 4096 e + j an integer (exact as a double) and l1p = log1p(d), d = m
// 2^{-j/4096} - 1 (|d| <= 8.5e-5), for callers that scale the two parts
// themselves (log_tab's reduction, a = 2^e m, j = round(4096 log2 m)).  No
// FP64 arithmetic: d = M_m M_t 2^-105 - 1 from the 53-bit significands of m
// and of 2^{(4096-j)/4096} by a 64 x 64-bit high product (exact to 2^-62), the
// series d - d^2/2 + d^3/3 (truncation below 2e-17 absolute) in 64-bit fixed
// point, and l1p rounded to a double from its leading bit.  Subnormal a is
// scaled as in log_tab.  eoff: the parts of log(a 2^eoff) (nd shifted by
// 4096 eoff, exactly).
__device__ __forceinline__ double log_tab_parts(double a, const double* __restrict__ tab,
                                                double& nd, int eoff = 0) {
  int hi = __double2hiint(a);
  int lo = __double2loint(a);
  int e = 0;
  if (hi < 0x00100000) {  // subnormal: scale into the normal range
    a *= 0x1p54;
    e = -54;
    hi = __double2hiint(a);
    lo = __double2loint(a);
  }
  e += (hi >> 20) - 1023;
  const int mh = hi & 0x000fffff;
  const float mf = __int_as_float(0x3f800000 | (mh << 3) | ((unsigned)lo >> 29));
  float l2;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l2) : "f"(mf));
  const int j = __float2int_rn(l2 * (float)kExpTabSize);  // 0..4096
  nd = widen_f(__int2float_rn((e + eoff) * kExpTabSize + j));  // of a 2^eoff
  const unsigned long long Mm = ((unsigned long long)(unsigned)(mh | 0x00100000) << 32) | (unsigned)lo;
  long long dq;  // d 2^62
  if (j > 0) {
    const long long tb = __double_as_longlong(tab[(kExpTabSize - j) & (kExpTabSize - 1)]);
    const unsigned long long Mt = (unsigned long long)((tb & 0xfffffffffffffLL) | 0x10000000000000LL);
    dq = (long long)__umul64hi(Mm << 11, Mt << 10) - (1LL << 62);  // M_m M_t 2^-43 - 2^62
  } else {
    dq = (long long)(Mm << 10) - (1LL << 62);
  }
  const bool neg = dq < 0;
  const unsigned long long ad = (unsigned long long)(neg ? -dq : dq);      // < 2^49
  const unsigned long long d2 = __umul64hi(ad << 14, ad << 14) >> 26;      // d^2 2^62
  const unsigned long long d3 = __umul64hi(d2 << 20, ad << 14) >> 32;      // |d|^3 2^62
  const unsigned long long d33 = __umul64hi(d3, 0x5555555555555556ULL);    // |d|^3 / 3 2^62
  const long long q = (neg ? -(long long)(ad + d33) : (long long)(ad + d33)) - (long long)(d2 >> 1);
  // q 2^-62 as a double, rounded to nearest from its leading bit
  if (q == 0) return 0.0;
  const unsigned long long aq = (unsigned long long)(q < 0 ? -q : q);
  const int L = 63 - __clzll((long long)aq);  // <= 49
  const unsigned long long mant = (L > 52) ? ((aq + (1ULL << (L - 53))) >> (L - 52)) : (aq << (52 - L));
  const long long bits = ((long long)(L - 62 + 1023) << 52) + (long long)(mant - (1ULL << 52));
  return __longlong_as_double(q < 0 ? (bits | (long long)0x8000000000000000ULL) : bits);
}

// 1/a from the hardware approximation refined by Newton-Raphson steps
// r <- r + r (1 - a r) (each doubles the correct bits; two give full precision).
__device__ __forceinline__ double rcp_approx(double a) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(a));
  return r;
}
__device__ __forceinline__ double rcp_nr2(double a) {
  double r = rcp_approx(a);
  r = fma(r, fma(-a, r, 1.0), r);
  return fma(r, fma(-a, r, 1.0), r);
}
__device__ __forceinline__ double rcp_nr1(double a) {
  const double r = rcp_approx(a);
  return fma(r, fma(-a, r, 1.0), r);
}

// ---------------------------------------------------------------------------
// Work tally of one evaluation (kept in registers; summed per warp when the
// caller asked for counters).
struct Tally {
  unsigned nodes;       // integrand evaluations
  unsigned iters;       // window-end Newton iterations
  unsigned peak_iters;  // peak Newton iterations
  unsigned fail;        // evaluations returned as NaN
  unsigned fallback;    // learned windows replaced by the full search
  unsigned repairs;     // learned window ends moved by one Newton step
  unsigned series;      // evaluations taken by Temme's series (small x)
};

// The window of Sec. IV-B.  ts = t_max, cs = cosh ts, es = e^ts, [t0, t1] the
// integration range.  The window ends are the roots of
//   F(t) = nu (t - ts) - x (cosh t - cosh ts) + L  (+ ln 2 on the left),
// L = -log eps.  F differs from g(t) - g(ts) + L only by
// log((1 + e^{-2 nu t}) / (1 + e^{-2 nu ts})), which lies in (-ln 2, 0) right
// of the peak and in [0, ln 2] left of it, so these roots enclose the
// eps-window: the range is never narrower than the paper's.
struct Window64 {
  double ts, cs, es, t0, t1;
};

// FP32 start values for the FP64 Newton iterations (the FP32 search run to
// convergence on the same F); a value <= 0 means "none" for ts and t0.
struct Start32 {
  float ts, t0, t1, cs;  // cs: cosh ts as the FP32 search computed it
};

// FP32 helpers for Newton start values (only their side of the root matters).
__device__ __forceinline__ float log_start_f32(float v) {  // ln v, ~1e-6 relative
  float r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return 0.69314718f * r;
}

// a3: t_max = 0 when nu^2 <= x (g''(0) = nu^2 - x <= 0), else the root of
// g'(t) = nu tanh(nu t) - x sinh t, which is concave on t > 0, positive just
// right of 0 and negative at asinh(nu/x) (there nu tanh(nu t) < nu = x sinh t).
// Safeguarded Newton inside that bracket; steps from the left that leave it
// are clamped to its right end, from where Newton descends monotonically.
// Any point of the bracket is a valid shift (g(t) <= g(t_max)), so hitting
// the iteration cap is not an error.  The start is the FP32 root when the
// caller has one (then Newton stops once the step is below 1e-5 relative:
// one FP64 step), else a two-term Taylor estimate (steps below 1e-8
// relative).  Function values and steps are FP64, reciprocals by
// Newton-refined hardware approximations.  Returns ts, cosh ts and e^{ts}.
__device__ __forceinline__ void peak_f64(double x, double nu, const double* __restrict__ tab,
                                         float t_start, double& ts, double& cs, double& es,
                                         Tally& tl) {
  const double nu2 = nu * nu;
  if (!(nu2 > x)) {
    ts = 0.0;
    cs = 1.0;
    es = 1.0;
    return;
  }
  const float qf = (float)nu / (float)x;
  const float hif = log_start_f32(qf + sqrtf(fmaf(qf, qf, 1.0f)));  // asinh(nu/x)
  double hi = fma((double)hif, 2e-5, (double)hif) + 1e-6;
  double lo = 0.0;
  double t, rtol;
  if (t_start > 0.0f && (double)t_start < hi) {
    t = (double)t_start;
    rtol = 1e-5;
  } else {
    const float nu2f = (float)nu2, xf = (float)x;
    const float tc2 = (nu2f - xf) / fmaf(nu2f * nu2f, 1.0f / 3.0f, xf * (1.0f / 6.0f));
    t = ((double)tc2 < hi * hi) ? (double)sqrtf(tc2) : hi;
    rtol = 1e-8;
  }
  for (int it = 0; it < 40; ++it) {
    ++tl.peak_iters;
    const double e = exp_tab(t, tab);
    const double er = rcp_nr2(e);
    const double sh = 0.5 * (e - er), ch = 0.5 * (e + er);
    const double w = exp_tab(fmax(-2.0 * nu * t, -708.0), tab);
    const double r1 = rcp_nr2(1.0 + w);
    const double gp = fma(nu * (1.0 - w), r1, -x * sh);
    const double gpp = fma(nu2 * 4.0 * w, r1 * r1, -x * ch);
    if (gp > 0.0) lo = t; else hi = t;
    double tn;
    if (gpp < 0.0) {
      tn = fma(-gp, rcp_nr1(gpp), t);
      if (tn > hi) tn = hi;
      if (!(tn > lo)) tn = 0.5 * (lo + hi);
    } else {
      tn = 0.5 * (lo + hi);
    }
    const double dt = tn - t;
    t = tn;
    if (fabs(dt) <= rtol * t) break;
  }
  ts = t;
  es = exp_tab(t, tab);
  cs = 0.5 * (es + rcp_nr2(es));
}

// a4: window ends.  Newton on the concave F approaches t1 from the right and
// t0 from the left (after its first step, from any start), so every iterate
// past the first keeps the range at least as wide as the eps-window.  With
// FP32 roots as starts (inflated by 4e-6 towards their side) one FP64 step
// meets the 1e-5 stopping rule; otherwise the starts are FP32 bounds
// inflated by 2e-5 and the rule is 1e-8.
__device__ __forceinline__ Window64 window_f64(double x, double nu, double L,
                                               const double* __restrict__ tab, Tally& tl,
                                               const Start32* st = nullptr) {
  Window64 w;
  peak_f64(x, nu, tab, st ? st->ts : 0.0f, w.ts, w.cs, w.es, tl);
  const double ts = w.ts, cs = w.cs, es = w.es;
  // ---- t1: cosh t - cs >= ss d + cs d^2/2 for d = t - ts >= 0, so the root d
  // of L + (nu - x ss) d - x cs d^2/2 = 0 is a right bound; in the exponential
  // regime x e^t/2 >= L + x cs + nu t is one too.
  {
    double t, rtol;
    if (st != nullptr && (double)st->t1 > ts) {
      t = fma((double)st->t1, 4e-6, (double)st->t1) + 1e-6;
      rtol = 1e-5;
    } else {
      const float ssf = (float)(0.5 * (es - rcp_nr1(es)));
      const float af = (float)(x * cs), bf = (float)nu - (float)x * ssf, Lf = (float)L;
      const float df = (bf + sqrtf(fmaf(bf, bf, 2.0f * af * Lf))) / af;
      t = ts + (double)df * (1.0 + 2e-5);
      const double tb =
          (double)log_start_f32(2.0f * (Lf + af + (float)nu * (float)t) / (float)x) * (1.0 + 2e-5);
      if (tb < t) t = tb;
      rtol = 1e-8;
    }
    for (int it = 0; it < 40; ++it) {
      ++tl.iters;
      const double e = exp_tab(fmin(t, 709.0), tab);
      const double er = rcp_nr2(e);
      const double F = fma(nu, t - ts, -x * (0.5 * (e + er) - cs)) + L;
      const double Fp = fma(-0.5 * x, e - er, nu);
      const double dt = F * rcp_nr1(Fp);
      t -= dt;
      if (fabs(dt) <= rtol * t) break;
    }
    w.t1 = t;
  }
  // ---- t0: only when the peak is away from 0 and the integrand at 0 is
  // below the threshold; Newton from the left on the increasing part.
  w.t0 = 0.0;
  if (ts > 0.0) {
    const double Lp = L + kLn2;
    const double G0 = fma(-nu, ts, x * (cs - 1.0)) + Lp;
    if (G0 < 0.0) {
      double t, rtol;
      if (st != nullptr && st->t0 > 0.0f && (double)st->t0 < ts) {
        t = fmax(0.0, fma((double)st->t0, -4e-6, (double)st->t0) - 1e-6);
        rtol = 1e-5;
      } else {
        t = fmax(0.0, ts - Lp * rcp_nr1(nu));
        rtol = 1e-8;
      }
      for (int it = 0; it < 40; ++it) {
        ++tl.iters;
        const double e = exp_tab(t, tab);
        const double er = rcp_nr2(e);
        const double G = fma(nu, t - ts, -x * (0.5 * (e + er) - cs)) + Lp;
        const double Gp = fma(-0.5 * x, e - er, nu);
        double tn = fma(-G, rcp_nr1(Gp), t);
        if (tn < 0.0) tn = 0.0;
        const bool done = fabs(tn - t) <= rtol * fmax(tn, 1e-3);
        t = tn;
        if (done) break;
      }
      w.t0 = t;
    }
  }
  return w;
}

// 2 cosh H for 0 <= H <= 0.35 from its Taylor series in y = H^2 to y^7
// (truncation < 1e-20), correctly rounded to about an ulp.  The terms from
// y^5 on (below 1.6e-11) are summed in FP32 (their rounding is below 1e-18):
// 6 FP64 operations.
__device__ __forceinline__ double two_cosh_small(double H) {
  const double y = H * H;
  const float yf = f32_trunc(y);
  const float q = fmaf(fmaf(yf, 2.0f / 87178291200.0f, 2.0f / 479001600.0f), yf, 2.0f / 3628800.0f);
  double p = fma(widen_f(q), y, 2.0 / 40320.0);
  p = fma(p, y, 2.0 / 720.0);
  p = fma(p, y, 2.0 / 24.0);
  p = fma(p, y, 1.0);
  return fma(p, y, 2.0);
}

// Sum of the scaled integrand f(t)/f_s over `count` equispaced nodes
// t_j = t_start + j H, where
//   f(t) = e^{-x cosh t} cosh(nu t) = f_s exp(nu (t - ts) - x (cosh t - cs)) (1 + e^{-2 nu t}),
//   f_s = e^{nu ts - x cs} / 2.
// The exponent is kept in the scaled units of exp2s (times K = 4096/ln 2):
// its linear part A_j = K (nu (t_j - ts) + x cs) is accumulated, D_j =
// K x cosh t_j follows the three-term recurrence D_{j+1} = 2 cosh(H) D_j -
// D_{j-1} (one FMA; its rounding error grows like j ulp / (2 sinh H)), and
// e^{-2 nu t_j} is geometric: one exp2s per node.  first/last receive the
// scaled end values f_0, f_N and e0/eN the end values of exp(g(t) - g(ts))
// without the (1 + e^{-2 nu t}) factor (for the window check).
struct NodeSum {
  double S, first, last, e_first, e_last;
};
__device__ __forceinline__ NodeSum node_sum_f64(double t_start, double H, int count, double x,
                                                double nu, double ts, double cs,
                                                const double* __restrict__ tab) {
  const double xh = (0.5 * kExpScale) * x;
  double W = 1.0, c, D0, D1;
  if (bits_pos(t_start)) {
    const double e0 = exp_acc(t_start, tab), r0 = rcp_nr2(e0);
    W = exp_acc(fmax(-2.0 * nu * t_start, -708.0), tab);
    const double eh = exp_acc(H, tab), rh = rcp_nr2(eh);
    c = bits_le(H, 0.35) ? two_cosh_small(H) : eh + rh;
    D0 = xh * (e0 + r0);
    D1 = xh * fma(e0, eh, r0 * rh);
  } else {
    c = bits_le(H, 0.35) ? two_cosh_small(H) : exp_acc(H, tab) + rcp_nr2(exp_acc(H, tab));
    D0 = 2.0 * xh;
    D1 = xh * c;
  }
  const double rho = exp_acc(fmax(-2.0 * nu * H, -708.0), tab);
  double A = kExpScale * fma(nu, t_start - ts, x * cs);
  const double dA = kExpScale * (nu * H);
  NodeSum r;
  double s = 0.0, f = 0.0, ev = 0.0;
#pragma unroll 2  // two nodes' exponentials in flight per warp (measured +0.4 % over 1 and 4)
  for (int j = 0; j < count; ++j) {
    ev = exp2s_int<false>(A - D0, tab);
    f = fma(ev, W, ev);
    if (j == 0) {
      r.first = f;
      r.e_first = ev;
    }
    s += f;
    const double D2 = fma(c, D1, -D0);
    D0 = D1;
    D1 = D2;
    A += dA;
    W *= rho;
  }
  r.S = s;
  r.last = f;
  r.e_last = ev;
  return r;
}
// FP64 ops per node in node_sum_f64 (work accounting): 1 sub (exponent),
// 1 fma + 1 add (f, s), 1 fma (recurrence), 1 add + 1 mul; the exponential
// (exp2s_int) on the integer pipe.
constexpr int kNodeOps64 = 6;

// 2 cosh v for 0 <= v <= 0.75 from its Taylor series in y = v^2 to y^9
// (truncation < 2e-18); the terms from y^6 on (below 1.3e-10) in FP32: 7 FP64
// operations.
__device__ __forceinline__ double two_cosh_mid(double v) {
  const double y = v * v;
  const float yf = f32_trunc(y);
  float q = fmaf(yf, 2.0f / 6402373705728000.0f, 2.0f / 20922789888000.0f);
  q = fmaf(q, yf, 2.0f / 87178291200.0f);
  q = fmaf(q, yf, 2.0f / 479001600.0f);
  double p = fma(widen_f(q), y, 2.0 / 3628800.0);
  p = fma(p, y, 2.0 / 40320.0);
  p = fma(p, y, 2.0 / 720.0);
  p = fma(p, y, 2.0 / 24.0);
  p = fma(p, y, 1.0);
  return fma(p, y, 2.0);
}

// 2 cosh v for v >= 0: two_cosh_small up to 0.35 (6 FP64 ops), two_cosh_mid
// up to 0.75 (7), e^v + e^{-v} above (13).  The tier is chosen once for the
// active lanes of the warp (a vote): lanes of a warp mostly agree, and a
// per-lane select would evaluate several tiers.
__device__ __forceinline__ double two_cosh_warp(double v, const double* __restrict__ tab) {
  const bool small = bits_le(v, 0.35), mid = bits_le(v, 0.75);
  const unsigned act = __activemask();
  if (__all_sync(act, small)) return two_cosh_small(v);
  if (__all_sync(act, mid)) return two_cosh_mid(v);
  const double e = exp_acc(v, tab), big = e + rcp_nr2(e);
  if (!__any_sync(act, mid)) return big;
  return mid ? two_cosh_mid(v) : big;
}

// 2 cosh(h) for the quantised steps h = 2^e (1 + k/256), e = -12..0,
// k = 0..255 (index (e + 12) 256 + k), correctly rounded (gen_cosh_table.py).
constexpr int kCoshTabSize = 3328;
static __device__ const double kCoshTab[kCoshTabSize] = {
#include "bk_cosh_table.inc"
};

// The step h rounded up to 8 significand bits (hq >= h: N hq still covers the
// window, and the strip bound's error grows by at most e^{2 pi a/h 2^-8},
// a factor 1.13 at tol = 1e-13) and its index in kCoshTab, or -1 when hq is
// outside [2^-12, 2).
__device__ __forceinline__ float quantise_step(float h, int& idx) {
  const int up = (__float_as_int(h) + 0x7fff) & ~0x7fff;
  const int i = (up >> 15) - ((127 - 12) << 8);
  idx = (h > 0.0f && i >= 0 && i < 3328) ? i : -1;
  return __int_as_float(up);
}

// e^{-2 nu h} for a step h and nu >= 0, by the accurate set-up exponential:
// the ratio of the node loop's geometric factor e^{-2 nu t_j}.
__device__ __forceinline__ double decay_step(double nu, double h, const double* __restrict__ tab) {
  return exp_acc(fmax(-2.0 * nu * h, -708.0), tab);
}

// decay_step for the steps of kCoshTab (h_k = 2^e (1 + j/256), k = (e + 12)
// 256 + j), as node_sum_cosh would compute it: the per-launch table of the
// Matern tile writers, whose nu is fixed.
__device__ __forceinline__ double decay_entry(double nu, int k, const double* __restrict__ tab) {
  const double h = __hiloint2double(((k >> 8) - 12 + 1023) << 20 | ((k & 255) << 12), 0);
  return decay_step(nu, h, tab);
}

// log2 v of a positive finite double to about 1e-6, on the integer, FP32 and
// MUFU pipes: the exponent field plus lg2 of the leading 23 significand bits.
__device__ __forceinline__ float log2_f64_approx(double v) {
  const int hi = __double2hiint(v);
  const float m = __int_as_float(0x3f800000 | ((hi & 0x000fffff) << 3) |
                                 (int)((unsigned)__double2loint(v) >> 29));
  float lm;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(lm) : "f"(m));
  // the unbiased exponent as a float, exactly, by the magic-number trick
  const float e = __int_as_float(0x4b400000 + ((hi >> 20) & 0x7ff)) - 12583935.0f;
  return e + lm;
}

// The same sum without centring, for the checked windows of scale_f64:
//   f(t_j) = (e^{nu t_start} / 2) e^{-x cosh t_j} C_j,
//   C_j = 2 e^{-nu t_start} cosh(nu t_j) = e^{nu (t_j - t_start)} (1 + W_j),
//   W_j = e^{-2 nu t_j} = e^{-2 nu t_start} r^j, r = e^{-2 nu H}.
// D_j = K x cosh t_j follows the three-term recurrence D_{j+1} = 2 cosh(H)
// D_j - D_{j-1} (one FP64 FMA); the factor e^{nu (t_j - t_start)} joins the
// exponent as G_j = j K nu H, a running sum in 64-bit fixed point (units of
// 2^-40, exact steps: no rounding growth), so that node j's term is
// 2^{-(D_j - G_j)/4096} (1 + W_j) with the exponential from D_j - G_j on the
// integer pipe (exp2s_fix) and W_j a geometric sequence in fixed point (units
// of 2^-63, one 64 x 64-bit high product per node, its truncation below 2^-63
// a step), 1 + W_j rounded to a double by integer operations.  A node costs
// the D recurrence and the summing FMA: 2 FP64 operations, and the set-up
// needs neither cosh t* nor the centring exponentials.  Each factor must stay
// in the double range, x cosh t_j <= 690 (D_j below 2^22) and nu (t_j -
// t_start) <= 600 (G_j below 2^22, the terms below 2^880); cosh_loop_ok
// states the conditions.  Returns S = sum_j e^{-x cosh t_j} C_j and the end
// terms.
struct NodeSumC {
  double S;                   // the trapezoid sum, end weights 1/2 included
  float l2_first, l2_last;    // log2 of the unweighted end terms (window check)
  bool pos;                   // the last term is positive
};
// step_idx: the step's index in kCoshTab (or -1); wnu: a table of
// decay_step(nu, h) on the same steps for this nu (or null).  The weights 1/2
// of the end nodes are folded into their terms (at t_start = 0, (1 + W_0)/2 =
// 1), and the end terms' logs for the window check come from the factors on
// the FP32/integer pipes, so the ends cost no extra FP64 products.
constexpr double kExpScale40 = kExpScale * 0x1p40;  // K in units of 2^-40 (exact scaling)
__device__ __forceinline__ NodeSumC node_sum_cosh(double t_start, double H, int count, double xh,
                                                  double nu, const double* __restrict__ tab,
                                                  int step_idx, const double* __restrict__ wnu) {
  const bool start_pos = bits_pos(t_start);
  double c, D0, D1, C0h = 1.0;
  unsigned long long Wq = 1ULL << 63;  // W_0 2^63 (W_0 = 1 at t_start = 0)
  if (start_pos) {
    const double e0 = exp_acc(t_start, tab), r0 = rcp_nr2(e0);
    const double eh = exp_acc(H, tab), rh = rcp_nr2(eh);
    c = bits_le(H, 0.35) ? two_cosh_small(H) : eh + rh;
    D0 = xh * (e0 + r0);
    D1 = xh * fma(e0, eh, r0 * rh);
    const double W = exp_acc(fmax(-2.0 * nu * t_start, -708.0), tab);
    C0h = fma(W, 0.5, 0.5);
    Wq = fix63_unit(W);
  } else {
    c = (step_idx >= 0) ? kCoshTab[step_idx] : two_cosh_warp(H, tab);
    // D0 = 2 xh by its exponent (xh is normal: the callers' x lies in the
    // FP32 search's range and x cosh t1 <= 690)
    D0 = __hiloint2double(__double2hiint(xh) + (1 << 20), __double2loint(xh));
    D1 = xh * c;
  }
  const unsigned long long Rq =  // r 2^64
      fix64_unit((step_idx >= 0 && wnu != nullptr) ? wnu[step_idx] : decay_step(nu, H, tab));
  const long long Gs = __double2ll_rn(nu * H * kExpScale40);  // K nu H 2^40
  long long G = 0;                                            // G_j 2^40
  NodeSumC r;
  // the first term times 1/2: D_0 with G_0 = 0, (1 + W_0)/2 = C0h
  double s = exp2s_fix<0>(fix40_node(D0), tab);
  r.l2_first = 0.0f;
  if (start_pos) {
    r.l2_first = log2_f64_approx(s) + log2_f64_approx(C0h) + 1.0f;
    s *= C0h;
  }
#pragma unroll 2
  for (int j = 1; j < count - 1; ++j) {
    const double D2 = fma(c, D1, -D0);
    D0 = D1;
    D1 = D2;
    G += Gs;
    Wq = __umul64hi(Wq, Rq);
    s = fma(exp2s_fix<0>(fix40_node(D0) - G, tab), one_plus_w(Wq), s);
  }
  {  // the last node (D_N after the loop), weight 1/2 folded into E; count >= 3
    G += Gs;
    Wq = __umul64hi(Wq, Rq);
    const double Eh = exp2s_fix<-1>(fix40_node(D1) - G, tab);
    const double w = one_plus_w(Wq);
    s = fma(Eh, w, s);
    r.l2_last = log2_f64_approx(Eh) + log2_f64_approx(w) + 1.0f;
    r.pos = bits_pos(Eh);
  }
  r.S = s;
  return r;
}
// FP64 ops per node of node_sum_cosh: 1 fma (sum), 1 fma (the D recurrence);
// the exponential, G and W run on the integer pipe.
constexpr int kNodeOps64Cosh = 2;

// Whether node_sum_cosh may take a window [t0, t1] of N intervals (FP32
// tests on truncated copies).  Rounding in the D recurrence reaches node j
// amplified by about j / (2 sinh h) relative to D_j; the test bounds N^2 by
// 2^16 max(nu (t1 - t0), 1) (every window of up to 256 intervals passes).
// Range: x cosh t1 <= 690 (cosh t <= (e^t + 1)/2)
// and nu (t1 - t0) <= 600.  NaN fails.
__device__ __forceinline__ bool cosh_loop_ok(float x, float nu, float t0, float t1, int N) {
  const float nw = nu * (t1 - t0), nf = (float)N;
  constexpr float kLog2ef_ = 1.44269504f;
  float e1;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e1) : "f"(t1 * kLog2ef_));
  return nf * nf <= 65536.0f * fmaxf(nw, 1.0f) && nw <= 600.0f && x * (e1 + 1.0f) <= 1380.0f;
}


// ln(2 / tol) for the plain form: tol = 1e-13 keeps the quadrature error
// about three orders below the 1e-10 relative accuracy the form promises.
constexpr float kPlainLog2OverTol = 30.6267f;
constexpr int kPlainMaxNodes = 1024;

// ---------------------------------------------------------------------------
// a5: node count.  For f analytic in the strip |Im t| < a with
// int |f(t + i s)| dt <= M(a) I for |s| < a, the trapezoid rule with step h
// on the whole line errs by at most 2 M(a) I / (e^{2 pi a / h} - 1)
// (Trefethen & Weideman, SIAM Review 56 (2014), Thm 5.1).  Here
// |f(t + i a)| <= e^{-x cos(a) cosh t} cosh(nu t), so M(a) <= K_nu(x cos a) /
// K_nu(x), estimated by (cos a)^{-nu} e^{x (1 - cos a)} (the small- and
// large-x behaviour of K_nu).  The step is the largest h over 16 strip
// widths a_k = (k + 1/2) pi/32 with 2 pi a_k / h >= ln(2/tol) + nu lam_k + x mu_k,
// lam_k = -ln cos a_k, mu_k = 1 - cos a_k, and N = ceil((t1 - t0)/h).
// The arithmetic is FP32: N only needs a few correct digits.
static __constant__ float kStripA[16] = {
    4.908738521e-02f, 1.472621556e-01f, 2.454369261e-01f, 3.436116965e-01f,
    4.417864669e-01f, 5.399612373e-01f, 6.381360078e-01f, 7.363107782e-01f,
    8.344855486e-01f, 9.326603190e-01f, 1.030835089e+00f, 1.129009860e+00f,
    1.227184630e+00f, 1.325359401e+00f, 1.423534171e+00f, 1.521708942e+00f};
static __constant__ float kStripLam[16] = {
    1.205269841e-03f, 1.088249011e-02f, 3.042698822e-02f, 6.023412881e-02f,
    1.009377626e-01f, 1.534675349e-01f, 2.191421532e-01f, 2.998206135e-01f,
    3.981534711e-01f, 5.180192619e-01f, 6.653321421e-01f, 8.496721254e-01f,
    1.087999247e+00f, 1.414775403e+00f, 1.919157882e+00f, 3.014554825e+00f};
static __constant__ float kStripMu[16] = {
    1.204543795e-03f, 1.082349004e-02f, 2.996874681e-02f, 5.845593482e-02f,
    9.601070688e-02f, 1.422713900e-01f, 1.967924685e-01f, 2.590488746e-01f,
    3.284410452e-01f, 4.043006955e-01f, 4.858972558e-01f, 5.724449066e-01f,
    6.631101466e-01f, 7.570198201e-01f, 8.532695255e-01f, 9.509323257e-01f};

// Returns N in [2, n_max], or n_max + 1 when the bound asks for more nodes.
// a / (ln(2/tol) + nu lam(a) + x mu(a)) is quasi-concave in a (a linear
// numerator over a positive convex denominator), so its samples rise to one
// maximum and then fall: the scan starts at the widest strip, where the
// maximum lies for most points (the last or second-to-last sample on the
// Matern workloads), and stops at the first decrease.  Every a gives a valid
// bound, so a stop at a rounding-level wiggle can only cost a node, not
// accuracy.  The index is the same for all lanes still scanning, so the
// constant-memory reads stay uniform.
__device__ __forceinline__ int strip_node_count(float x, float nu, float width, float log2_over_tol,
                                                int n_max) {
  float bn = kStripA[15];
  float bd = fmaf(nu, kStripLam[15], fmaf(x, kStripMu[15], log2_over_tol));
  for (int k = 14; k >= 0; --k) {
    const float d = fmaf(nu, kStripLam[k], fmaf(x, kStripMu[k], log2_over_tol));
    if (!(kStripA[k] * bd > bn * d)) break;
    bn = kStripA[k];
    bd = d;
  }
  // the step and ceil(width / h) need only a few digits (every strip width
  // gives a valid bound): MUFU reciprocals instead of IEEE divisions
  float rb, rh;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rb) : "f"(bd));
  const float h = 6.28318531f * bn * rb;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rh) : "f"(h));
  const float nf = ceilf(width * rh);
  if (!(nf <= (float)n_max)) return n_max + 1;
  return nf < 2.0f ? 2 : (int)nf;
}

// The plain form's window from FP32 roots of the same F (st): t* as found,
// 0 where the FP32 test found nu^2 <= x (any point is a valid shift: g(t) -
// g(t*) is what the nodes evaluate, in FP64), the ends widened by 2e-5
// relative and 1e-5 absolute towards their side, far beyond the FP32 error
// of the roots; cosh t* and e^{t*} in FP64.
// The ends are then checked on the computed end nodes (scale3_f64; scale_f64
// widens its ends the same way).
__device__ __forceinline__ Window64 window_from_start(double x, double nu, const Start32& st,
                                                      const double* __restrict__ tab) {
  Window64 w;
  w.ts = widen_f(st.ts);  // 0 when the FP32 search found nu^2 <= x
  if (st.ts > 0.0f) {
    w.es = exp_tab(w.ts, tab);
    w.cs = 0.5 * (w.es + rcp_nr2(w.es));
  } else {
    w.es = 1.0;
    w.cs = 1.0;
  }
  const double t1 = widen_f(st.t1), t0 = widen_f(st.t0);
  w.t1 = fma(t1, 2e-5, t1) + 1e-5;
  w.t0 = (st.t0 > 0.0f && st.ts > 0.0f) ? fmax(0.0, fma(t0, -2e-5, t0) - 1e-5) : 0.0;
  return w;
}

// a6/a7: trapezoid on [t0, t1] with N intervals from the strip bound, in the
// log domain: K = e^{scale} h S with scale = nu ts - x cs - ln 2 and S the
// weighted sum of the scaled integrand (node_sum_f64).
struct Scaled64 {
  double scale, hS;
  unsigned nodes, iters, peak_iters, fail;
};

// The FP64 search window (window_f64 from its own start bounds) and its
// quadrature.  Kept out of line: it is the rare path of the plain form
// (check failures, points outside the FP32 search region, or every point
// under bk_opts.search_f64), and inlining it would cost the common path
// registers.  Returns NaN (and fail = 1) when N would exceed n_max.
static __device__ __noinline__ Scaled64 scaled_search_f64(double x, double nu, float log2_over_tol,
                                                   int n_max, const double* __restrict__ tab) {
  Tally tl{0u, 0u, 0u, 0u, 0u, 0u, 0u};
  Scaled64 r;
  const Window64 w = window_f64(x, nu, kLogInvEps64, tab, tl);
  const double width = w.t1 - w.t0;
  const int N = strip_node_count((float)x, (float)nu, (float)width, log2_over_tol, n_max);
  if (N > n_max) {
    r.scale = r.hS = __longlong_as_double(0x7ff8000000000000LL);
    r.nodes = 0;
    r.fail = 1;
  } else {
    const double h = width * rcp_nr2((double)N);
    const NodeSum ns = node_sum_f64(w.t0, h, N + 1, x, nu, w.ts, w.cs, tab);
    r.hS = h * (ns.S - 0.5 * (ns.first + ns.last));
    r.scale = fma(nu, w.ts, -x * w.cs) - kLn2;
    r.nodes = N + 1;
    r.fail = 0;
  }
  r.iters = tl.iters;
  r.peak_iters = tl.peak_iters;
  return r;
}

__device__ __forceinline__ double take_search(const Scaled64& r, double& hS, Tally& tl) {
  tl.nodes += r.nodes;
  tl.iters += r.iters;
  tl.peak_iters += r.peak_iters;
  tl.fail += r.fail;
  hS = r.hS;
  return r.scale;
}

// The plain form's K_nu in scaled form for x = xh 2/K (xh = x 2048/ln 2,
// the node loop's half-scaled argument, which the callers form directly):
// returns the scale and sets hS (K = e^{scale} hS; on the checked windows hS
// holds the step halved, and the scale is 0 for windows that start at
// t = 0).  With FP32 start values (st) the window is taken from
// them (the ends widened as in window_from_start) and checked on the
// computed end nodes against the rule of window_f64, whose F bounds these
// from above: e(t1) <= eps and, for t0 > 0, 2 e(t0) <= eps, where e(t) =
// exp(g(t) - g(t*)) with g(t) = nu t - x cosh t, and a finite positive sum.
// A window that fails is replaced by the FP64 search (tl.fallback); without
// st, the FP64 search.
//  - node_sum_cosh where cosh_loop_ok: scale nu t0 - ln 2.  The check takes
//    log2 e(t) = log2 f_t - log2(1 + e^{-2 nu t}) - (nu (t* - t0) - x cosh t*)
//    log2 e with log2 f_t from the end term's FP64 factors (to ~5e-7) and
//    FP32 values of the rest (cosh t* as the FP32 search computed it):
//    error below about 3e-4 in log2 e, i.e. the thresholds hold to a factor
//    2^{3e-4}.
//  - node_sum_f64 elsewhere (centred at t*, cosh t* in FP64): scale
//    nu t* - x cosh t* - ln 2, the check on its FP64 end values.
constexpr double kTwoOverK = 2.0 / kExpScale;  // x = xh 2/K (ln2 / 2048)
__device__ __forceinline__ double scale_f64(double xh, double nu, float log2_over_tol, int n_max,
                                            const double* __restrict__ tab, double& hS,
                                            Tally& tl, const Start32* st = nullptr,
                                            const double* __restrict__ wnu = nullptr) {
  constexpr double kEps64 = 0x1p-52;
  if (st == nullptr)
    return take_search(scaled_search_f64(xh * kTwoOverK, nu, log2_over_tol, n_max, tab), hS, tl);
  // The window's geometry in FP32, taken exactly to FP64: the ends widened by
  // 2e-5 relative and 1e-5 absolute (as window_from_start), h = (t1 - t0)/N
  // rounded up to 8 significand bits (quantise_step, so that 2 cosh h comes
  // from kCoshTab).  The trapezoid rule of step h over [t0, t0 + N h] needs
  // nothing more of h: its last node lies at most 0.4 % beyond t1, and the
  // check reads the computed end terms.
  const float t1f = fmaf(st->t1, 2e-5f, st->t1) + 1e-5f;
  const float t0f = (st->t0 > 0.0f && st->ts > 0.0f) ? fmaxf(0.0f, fmaf(st->t0, -2e-5f, st->t0) - 1e-5f)
                                                     : 0.0f;
  const float xf = f32_trunc(xh) * (float)kTwoOverK, nuf = f32_trunc(nu), wf = t1f - t0f;
  const int N = strip_node_count(xf, nuf, wf, log2_over_tol, n_max);
  if (N <= n_max) {
    int step_idx;
    const float hq = quantise_step(__fdividef(wf, (float)N), step_idx);
    const float tnf = fmaf((float)N, hq, t0f);  // the last node
    const double t0 = widen_f(t0f), h = widen_f(hq);
    tl.nodes += N + 1;
    if (cosh_loop_ok(xf, nuf, t0f, tnf, N)) {
      const NodeSumC ns = node_sum_cosh(t0, h, N + 1, xh, nu, tab, step_idx, wnu);
      constexpr float kL2e = 1.44269504f;
      const float G = fmaf(nuf, st->ts - t0f, -xf * st->cs) * kL2e;  // log2 of the peak term
      float w1;
      asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(w1) : "f"(-2.0f * kL2e * nuf * tnf));
      float lw1;
      asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(lw1) : "f"(1.0f + w1));
      bool ok = ns.pos && ns.l2_last - lw1 - G <= -52.0f && bits_pos(ns.S) &&
                bits_le(ns.S, 1e300);
      if (bits_pos(t0)) {
        float w0, lw0;
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(w0) : "f"(-2.0f * kL2e * nuf * t0f));
        asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(lw0) : "f"(1.0f + w0));
        ok = ok && ns.l2_first - lw0 - G <= -53.0f;
      }
      if (ok) {
        // the 1/2 of the sum's scale e^{nu t0}/2 goes into the step (exact
        // in FP32), so that the common window (t0 = 0) returns scale 0
        hS = widen_f(0.5f * hq) * ns.S;
        return bits_pos(t0) ? nu * t0 : 0.0;
      }
    } else {
      const double x = xh * kTwoOverK;
      Window64 w;
      w.ts = widen_f(st->ts);  // 0 when the FP32 search found nu^2 <= x
      if (st->ts > 0.0f) {
        w.es = exp_tab(w.ts, tab);
        w.cs = 0.5 * (w.es + rcp_nr2(w.es));
      } else {
        w.es = 1.0;
        w.cs = 1.0;
      }
      const NodeSum ns = node_sum_f64(t0, h, N + 1, x, nu, w.ts, w.cs, tab);
      // e_last <= eps, (t0 == 0 or 2 e_first <= eps), 0 < S < 1e300, as integer tests
      if (bits_le(ns.e_last, kEps64) && (!bits_pos(t0) || bits_le(ns.e_first, 0.5 * kEps64)) &&
          bits_pos(ns.S) && bits_le(ns.S, 1e300)) {
        hS = widen_f(0.5f * hq) * (ns.S - 0.5 * (ns.first + ns.last));
        return fma(nu, w.ts, -x * w.cs);
      }
    }
  }
  ++tl.fallback;
  return take_search(scaled_search_f64(xh * kTwoOverK, nu, log2_over_tol, n_max, tab), hS, tl);
}

// ---------------------------------------------------------------------------
// Derivatives of K_nu(x) on the same nodes (not in the paper; for
// gradient-based MLE).  Differentiating the integral under the sign,
//   -dK/dx  = int cosh(t) f(t) dt,   dK/dnu = int t sinh(nu t) e^{-x cosh t} dt,
// and with the scaled integrand of node_sum_f64,
//   cosh(t) f/f_s = (D_j / (K x)) f_j / f_s,   t sinh(nu t) e^{-x cosh t} / f_s
//   = t_j e^{a_j} (1 - e^{-2 nu t_j}),
// so the node loop carries two more sums (4 more FP64 operations per node).
// The window must hold the integrand of -dK/dx, which decays like that of
// K_{nu+1}: it is the union of the windows of orders nu and nu + 1.
struct NodeSum3 {
  double S, Sx, Sn;                 // sums for K, -dK/dx (times K x), dK/dnu
  double f0, fN, fx0, fxN, fn0, fnN;  // end terms of each sum
  double e_first, e_last;
};
__device__ __forceinline__ NodeSum3 node_sum3_f64(double t_start, double H, int count, double x,
                                                  double nu, double ts, double cs,
                                                  const double* __restrict__ tab) {
  const double xh = (0.5 * kExpScale) * x;
  double W = 1.0, c, D0, D1;
  if (bits_pos(t_start)) {
    const double e0 = exp_acc(t_start, tab), r0 = rcp_nr2(e0);
    W = exp_acc(fmax(-2.0 * nu * t_start, -708.0), tab);
    const double eh = exp_acc(H, tab), rh = rcp_nr2(eh);
    c = bits_le(H, 0.35) ? two_cosh_small(H) : eh + rh;
    D0 = xh * (e0 + r0);
    D1 = xh * fma(e0, eh, r0 * rh);
  } else {
    c = bits_le(H, 0.35) ? two_cosh_small(H) : exp_acc(H, tab) + rcp_nr2(exp_acc(H, tab));
    D0 = 2.0 * xh;
    D1 = xh * c;
  }
  const double rho = exp_acc(fmax(-2.0 * nu * H, -708.0), tab);
  double A = kExpScale * fma(nu, t_start - ts, x * cs);
  const double dA = kExpScale * (nu * H);
  NodeSum3 r;
  double s = 0.0, sx = 0.0, sn = 0.0, t = t_start, ev = 0.0, f = 0.0, fx = 0.0, fn = 0.0;
  for (int j = 0; j < count; ++j) {
    ev = exp2s_int<false>(A - D0, tab);
    f = fma(ev, W, ev);
    fx = D0 * f;
    fn = fma(-ev, W, ev) * t;
    if (j == 0) {
      r.f0 = f;
      r.fx0 = fx;
      r.fn0 = fn;
      r.e_first = ev;
    }
    s += f;
    sx += fx;
    sn += fn;
    const double D2 = fma(c, D1, -D0);
    D0 = D1;
    D1 = D2;
    A += dA;
    W *= rho;
    t += H;
  }
  r.S = s;
  r.Sx = sx;
  r.Sn = sn;
  r.fN = f;
  r.fxN = fx;
  r.fnN = fn;
  r.e_last = ev;
  return r;
}

// K, -dK/dx and dK/dnu in scaled form: returns the scale sc and sets
// hS = h S, hSx = h Sx / (K x) and hSn = h Sn, so that K = e^sc hS,
// dK/dx = -e^sc hSx, dK/dnu = e^sc hSn.  st / st1: FP32 roots for the orders
// nu and nu + 1 (both or neither); the window is their union, checked in FP64
// on K's end nodes as in scale_f64; without roots, or when the check fails,
// the union of the FP64 search windows.
__device__ __forceinline__ double scale3_f64(double x, double nu, const double* __restrict__ tab,
                                             const Start32* st, const Start32* st1,
                                             double& hS, double& hSx, double& hSn, Tally& tl) {
  constexpr double kEps64 = 0x1p-52;
  Window64 w;
  bool check = (st != nullptr && st1 != nullptr);
  if (check) {
    w = window_from_start(x, nu, *st, tab);
    const Window64 w1 = window_from_start(x, nu + 1.0, *st1, tab);
    w.t0 = fmin(w.t0, w1.t0);
    w.t1 = fmax(w.t1, w1.t1);
  }
  for (int attempt = 0; attempt < 2; ++attempt) {
    if (!check) {
      w = window_f64(x, nu, kLogInvEps64, tab, tl);
      const Window64 w1 = window_f64(x, nu + 1.0, kLogInvEps64, tab, tl);
      w.t0 = fmin(w.t0, w1.t0);
      w.t1 = fmax(w.t1, w1.t1);
    }
    const double width = w.t1 - w.t0;
    const int N = strip_node_count((float)x, (float)(nu + 1.0), (float)width, kPlainLog2OverTol,
                                   kPlainMaxNodes);
    if (N > kPlainMaxNodes) {
      if (check) {
        ++tl.fallback;
        check = false;
        continue;
      }
      ++tl.fail;
      hS = hSx = hSn = __longlong_as_double(0x7ff8000000000000LL);
      return hS;
    }
    const double h = width * rcp_nr2((double)N);
    const NodeSum3 ns = node_sum3_f64(w.t0, h, N + 1, x, nu, w.ts, w.cs, tab);
    tl.nodes += N + 1;
    if (check && !(ns.e_last <= kEps64 && (w.t0 == 0.0 || 2.0 * ns.e_first <= kEps64) &&
                   ns.S > 0.0 && ns.S < 1e300)) {
      ++tl.fallback;
      check = false;
      continue;
    }
    hS = h * (ns.S - 0.5 * (ns.f0 + ns.fN));
    hSx = h * (ns.Sx - 0.5 * (ns.fx0 + ns.fxN)) * rcp_nr2(kExpScale * x);
    hSn = h * (ns.Sn - 0.5 * (ns.fn0 + ns.fnN));
    break;
  }
  return fma(nu, w.ts, -x * w.cs) - kLn2;
}

// The paper's fixed window (Algorithm 2, x >= 0.1 branch, Sec. IV-C): the
// trapezoid on [0, t1] with b bins, h = t1/b, weights 1/2 at both ends,
// shifted by the largest node value (t_lmax).  The shift is taken at the
// node with the largest nu t - x cosh t (g without its log(1 + e^{-2 nu t})
// term: any shift is exact, this one keeps every scaled node <= 2).  Pass 1
// finds it, pass 2 sums exp2s of the scaled exponents (clamped below at
// e^-1000, far under the double range) times (1 + e^{-2 nu t}); cosh t_m by
// the three-term recurrence, all in the scaled units of node_sum_f64.
// Returns the scale (the shift minus ln 2) and sets h S.
__device__ __forceinline__ double fixed_scale_f64(double x, double nu, double t1, int bins,
                                                  const double* __restrict__ tab, double& hS,
                                                  Tally& tl) {
  const double h = t1 * rcp_nr2((double)bins);
  double c;
  if (h <= 0.35) {
    c = two_cosh_small(h);
  } else {
    const double eh = exp_acc(h, tab);
    c = eh + rcp_nr2(eh);
  }
  const double D0i = kExpScale * x, D1i = 0.5 * c * D0i, dA = kExpScale * (nu * h);
  double D0 = D0i, D1 = D1i, A = 0.0, amax = -1e300;
  for (int m = 0; m <= bins; ++m) {
    amax = fmax(amax, A - D0);
    const double D2 = fma(c, D1, -D0);
    D0 = D1;
    D1 = D2;
    A += dA;
  }
  const double rho = exp_acc(fmax(-2.0 * nu * h, -708.0), tab);
  D0 = D0i;
  D1 = D1i;
  A = -amax;
  double W = 1.0, s = 0.0, f = 0.0, first = 0.0;
  for (int m = 0; m <= bins; ++m) {
    const double ev = exp2s(fmax(A - D0, -1000.0 * kExpScale), tab);
    f = fma(ev, W, ev);
    if (m == 0) first = f;
    s += f;
    const double D2 = fma(c, D1, -D0);
    D0 = D1;
    D1 = D2;
    A += dA;
    W *= rho;
  }
  tl.nodes += 2 * (bins + 1);
  hS = h * (s - 0.5 * (first + f));
  return amax * kExpC1 - kLn2;
}


}  // namespace bk
