// Oracle for the K_nu / Matern hot path.
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes
// or calls this file; only tests, the smoke check and the CPU-baseline leg of
// the benchmark load it.  It shares no code, header, constant or helper with
// the CUDA path.
//
// Everything is plain, slow and written to be checked against the paper by
// eye, in `long double` (x87 80-bit on x86-64, IEEE binary128 on aarch64).
//
//  * oracle_log_besselk: K_nu(x) by its definition, the integral of Eq.
//    (integral) (Sec. IV-B), evaluated by a dense composite trapezoid rule on
//    [0, T] with step halving until two successive halvings agree.  The
//    integrand is even and entire in t, so the rule converges very fast; the
//    window is found by plain stepping, not by root finding.
//  * oracle_besselk_temme: the independent series route of Sec. IV-A
//    (Eq. (temme_main), the p/q/f recurrences, the start values Eqs.
//    (temme_initpq)/(temme_initf) and Campbell's forward recurrence Eq.
//    (recurrence)).  Used only as a cross-check of the integral for small x.
//  * oracle_window: the epsilon-window of Sec. IV-B, [t0, t1] = {t : g(t) >=
//    log(eps) + g(t_max)}, found by bracketing (FINDRANGE-style doubling) and
//    pure bisection.  Produces labels for the learned window.
//  * oracle_min_nodes: the smallest trapezoid interval count N on that window
//    whose result lies within a relative tolerance of oracle_log_besselk.
//  * oracle_matern_*: the Matern entry of Sec. III-A, with sigma^2 on r == 0
//    as in Algorithm 3.
//  * oracle_fixed_window_log_k: the paper's refined integration branch
//    (Algorithm 2, else-branch): fixed [0, t1], b bins, shift by the largest
//    node value, trapezoid weights multiplying the exponential.
//  * oracle_besselk_grad_batch: dK/dx and dK/dnu by differentiating the
//    integral under the sign (not in the paper; for gradient-based MLE).
//
// Pins (tests/test_oracle_pins.py): closed forms for nu = 1/2, 3/2, 5/2,
// recurrence Eq. (recurrence), the Wronskian with a library I_nu, small- and
// large-x limits, scipy's kv, the Temme series against the integral, and the
// window's defining property checked on a dense grid.

#include <cmath>
#include <cfloat>
#include <cstdint>
#include <cstring>
#include <cstdlib>
#ifdef _OPENMP
#include <omp.h>
#endif

#include <limits>

typedef long double ld;

static const ld kLn2 = 0.693147180559945309417232121458176568075500134L;
static const ld kPi = 3.141592653589793238462643383279502884197169399L;
static const ld kEulerGamma = 0.577215664901532860606512090082402431042159336L;

// ---------------------------------------------------------------------------
// Eq. (logintegrand): g(t) = log cosh(nu t) - x cosh t.
// log cosh(y) is written as |y| + log(1 + e^{-2|y|}) - log 2 so that it does
// not overflow for large |nu t|.
// Written once for a real type R (long double for the oracle proper; double
// for the FP64 instance used on large samples), with std:: functions, whose
// long double overloads are expl, log1pl, coshl, ...
template <typename R>
static R log_cosh_t(R y) {
  y = std::fabs(y);
  return y + std::log1p(std::exp(R(-2) * y)) - R(kLn2);
}

template <typename R>
static R g_of_t(R t, R x, R nu) { return log_cosh_t<R>(nu * t) - x * std::cosh(t); }

static ld log_cosh(ld y) { return log_cosh_t<ld>(y); }
static ld g_of(ld t, ld x, ld nu) { return g_of_t<ld>(t, x, nu); }

// g'(t) = nu tanh(nu t) - x sinh t.
static ld gprime_of(ld t, ld x, ld nu) { return nu * tanhl(nu * t) - x * sinhl(t); }

// ---------------------------------------------------------------------------
// K_nu(x) by the dense trapezoid rule.  Returns log K; *status = 0 on success,
// 1 if the window search or the halving loop did not finish.  R is the real
// type of every step (long double: the oracle proper; double: its FP64
// instance, for samples too large for software binary128 on aarch64).
template <typename R>
static R dense_log_k_t(R x, R nu, int* status) {
  *status = 0;
  nu = std::fabs(nu);  // K_{-nu} = K_nu: the integrand only depends on |nu|.

  // Window [0, T]: walk outward in steps of 1/64 keeping the running maximum
  // of g; stop once g has fallen 90 below it.  Before the peak g increases
  // (it is unimodal), so the stop can only happen past the peak.  The part
  // beyond T is below e^{-90} of the peak value.
  const R step = R(1) / R(64);
  R gmax = g_of_t<R>(R(0), x, nu);
  R T = R(0);
  for (long k = 1; k <= 64L * 200L; ++k) {
    R t = step * (R)k;
    R gt = g_of_t<R>(t, x, nu);
    if (gt > gmax) gmax = gt;
    if (gt < gmax - R(90)) { T = t; break; }
  }
  if (T == R(0)) { *status = 1; return NAN; }

  // The narrowest feature of the integrand is the peak, whose width is at
  // least (x^2 + nu^2)^{-1/4} (|g''| at the peak is at most x cosh t*,
  // and x sinh t* <= nu there).  Start with a step well below both that
  // width and 1/32, then halve.
  R h_start = R(0.25) / std::pow(x * x + nu * nu + R(1), R(0.25));
  if (h_start > R(1) / R(32)) h_start = R(1) / R(32);
  long M = (long)std::ceil(T / h_start);
  if (M < 64) M = 64;

  // Trapezoid on M intervals: endpoints weight 1/2, interior weight 1.  The
  // terms are exp(g(t) - gmax) so nothing overflows; K = e^{gmax} h S.
  R S = R(0.5) * (std::exp(g_of_t<R>(R(0), x, nu) - gmax) + std::exp(g_of_t<R>(T, x, nu) - gmax));
  for (long m = 1; m < M; ++m) {
    R t = T * (R)m / (R)M;
    S += std::exp(g_of_t<R>(t, x, nu) - gmax);
  }
  R prev = (T / (R)M) * S;

  // Two successive halvings must agree to 64 units of the type's epsilon
  // (at least 1e-30; 1e-17 for the x87 80-bit type).
  R tol = R(64) * std::numeric_limits<R>::epsilon();
  if (tol < R(1e-30)) tol = R(1e-30);
  if (tol < R(1e-17) && std::numeric_limits<R>::digits > 53 &&
      std::numeric_limits<R>::digits < 100)
    tol = R(1e-17);
  int agree = 0;
  for (int level = 0; level < 14; ++level) {
    // Halving adds the midpoints of the current intervals.
    R add = R(0);
    for (long m = 0; m < M; ++m) {
      R t = T * (R)(2 * m + 1) / (R)(2 * M);
      add += std::exp(g_of_t<R>(t, x, nu) - gmax);
    }
    S += add;
    M *= 2;
    R cur = (T / (R)M) * S;
    if (std::fabs(cur - prev) <= tol * cur) {
      if (++agree == 2) return gmax + std::log(cur);
    } else {
      agree = 0;
    }
    prev = cur;
  }
  *status = 1;
  return NAN;
}

static ld dense_log_k(ld x, ld nu, int* status) { return dense_log_k_t<ld>(x, nu, status); }

// ---------------------------------------------------------------------------
// Temme's series, Sec. IV-A, for |mu| <= 1/2, giving K_mu and K_{mu+1}.
//   c_k = (x^2/4)^k / k!,   K_mu = sum c_k f_k,   K_{mu+1} = (2/x) sum c_k h_k,
//   h_k = -k f_k + p_k,  p_k = p_{k-1}/(k - mu),  q_k = q_{k-1}/(k + mu),
//   f_k = (k f_{k-1} + p_{k-1} + q_{k-1}) / (k^2 - mu^2),
//   p_0 = (1/2)(x/2)^{-mu} Gamma(1+mu),  q_0 = (1/2)(x/2)^{mu} Gamma(1-mu),
//   f_0 = (mu pi / sin(mu pi)) [cosh(s) G1(mu) + (sinh(s)/s) ln(2/x) G2(mu)],
//   s = mu ln(2/x),  G1 = [1/Gamma(1-mu) - 1/Gamma(1+mu)] / (2 mu),
//   G2 = [1/Gamma(1-mu) + 1/Gamma(1+mu)] / 2.
// The paper leaves s, G1 and G2 undefined; these are Temme's (1975)
// definitions.  G1 at mu = 0 is its limit -gamma_E.
static void temme_mu(ld x, ld mu, ld* k_mu, ld* k_mu1, int* status) {
  *status = 0;
  const ld lx = logl(2.0L / x);
  const ld s = mu * lx;
  ld g1, g2;
  const ld rg_minus = 1.0L / tgammal(1.0L - mu);
  const ld rg_plus = 1.0L / tgammal(1.0L + mu);
  if (mu == 0.0L) {
    g1 = -kEulerGamma;
  } else {
    g1 = (rg_minus - rg_plus) / (2.0L * mu);
  }
  g2 = 0.5L * (rg_minus + rg_plus);
  const ld fact = (mu == 0.0L) ? 1.0L : (mu * kPi) / sinl(mu * kPi);
  const ld shs = (s == 0.0L) ? 1.0L : sinhl(s) / s;
  ld f = fact * (coshl(s) * g1 + shs * lx * g2);
  ld p = 0.5L * powl(0.5L * x, -mu) * tgammal(1.0L + mu);
  ld q = 0.5L * powl(0.5L * x, mu) * tgammal(1.0L - mu);
  ld c = 1.0L;
  const ld y = 0.25L * x * x;
  ld sum_f = c * f;
  ld sum_h = c * p;  // h_0 = -0*f_0 + p_0
  int k;
  for (k = 1; k <= 15000; ++k) {
    f = ((ld)k * f + p + q) / ((ld)k * (ld)k - mu * mu);
    p = p / ((ld)k - mu);
    q = q / ((ld)k + mu);
    c = c * y / (ld)k;
    const ld tf = c * f;
    const ld th = c * (p - (ld)k * f);
    sum_f += tf;
    sum_h += th;
    if (fabsl(tf) <= LDBL_EPSILON * fabsl(sum_f) * 0.25L &&
        fabsl(th) <= LDBL_EPSILON * fabsl(sum_h) * 0.25L)
      break;
  }
  if (k > 15000) *status = 1;
  *k_mu = sum_f;
  *k_mu1 = (2.0L / x) * sum_h;
}

// Campbell: nu = mu + M with M = floor(nu + 1/2), then Eq. (recurrence)
// K_{eta+1} = (2 eta / x) K_eta + K_{eta-1} upward from K_mu, K_{mu+1}.
static ld temme_k(ld x, ld nu, int* status) {
  nu = fabsl(nu);
  const long M = (long)floorl(nu + 0.5L);
  const ld mu = nu - (ld)M;
  ld km, km1;
  temme_mu(x, mu, &km, &km1, status);
  if (M == 0) return km;
  ld prev = km, cur = km1;  // K_mu, K_{mu+1}
  for (long j = 1; j < M; ++j) {
    const ld eta = mu + (ld)j;
    const ld next = (2.0L * eta / x) * cur + prev;
    prev = cur;
    cur = next;
  }
  return cur;
}

// ---------------------------------------------------------------------------
// The epsilon-window of Sec. IV-B.  t* = 0 when nu^2 <= x, else the unique
// positive root of g'.  t0 and t1 are the ends of {t : g(t) >= log eps + g(t*)}.
// Brackets are found by doubling (the FINDRANGE idea: the smallest power of
// two past the crossing), then refined by bisection only.
static ld bisect_decreasing_root(ld lo, ld hi, ld x, ld nu, ld target) {
  // g(lo) >= target > g(hi), g decreasing on [lo, hi].
  for (int it = 0; it < 400; ++it) {
    ld mid = 0.5L * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (g_of(mid, x, nu) >= target) lo = mid; else hi = mid;
  }
  return 0.5L * (lo + hi);
}

static void window_ld(ld x, ld nu, ld log_eps, ld* ts, ld* t0, ld* t1, ld* gs) {
  nu = fabsl(nu);
  ld tstar = 0.0L;
  if (nu * nu > x) {
    // FINDRANGE: smallest m (from -30 upward) with g'(2^m) < 0.
    ld hi = ldexpl(1.0L, -30);
    while (gprime_of(hi, x, nu) >= 0.0L) hi *= 2.0L;
    ld lo = 0.5L * hi;
    if (hi == ldexpl(1.0L, -30)) lo = 0.0L;
    // g' > 0 on (0, t*) and < 0 beyond: bisect.
    for (int it = 0; it < 400; ++it) {
      ld mid = 0.5L * (lo + hi);
      if (mid <= lo || mid >= hi) break;
      if (gprime_of(mid, x, nu) > 0.0L) lo = mid; else hi = mid;
    }
    tstar = 0.5L * (lo + hi);
  }
  const ld gstar = g_of(tstar, x, nu);
  const ld target = gstar + log_eps;

  ld left = 0.0L;
  if (tstar > 0.0L && g_of(0.0L, x, nu) < target) {
    // g increasing on [0, t*]: bisect for g = target.
    ld lo = 0.0L, hi = tstar;
    for (int it = 0; it < 400; ++it) {
      ld mid = 0.5L * (lo + hi);
      if (mid <= lo || mid >= hi) break;
      if (g_of(mid, x, nu) < target) lo = mid; else hi = mid;
    }
    left = 0.5L * (lo + hi);
  }
  // Right end: smallest k with g(t* + 2^k) < target, then bisect.
  ld d = ldexpl(1.0L, -30);
  while (g_of(tstar + d, x, nu) >= target) d *= 2.0L;
  ld lo = (d == ldexpl(1.0L, -30)) ? tstar : tstar + 0.5L * d;
  ld right = bisect_decreasing_root(lo, tstar + d, x, nu, target);

  *ts = tstar;
  *t0 = left;
  *t1 = right;
  *gs = gstar;
}

// Trapezoid with N intervals on [a, b] (the quadrature of Eq. (refined), read
// with the weights multiplying the exponential), shifted by gshift.
static ld trapezoid_log_k(ld x, ld nu, ld a, ld b, long N, ld gshift) {
  const ld h = (b - a) / (ld)N;
  ld S = 0.0L;
  for (long m = 0; m <= N; ++m) {
    const ld t = a + h * (ld)m;
    const ld w = (m == 0 || m == N) ? 0.5L : 1.0L;
    S += w * expl(g_of(t, x, nu) - gshift);
  }
  return gshift + logl(h * S);
}

// ---------------------------------------------------------------------------
extern "C" {

int oracle_long_double_digits(void) { return LDBL_MANT_DIG; }

double oracle_log_besselk(double x, double nu, int* status) {
  int st = 0;
  if (!(x > 0.0)) {
    if (status) *status = 2;
    return (x == 0.0) ? INFINITY : NAN;
  }
  ld r = dense_log_k((ld)x, (ld)nu, &st);
  if (status) *status = st;
  return (double)r;
}

double oracle_besselk(double x, double nu) {
  if (x == 0.0) return INFINITY;
  if (!(x > 0.0)) return NAN;
  int st = 0;
  ld r = dense_log_k((ld)x, (ld)nu, &st);
  if (st) return NAN;
  return (double)expl(r);
}

void oracle_besselk_batch(const double* x, const double* nu, double* out, double* log_out,
                          int64_t n, int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
#endif
  for (int64_t i = 0; i < n; ++i) {
    double xi = x[i];
    if (xi == 0.0) { out[i] = INFINITY; if (log_out) log_out[i] = INFINITY; continue; }
    if (!(xi > 0.0)) { out[i] = NAN; if (log_out) log_out[i] = NAN; continue; }
    int st = 0;
    ld r = dense_log_k((ld)xi, (ld)nu[i], &st);
    out[i] = st ? NAN : (double)expl(r);
    if (log_out) log_out[i] = st ? NAN : (double)r;
  }
}

// Derivatives of K_nu(x), by differentiating the integral of Eq. (integral)
// under the integral sign:
//   -dK/dx  = int_0^inf cosh(t) e^{-x cosh t} cosh(nu t) dt,
//    dK/dnu = int_0^inf t sinh(nu t) e^{-x cosh t} dt,
// by the same dense trapezoid as dense_log_k (window by stepping, halving to
// agreement) applied to the logs of these integrands, both positive for
// x > 0, nu > 0 and even in t (so the rule on [0, T] keeps its fast
// convergence).  kind 1: -dK/dx, kind 2: dK/dnu.  Returns the log.
static ld log_sinh_pos(ld y) { return y + log1pl(-expl(-2.0L * y)) - kLn2; }

static ld deriv_log_integrand(ld t, ld x, ld nu, int kind) {
  if (kind == 1) return g_of(t, x, nu) + logl(coshl(t));
  if (t == 0.0L || nu == 0.0L) return -INFINITY;
  return logl(t) + log_sinh_pos(nu * t) - x * coshl(t);
}

static ld dense_log_deriv(ld x, ld nu, int kind, int* status) {
  *status = 0;
  const ld step = 1.0L / 64.0L;
  ld gmax = deriv_log_integrand(0.0L, x, nu, kind);
  ld T = 0.0L;
  for (long k = 1; k <= 64L * 200L; ++k) {
    ld t = step * (ld)k;
    ld gt = deriv_log_integrand(t, x, nu, kind);
    if (gt > gmax) gmax = gt;
    if (gt < gmax - 90.0L) { T = t; break; }
  }
  if (T == 0.0L) { *status = 1; return NAN; }
  ld h_start = 0.25L / powl(x * x + nu * nu + 1.0L, 0.25L);
  if (h_start > 1.0L / 32.0L) h_start = 1.0L / 32.0L;
  long M = (long)ceill(T / h_start);
  if (M < 64) M = 64;
  ld S = 0.5L * (expl(deriv_log_integrand(0.0L, x, nu, kind) - gmax) +
                 expl(deriv_log_integrand(T, x, nu, kind) - gmax));
  for (long m = 1; m < M; ++m)
    S += expl(deriv_log_integrand(T * (ld)m / (ld)M, x, nu, kind) - gmax);
  ld prev = (T / (ld)M) * S;
  ld tol = 64.0L * LDBL_EPSILON;
  if (tol < 1e-30L) tol = 1e-30L;
  if (tol < 1e-17L && LDBL_MANT_DIG < 100) tol = 1e-17L;
  int agree = 0;
  for (int level = 0; level < 14; ++level) {
    ld add = 0.0L;
    for (long m = 0; m < M; ++m)
      add += expl(deriv_log_integrand(T * (ld)(2 * m + 1) / (ld)(2 * M), x, nu, kind) - gmax);
    S += add;
    M *= 2;
    ld cur = (T / (ld)M) * S;
    if (fabsl(cur - prev) <= tol * cur) {
      if (++agree == 2) return gmax + logl(cur);
    } else {
      agree = 0;
    }
    prev = cur;
  }
  *status = 1;
  return NAN;
}

// K, dK/dx and dK/dnu (dK/dnu is odd in nu: K_{-nu} = K_nu).  NaN on failure.
void oracle_besselk_grad_batch(const double* x, const double* nu, double* k, double* dkdx,
                               double* dkdnu, int64_t n, int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
#endif
  for (int64_t i = 0; i < n; ++i) {
    const ld X = (ld)x[i], V = fabsl((ld)nu[i]);
    int s0 = 0, s1 = 0, s2 = 0;
    const ld lk = dense_log_k(X, V, &s0);
    const ld lx = dense_log_deriv(X, V, 1, &s1);
    k[i] = s0 ? NAN : (double)expl(lk);
    dkdx[i] = s1 ? NAN : (double)(-expl(lx));
    if (V == 0.0L) {
      dkdnu[i] = 0.0;
    } else {
      const ld ln = dense_log_deriv(X, V, 2, &s2);
      const double d = s2 ? NAN : (double)expl(ln);
      dkdnu[i] = (nu[i] < 0.0) ? -d : d;
    }
  }
}

double oracle_besselk_temme(double x, double nu, int* status) {
  int st = 0;
  ld r = temme_k((ld)x, (ld)nu, &st);
  if (status) *status = st;
  return (double)r;
}

// Window labels: out[0..3] = (t*, t0, t1, g(t*)).
void oracle_window(double x, double nu, double log_eps, double* out) {
  ld ts, t0, t1, gs;
  window_ld((ld)x, (ld)nu, (ld)log_eps, &ts, &t0, &t1, &gs);
  out[0] = (double)ts;
  out[1] = (double)t0;
  out[2] = (double)t1;
  out[3] = (double)gs;
}

void oracle_window_batch(const double* x, const double* nu, double log_eps, double* out,
                         int64_t n, int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
  for (int64_t i = 0; i < n; ++i) oracle_window(x[i], nu[i], log_eps, out + 4 * i);
}

// log of the N-interval trapezoid on [t0, t1] (Eq. (refined)), shifted by the
// largest node value of g (any shift gives the same sum; this one avoids
// overflow).
double oracle_window_trapezoid_log_k(double x, double nu, double t0, double t1, int64_t N) {
  const ld X = (ld)x, V = fabsl((ld)nu), a = (ld)t0, b = (ld)t1;
  const ld h = (b - a) / (ld)N;
  ld gl = -INFINITY;
  for (long m = 0; m <= (long)N; ++m) {
    const ld gm = g_of(a + h * (ld)m, X, V);
    if (gm > gl) gl = gm;
  }
  return (double)trapezoid_log_k(X, V, a, b, (long)N, gl);
}

// Smallest N in [1, nmax] such that the N-interval trapezoid on the
// eps-window is within rel_tol of the dense integral; 0 if none.
int64_t oracle_min_nodes(double x, double nu, double log_eps, double rel_tol, int64_t nmax) {
  ld ts, a, b, gs;
  window_ld((ld)x, (ld)nu, (ld)log_eps, &ts, &a, &b, &gs);
  int st = 0;
  const ld ref = dense_log_k((ld)x, (ld)nu, &st);
  if (st) return 0;
  for (long N = 1; N <= (long)nmax; ++N) {
    const ld v = trapezoid_log_k((ld)x, fabsl((ld)nu), a, b, N, gs);
    // |K_N / K - 1| <= rel_tol  <=>  |expm1(log K_N - log K)| <= rel_tol
    if (fabsl(expm1l(v - ref)) <= (ld)rel_tol) return (int64_t)N;
  }
  return 0;
}

// Labels of the learned window: out[6*i ..] = (t*, t0, t1, g(t*), N, T_ref)
// where [t0, t1] is the eps-window (bisection, as oracle_window), N the
// smallest interval count whose trapezoid on that window is within rel_tol of
// the 512-interval trapezoid on the same window (T_ref; the window's own
// truncation is not part of N's job), or 0 if none up to nmax.
void oracle_window_labels_batch(const double* x, const double* nu, double log_eps, double rel_tol,
                                int64_t nmax, double* out, int64_t n, int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
  for (int64_t i = 0; i < n; ++i) {
    ld ts, a, b, gs;
    const ld X = (ld)x[i], V = fabsl((ld)nu[i]);
    window_ld(X, V, (ld)log_eps, &ts, &a, &b, &gs);
    const ld ref = trapezoid_log_k(X, V, a, b, 512, gs);
    long found = 0;
    for (long N = 1; N <= (long)nmax; ++N) {
      const ld v = trapezoid_log_k(X, V, a, b, N, gs);
      if (fabsl(expm1l(v - ref)) <= (ld)rel_tol) { found = N; break; }
    }
    double* o = out + 6 * i;
    o[0] = (double)ts;
    o[1] = (double)a;
    o[2] = (double)b;
    o[3] = (double)gs;
    o[4] = (double)found;
    o[5] = (double)ref;
  }
}

void oracle_min_nodes_batch(const double* x, const double* nu, double log_eps, double rel_tol,
                            int64_t nmax, int64_t* out, int64_t n, int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
#endif
  for (int64_t i = 0; i < n; ++i) out[i] = oracle_min_nodes(x[i], nu[i], log_eps, rel_tol, nmax);
}

// The paper's refined integration branch (Algorithm 2, x >= 0.1 part): window
// fixed to [0, t1] (t1 = 9 in the paper), b bins, shift by the largest node
// value of g, trapezoid weights c_0 = c_b = 1/2 multiplying the exponential.
double oracle_fixed_window_log_k(double x, double nu, double t1, int64_t b) {
  const ld X = (ld)x, V = fabsl((ld)nu);
  const ld h = (ld)t1 / (ld)b;
  ld gl = -INFINITY;
  for (long m = 0; m <= (long)b; ++m) {
    ld gm = g_of(h * (ld)m, X, V);
    if (gm > gl) gl = gm;
  }
  ld S = 0.0L;
  for (long m = 0; m <= (long)b; ++m) {
    const ld c = (m == 0 || m == (long)b) ? 0.5L : 1.0L;
    S += h * c * expl(g_of(h * (ld)m, X, V) - gl);
  }
  return (double)(gl + logl(S));
}

// ---------------------------------------------------------------------------
// Matern covariance, Sec. III-A:
//   M(r) = sigma^2 / (2^{nu-1} Gamma(nu)) (r/beta)^nu K_nu(r/beta),
// with M = sigma^2 where the distance is exactly zero (Algorithm 3).
// Evaluated in the log domain, everything in long double.
static ld matern_ld(ld xi, ld yi, ld xj, ld yj, ld sigma2, ld beta, ld nu, int* status) {
  *status = 0;
  const ld dx = xj - xi, dy = yj - yi;
  const ld r = sqrtl(dx * dx + dy * dy);
  if (r == 0.0L) return sigma2;
  const ld z = r / beta;
  const ld logk = dense_log_k(z, nu, status);
  const ld logc = logl(sigma2) - (nu - 1.0L) * kLn2 - lgammal(nu);
  return expl(logc + nu * logl(z) + logk);
}

// Entries (I[k], J[k]) of the matrix for locations in SoA layout
// locs = [x_0..x_{n-1}, y_0..y_{n-1}].
void oracle_matern_entries(const double* locs, int64_t n, const int64_t* I, const int64_t* J,
                           int64_t m, double sigma2, double beta, double nu, double* out,
                           int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
#endif
  for (int64_t k = 0; k < m; ++k) {
    const int64_t i = I[k], j = J[k];
    int st = 0;
    ld v = matern_ld((ld)locs[i], (ld)locs[n + i], (ld)locs[j], (ld)locs[n + j], (ld)sigma2,
                     (ld)beta, (ld)nu, &st);
    out[k] = st ? NAN : (double)v;
  }
}

// Full m x n block between two location sets, column-major, out[i + j*ld].
void oracle_matern_block(const double* locs1, int64_t m, const double* locs2, int64_t n,
                         double sigma2, double beta, double nu, double* out, int64_t ld_,
                         int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for collapse(2) schedule(dynamic, 8)
#endif
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < m; ++i) {
      int st = 0;
      ld v = matern_ld((ld)locs1[i], (ld)locs1[m + i], (ld)locs2[j], (ld)locs2[n + j],
                       (ld)sigma2, (ld)beta, (ld)nu, &st);
      out[i + j * ld_] = st ? NAN : (double)v;
    }
}

// The FP64 instance of the oracle (dense_log_k_t<double>): K_nu(x) and its
// log for large samples; agrees with the long double oracle to about 1e-13
// relative over the region of Sec. IV-C (pinned in the tests).
void oracle_besselk_batch_f64(const double* x, const double* nu, double* out, double* log_out,
                              int64_t n, int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
  for (int64_t i = 0; i < n; ++i) {
    const double xi = x[i];
    if (xi == 0.0) { out[i] = INFINITY; if (log_out) log_out[i] = INFINITY; continue; }
    if (!(xi > 0.0)) { out[i] = NAN; if (log_out) log_out[i] = NAN; continue; }
    int st = 0;
    const double r = dense_log_k_t<double>(xi, nu[i], &st);
    out[i] = st ? NAN : std::exp(r);
    if (log_out) log_out[i] = st ? NAN : r;
  }
}

// Matern entries (I[k], J[k]) by the FP64 instance: the steps of matern_ld
// in double.
void oracle_matern_entries_f64(const double* locs, int64_t n, const int64_t* I, const int64_t* J,
                               int64_t m, double sigma2, double beta, double nu, double* out,
                               int nthreads) {
  const double logc = std::log(sigma2) - (nu - 1.0) * (double)kLn2 - std::lgamma(nu);
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
  for (int64_t k = 0; k < m; ++k) {
    const int64_t i = I[k], j = J[k];
    const double dx = locs[j] - locs[i], dy = locs[n + j] - locs[n + i];
    const double r = std::sqrt(dx * dx + dy * dy);
    if (r == 0.0) { out[k] = sigma2; continue; }
    const double z = r / beta;
    int st = 0;
    const double logk = dense_log_k_t<double>(z, nu, &st);
    out[k] = st ? NAN : std::exp(logc + nu * std::log(z) + logk);
  }
}

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

}  // extern "C"
