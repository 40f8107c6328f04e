// Host planner: algorithmic parameters, Bessel-root nodes, the recursive
// partition, the stacked-column weight tables and the near-field Bessel
// table of a plan. Pure host C++; no CUDA call is made here.
//
// References are to Townsend, arXiv:1501.01652 (sections, equations, tables).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <utility>
#include <vector>

#include "plan.h"

namespace hk {
namespace {

constexpr double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------------------
// Double-double arithmetic (head + tail), used for plan-time Bessel values.
// Sums renormalise once (head two-sum, tails added); products take the exact
// head product from an FMA and fold the cross terms into its error by FMAs;
// quotients multiply by a reciprocal refined with one Newton step.
// ---------------------------------------------------------------------------
struct DD {
  double h, l;
};
inline DD ddv(double a) { return DD{a, 0.0}; }
// (s, e) with |e| small against s, renormalised so that h = fl(s + e)
inline DD dd_fast(double s, double e) {
  const double h = s + e;
  return DD{h, e - (h - s)};
}
inline DD dd_add(DD a, DD b) {
  double s = a.h + b.h, v = s - a.h;
  double e = (a.h - (s - v)) + (b.h - v);
  e += a.l + b.l;
  return dd_fast(s, e);
}
inline DD dd_neg(DD a) { return DD{-a.h, -a.l}; }
inline DD dd_mul(DD a, DD b) {
  const double p = a.h * b.h;
  return dd_fast(p, std::fma(a.l, b.h, std::fma(a.h, b.l, std::fma(a.h, b.h, -p))));
}
// 1/b: x0 = fl(1/b.h), then x1 = x0 + x0 (1 - b x0); the residual 1 - b x0 is ~2^-53, so one step
// leaves a relative error of order 2^-104.
inline DD dd_recip(DD b) {
  const double x0 = 1.0 / b.h;
  const DD res = dd_add(ddv(1.0), dd_neg(dd_mul(b, ddv(x0))));
  return dd_add(ddv(x0), dd_mul(ddv(x0), res));
}
inline DD dd_scale(DD a, double p2) { return DD{a.h * p2, a.l * p2}; }
const DD kPiDD = {3.141592653589793116, 1.2246467991473532072e-16};

// J_lambda(z) for lambda = 0..L (z > 0) by Miller's backward recurrence
// J_{k-1} = (2k/z) J_k - J_{k+1} (DLMF 3.6(vi)), started from zero above max(z, L). The scale
// comes from the sum of squares J_0^2 + 2 sum_{k>=1} J_k^2 = 1 (DLMF 10.23.3), whose terms are
// all positive; its sign from J_0 + 2 sum_{k>=1} J_{2k} = 1 (DLMF 10.12.4). Double-double.
void miller_all(DD z, int L, std::vector<DD>& out) {
  const int top = 2 * (((int)z.h + 90 + L) / 2 + 1);
  std::vector<DD> v((size_t)top + 2, ddv(0.0));
  const DD twoz = dd_scale(dd_recip(z), 2.0);
  v[top] = ddv(0x1p-140);
  for (int k = top; k >= 1; --k) {
    v[k - 1] = dd_add(dd_mul(dd_mul(ddv((double)k), twoz), v[k]), dd_neg(v[k + 1]));
    if (std::fabs(v[k - 1].h) > 1e100)  // keeps the squares below in range
      for (int i = k - 1; i <= top; ++i) v[i] = dd_scale(v[i], 0x1p-400);
  }
  DD sq = dd_mul(v[0], v[0]), lin = v[0];
  for (int k = 1; k <= top; ++k) {
    sq = dd_add(sq, dd_scale(dd_mul(v[k], v[k]), 2.0));
    if ((k & 1) == 0) lin = dd_add(lin, dd_scale(v[k], 2.0));
  }
  // 1/sqrt(sq): from the FP64 root, one Newton step y1 = y0 (3 - sq y0^2) / 2
  const double y0 = 1.0 / std::sqrt(sq.h);
  const DD t = dd_add(ddv(3.0), dd_neg(dd_mul(sq, dd_mul(ddv(y0), ddv(y0)))));
  DD inv = dd_scale(dd_mul(ddv(y0), t), 0.5);
  if (lin.h < 0) inv = dd_neg(inv);
  out.resize(L + 1);
  for (int i = 0; i <= L; ++i) out[i] = dd_mul(v[i], inv);
}

// ---------------------------------------------------------------------------
// Hankel expansion coefficients (Eq. 4)
// ---------------------------------------------------------------------------
// a_m(nu) = prod_{i=1}^m (4nu^2 - (2i-1)^2) / (m! 8^m), m = 0..mmax.
void hankel_a(int nu, int mmax, double* a) {
  double mu4 = 4.0 * (double)nu * (double)nu;
  a[0] = 1.0;
  for (int m = 1; m <= mmax; ++m) a[m] = a[m - 1] * (mu4 - (2.0 * m - 1.0) * (2.0 * m - 1.0)) / (8.0 * m);
}

// exp(i pi q / 4) for integer q, with exact values.
cplx expi_quarter_pi(int q) {
  const double h = 0.70710678118654752440;
  static const double cr[8] = {1, h, 0, -h, -1, -h, 0, h};
  static const double ci[8] = {0, h, 1, h, 0, -h, -1, -h};
  int r = ((q % 8) + 8) % 8;
  return cplx(cr[r], ci[r]);
}

// J_lam(z) ~ Re[ e^{iz} sum_{j<2M} c_j(lam) z^{-(j+1/2)} ] with
// c_j(lam) = sqrt(2/pi) e^{-i(2lam+1)pi/4} i^j a_j(lam): Eq. (4) written with
// cos(mu) = Re e^{i mu}, sin(mu) = Im e^{i mu}, mu = z - (2lam+1)pi/4.
void hankel_c(int lam, int M, cplx* c) {
  double a[64];
  hankel_a(lam, 2 * M - 1, a);
  const double s2p = 0.79788456080286535588;  // sqrt(2/pi)
  for (int j = 0; j < 2 * M; ++j) c[j] = s2p * a[j] * expi_quarter_pi(2 * j - 2 * lam - 1);
}

// Rearranged truncated Neumann/Taylor sum of Section 5.1: for perturbed
// arguments, J_nu(x(v+w)) ~ sum_{u=0}^{2T+K-3} (x w)^u sum_lam g_{u,lam} J_lam(x v), with
// g collecting (-1)^t 2^{-u} / (t!(u-t)!) [J_{nu-s} + (-1)^s J_{nu+s}], s = u - 2t,
// t from max(ceil((u-K+1)/2), 0) to min(floor(u/2), T-1), and the s = 0 term halved
// (the primed sums). Returns (lam, g) pairs for one u.
std::vector<std::pair<int, double>> neumann_terms(int nu, int K, int T, int u) {
  std::vector<std::pair<int, double>> out;
  int a = u - K + 1;
  int tlo = a <= 0 ? 0 : (a + 1) / 2;
  int thi = std::min(u / 2, T - 1);
  for (int t = tlo; t <= thi; ++t) {
    int s = u - 2 * t;
    double c = (t & 1) ? -1.0 : 1.0;
    c = std::ldexp(c, -u);
    for (int i = 2; i <= t; ++i) c /= i;
    for (int i = 2; i <= u - t; ++i) c /= i;
    if (s == 0) {
      out.push_back({nu, c});
    } else {
      out.push_back({nu - s, c});
      out.push_back({nu + s, (s & 1) ? -c : c});
    }
  }
  return out;
}

double factorial(int n) {
  double f = 1.0;
  for (int i = 2; i <= n; ++i) f *= i;
  return f;
}

// ---------------------------------------------------------------------------
// Bessel roots j_{0,n} as b_n = j_{0,n} - (n-1/4)pi (Lemma 3.2)
// ---------------------------------------------------------------------------
// The two series of Eq. (4) at once: S(z) = sum_{m<=L} a_m(lam) (i/z)^m, so that Re S = P(z)
// (the cosine series, sum (-1)^k a_2k z^-2k) and Im S = Q(z) (the sine series,
// sum (-1)^k a_2k+1 z^-2k-1). L is the last index before the terms stop shrinking or drop below
// 2^-70; S is summed by Horner's rule in the complex variable w = i/z, from the smallest term
// up: S <- a_m + w S, where multiplying by w maps (x, y) to (-y/z, x/z).
struct HankelA {
  double a[96];
  explicit HankelA(int lam) { hankel_a(lam, 95, a); }
};
cplx hankel_pq(int lam, double z) {
  static const HankelA a0(0), a1(1);  // the orders used here: roots of J_0, J_1 at those roots
  HankelA own(lam < 2 ? 0 : lam);
  const double* a = lam == 0 ? a0.a : lam == 1 ? a1.a : own.a;
  const double iz = 1.0 / z;
  int L = 0;
  double mag = std::fabs(a[0]), zm = 1.0;
  for (int m = 1; m < 95; ++m) {
    zm *= iz;
    const double next = std::fabs(a[m]) * zm;
    if (next > mag || mag < 0x1p-70) break;
    mag = next;
    L = m;
  }
  double x = a[L], y = 0.0;
  for (int m = L - 1; m >= 0; --m) {
    const double nx = a[m] - y * iz;
    y = x * iz;
    x = nx;
  }
  return cplx(x, y);
}

// Large roots: from Eq. (4) with lam = 0, J_0(z) ~ sqrt(2/(pi z)) Re[e^{i mu} S(z)] with
// mu = z - pi/4 = (n-1/2)pi + b, so J_0 = 0 <=> Re[i e^{ib} S] = 0 <=> b = atan(-Q/P),
// z = (n-1/4)pi + b. The map b -> atan(-Q/P) contracts by ~1/(8 z^2); its fixed point keeps
// b's full relative accuracy.
double root_offset_large(double n) {
  const double beta = (n - 0.25) * kPi;
  double b = 0.125 / beta;
  for (int it = 0; it < 12; ++it) {
    const cplx S = hankel_pq(0, beta + b);
    const double nb = std::atan(-S.imag() / S.real());
    const bool done = std::fabs(nb - b) <= 1e-19 * b;
    b = nb;
    if (done) break;
  }
  return b;
}

// Small roots (z < 30, where Eq. (4) is not accurate to double-double): Halley's iteration on
// J_0 in double-double from the large-root formula's guess. With f = J_0, f' = -J_1 and
// f'' = J_1/z - J_0 (Bessel's equation), the step is -2 f f' / (2 f'^2 - f f''); J_0 and J_1
// come from Miller's recurrence at z = (n-1/4)pi + b.
double root_offset_small(int64_t n) {
  const DD base = dd_mul(kPiDD, ddv(n - 0.25));
  DD b = ddv(root_offset_large(n));
  std::vector<DD> J;
  for (int it = 0; it < 8; ++it) {
    const DD z = dd_add(base, b);
    miller_all(z, 1, J);
    const DD f = J[0], fp = dd_neg(J[1]);
    const DD fpp = dd_add(dd_mul(J[1], dd_recip(z)), dd_neg(J[0]));
    const DD num = dd_scale(dd_mul(f, fp), -2.0);
    const DD den = dd_add(dd_scale(dd_mul(fp, fp), 2.0), dd_neg(dd_mul(f, fpp)));
    const DD step = dd_mul(num, dd_recip(den));
    b = dd_add(b, step);
    if (std::fabs(step.h) < 1e-32 * std::fabs(b.h)) break;
  }
  return b.h + b.l;
}

// sin and cos of pi*A/B (integers, B > 0). The angle is reduced in integers to an octant:
// with a = A mod 2B, the angle is (pi/4)(o + r/B), o = floor(4a/B) in 0..7, r = 4a - oB in
// [0, B). In an even octant it is o/2 quarter turns plus theta = (pi/4)(r/B); in an odd one,
// (o+1)/2 quarter turns minus theta' = (pi/4)((B-r)/B); both angles lie in [0, pi/4], where
// sin and cos keep full relative accuracy.
void sincospi_ratio(int64_t A, int64_t B, double* s, double* c) {
  const int64_t twoB = 2 * B;
  const int64_t a = ((A % twoB) + twoB) % twoB;
  const int64_t o = (4 * a) / B;
  const int64_t r = 4 * a - o * B;
  const bool odd = (o & 1) != 0;
  const double th = 0.25 * kPi * ((double)(odd ? B - r : r) / (double)B);
  double x = std::cos(th), y = odd ? -std::sin(th) : std::sin(th);  // e^{+-i theta}
  for (int64_t k = (o + (odd ? 1 : 0)) / 2 % 4; k > 0; --k) {  // times i per quarter turn
    const double t = x;
    x = -y;
    y = t;
  }
  *c = x;
  *s = y;
}

int64_t ceil_index(double tau, double shift) {
  // smallest integer i >= 1 with i + shift >= tau
  double v = std::ceil(tau - shift);
  int64_t i = (int64_t)v;
  while (i > 1 && (double)(i - 1) + shift >= tau) --i;
  while ((double)i + shift < tau) ++i;
  return std::max<int64_t>(i, 1);
}

}  // namespace

void j0_zero_offsets(int64_t count, double* b) {
  for (int64_t n = 1; n <= count; ++n) b[n - 1] = ((n - 0.25) * kPi < 30.0) ? root_offset_small(n) : root_offset_large(n);
}

// |J_1(j_{0,n})| with j_{0,n} = (n-1/4)pi + b_n. Large roots: Eq. (4) with nu = 1, whose phase
// z - 3pi/4 = (n-1)pi + b_n leaves |J_1| = sqrt(2/(pi z)) |P(z) cos b_n - Q(z) sin b_n| (P, Q the
// even and odd parts of the Hankel series, summed to its smallest term); small roots: Miller's
// recurrence in double-double at z.
double j1_at_j0_zero(int64_t n, double b) {
  if ((n - 0.25) * kPi < 30.0) {
    std::vector<DD> J;
    miller_all(dd_add(dd_mul(kPiDD, ddv(n - 0.25)), ddv(b)), 1, J);
    return std::fabs(J[1].h + J[1].l);
  }
  // Eq. (4), nu = 1: J_1(z) ~ sqrt(2/(pi z)) Re[e^{i mu} S(z)], mu = z - 3pi/4 = (n-1)pi + b,
  // and e^{i (n-1) pi} = +-1 drops out of the absolute value
  const double z = (n - 0.25) * kPi + b;
  const cplx S = hankel_pq(1, z);
  return std::sqrt(2.0 / (kPi * z)) * std::fabs((std::polar(1.0, b) * S).real());
}

void dht_inverse_weights(int64_t N, const double* b, double* v) {
  for (int64_t n = 1; n <= N; ++n) {
    const double j1 = j1_at_j0_zero(n, b[n - 1]);
    v[n - 1] = 2.0 / (j1 * j1);
  }
}

}  // namespace hk

// ---------------------------------------------------------------------------
// Host-only parameter formulas exported through the C ABI
// ---------------------------------------------------------------------------
extern "C" double hankel_s_nu_M(int nu, int M, double eps) {
  // Section 3.1: s^{(j+1)} = (sqrt(2)(|a_2M| + |a_2M+1|/s^{(j)}) / (sqrt(pi) eps))^{1/(2M+1/2)}, s^{(0)} = 1, four steps.
  double a[128];
  if (M < 1 || M > 60 || !(eps > 0)) return NAN;
  hk::hankel_a(nu, 2 * M + 1, a);
  double s = 1.0;
  for (int j = 0; j < 4; ++j)
    s = std::pow(std::sqrt(2.0) * (std::fabs(a[2 * M]) + std::fabs(a[2 * M + 1]) / s) / (std::sqrt(hk::kPi) * eps),
                 1.0 / (2.0 * M + 0.5));
  return s;
}

extern "C" double hankel_t_nu_T(int nu, int T, double eps) {
  // Section 3.2: t_{nu,T}(eps) ~ (2^{2T+nu} (T+nu)! T! eps)^{1/(2T+nu)}
  if (T < 1 || nu < 0 || !(eps > 0)) return NAN;
  double e = 2.0 * T + nu;
  double lg = e * std::log(2.0) + std::lgamma(T + nu + 1.0) + std::lgamma(T + 1.0) + std::log(eps);
  return std::exp(lg / e);
}

extern "C" double hankel_neumann_radius(int K, double eps) {
  // Eq. (10): |dz| <= (2/e) (eps/5.2)^{1/K}
  if (K < 1 || !(eps > 0)) return NAN;
  return 2.0 / std::exp(1.0) * std::pow(eps / 5.2, 1.0 / K);
}

extern "C" double hankel_p_K(int K, double eps) {
  // Eq. (23): p_K(eps) = e/(16 pi) (5.2/eps)^{1/K} + 1/4
  if (K < 1 || !(eps > 0)) return NAN;
  return std::exp(1.0) / (16.0 * hk::kPi) * std::pow(5.2 / eps, 1.0 / K) + 0.25;
}

extern "C" double hankel_q_T(int T, double eps) {
  // Eq. (24): q_T(eps) = eps^{-1/(2T)} / (16 pi (T!)^{1/T}) + 1/4
  if (T < 1 || !(eps > 0)) return NAN;
  return std::pow(eps, -1.0 / (2.0 * T)) / (16.0 * hk::kPi * std::pow(hk::factorial(T), 1.0 / T)) + 0.25;
}

namespace hk {

int choose_params(const hankel_options& o, HostPlan& hp) {
  hp.opt = o;
  if (o.N < 2 || o.N > (int64_t(1) << 24)) return HANKEL_EINVAL;
  if (!(o.eps > 0.0) || !(o.eps < 1.0)) return HANKEL_EINVAL;
  if (o.nu < 0 || o.nu > 64) return HANKEL_EINVAL;
  if (o.task < HANKEL_SCHLOMILCH || o.task > HANKEL_DHT) return HANKEL_EINVAL;
  if (o.task == HANKEL_DHT && o.nu != 0) return HANKEL_EINVAL;
  if (o.grid != HANKEL_GRID_UNIT && o.grid != HANKEL_GRID_PAPER) return HANKEL_EINVAL;
  if (o.max_nrhs < 1) return HANKEL_EINVAL;
  if (o.precision < HANKEL_PREC_AUTO || o.precision > HANKEL_PREC_MIXED) return HANKEL_EINVAL;
  if (o.task == HANKEL_SCHLOMILCH && (o.gamma < -1 || o.gamma > 1024)) return HANKEL_EINVAL;
  if (o.eps < 1e-16) return HANKEL_EUNSUPPORTED;
  if (o.precision == HANKEL_PREC_FP32 && o.eps < 1e-5) return HANKEL_EUNSUPPORTED;
  if (o.precision == HANKEL_PREC_DF64 && o.eps < 1e-11) return HANKEL_EUNSUPPORTED;
  // FP32 transform and near-field stages only where the accuracy goal allows them (eps >= 1e-5);
  // below that every stage is FP64 unless the caller opts into narrower arithmetic: double-float
  // transforms where their ~2^-48 rounding stays far below eps (DF64, or MIXED at eps >= 1e-11).
  // Nodes, phases and all plan tables stay FP64.
  const bool wide = o.precision == HANKEL_PREC_AUTO || o.precision == HANKEL_PREC_MIXED;
  hp.fp32 = (o.precision == HANKEL_PREC_FP32) || (wide && o.eps >= 1e-5);
  hp.df64 = !hp.fp32 && ((o.precision == HANKEL_PREC_DF64) || (o.precision == HANKEL_PREC_MIXED && o.eps >= 1e-11));

  const int64_t N = o.N;
  // Table 4: M = max(floor(0.3 log(1/eps)), 3), natural logarithm.
  hp.M = std::max((int)std::floor(0.3 * std::log(1.0 / o.eps)), 3);

  if (o.task == HANKEL_SCHLOMILCH) {
    hp.K = hp.T = hp.K2 = hp.T2 = 1;
    hp.U1 = hp.U2 = 1;
    hp.mu_max = o.nu;
  } else {
    // Section 5: K, T the smallest integers with p_K <= 30 and q_T <= 30 (Eqs. 23-24);
    // Section 6 (DHT rows): the smallest with 1.01 max(p_K, q_T) <= 30.
    auto smallest_K = [&](double fac) { int K = 1; while (fac * hankel_p_K(K, o.eps) > 30.0) ++K; return K; };
    auto smallest_T = [&](double fac) { int T = 1; while (fac * hankel_q_T(T, o.eps) > 30.0) ++T; return T; };
    if (o.task == HANKEL_FOURIER_BESSEL) {
      hp.K = hp.K2 = smallest_K(1.0);
      hp.T = hp.T2 = smallest_T(1.0);
      hp.U1 = 1;
      hp.U2 = 2 * hp.T + hp.K - 2;
      hp.mu_max = o.nu + hp.K - 1;
      hp.ncd = (int64_t)std::floor(std::max(hankel_p_K(hp.K, o.eps), hankel_q_T(hp.T, o.eps)));
    } else {
      hp.K = smallest_K(1.01);
      hp.T = smallest_T(1.01);
      hp.K2 = smallest_K(1.0);
      hp.T2 = smallest_T(1.0);
      hp.U1 = 2 * hp.T + hp.K - 2;
      hp.U2 = 2 * hp.T2 + hp.K2 - 2;
      hp.mu_max = (hp.K - 1) + (hp.K2 - 1);
      hp.nrd = (int64_t)std::floor(1.01 * std::max(hankel_p_K(hp.K, o.eps), hankel_q_T(hp.T, o.eps)));
      hp.ncd = (int64_t)std::floor(std::max(hankel_p_K(hp.K2, o.eps), hankel_q_T(hp.T2, o.eps)));
    }
    if (hp.U1 > kMaxU || hp.U2 > kMaxU) return HANKEL_EUNSUPPORTED;
  }
  hp.nrd = std::min(hp.nrd, N);
  hp.ncd = std::min(hp.ncd, N);
  // alpha from the largest order met in the expansion (all orders share one partition).
  hp.s = hankel_s_nu_M(hp.mu_max, hp.M, o.eps);
  hp.alpha = std::sqrt(hp.s / kPi);
  // Table 4: beta = min(3/log N, 1), P = ceil(log(30 alpha^{-1} N^{-1/2}) / log beta), at least 0.
  hp.beta = std::min(3.0 / std::log((double)N), 1.0);
  hp.P = 0;
  if (hp.beta < 1.0) {
    double v = std::log(30.0 / (hp.alpha * std::sqrt((double)N))) / std::log(hp.beta);
    hp.P = std::max(0, (int)std::ceil(v));
  }

  // Phase and partition coordinates of each task.
  if (o.task == HANKEL_SCHLOMILCH) {
    hp.Ua = 1; hp.Va = 1; hp.Vb = o.gamma;
    hp.y0 = (double)o.gamma;
    if (o.grid == HANKEL_GRID_UNIT) { hp.Ub = -1; hp.E = N - 1; hp.x0 = 1.0; hp.D = (double)(N - 1); }
    else { hp.Ub = 0; hp.E = N; hp.x0 = 0.0; hp.D = (double)N; }
  } else if (o.task == HANKEL_FOURIER_BESSEL) {
    hp.Ua = 4; hp.Va = 4; hp.Vb = -1;
    hp.y0 = -0.25;
    if (o.grid == HANKEL_GRID_UNIT) { hp.Ub = -4; hp.E = 16 * (N - 1); hp.x0 = 1.0; hp.D = (double)(N - 1); }
    else { hp.Ub = 0; hp.E = 16 * N; hp.x0 = 0.0; hp.D = (double)N; }
  } else {
    hp.Ua = 4; hp.Ub = -1; hp.Va = 4; hp.Vb = -1; hp.E = 16 * N + 12;
    hp.x0 = 0.25; hp.y0 = -0.25; hp.D = (double)N + 0.75;
  }
  return HANKEL_OK;
}

namespace {

void build_nodes(HostPlan& hp) {
  const hankel_options& o = hp.opt;
  const int64_t N = o.N;
  hp.r_true.assign(N, 0.0);
  hp.om_true.assign(N, 0.0);
  hp.rowvar.assign(N, 0.0);
  hp.rowpert.assign(N, 0.0);
  hp.omt.assign(N, 0.0);
  hp.betan.assign(N, 0.0);
  hp.colpow.assign(N, 1.0);
  if (o.task != HANKEL_SCHLOMILCH) {
    hp.b.assign(N + 1, 0.0);
    j0_zero_offsets(N + 1, hp.b.data());
  }
  for (int64_t k = 1; k <= N; ++k) {
    double r;
    if (o.task == HANKEL_DHT) {
      // r_k = j_{0,k}/j_{0,N+1} = r~_k + e_k, r~_k = (4k-1)/(4N+3),
      // e_k = (b_k (N+3/4) - b_{N+1} (k-1/4)) / (j_{0,N+1} (N+3/4)) (proof of Lemma 3.2).
      double jN1 = (N + 0.75) * kPi + hp.b[N];
      double rt = (double)(4 * k - 1) / (double)(4 * N + 3);
      double e = (hp.b[k - 1] * (N + 0.75) - hp.b[N] * (k - 0.25)) / (jN1 * (N + 0.75));
      hp.rowvar[k - 1] = rt;
      hp.rowpert[k - 1] = e;
      r = rt + e;
    } else {
      r = (o.grid == HANKEL_GRID_UNIT) ? (double)(k - 1) / (double)(N - 1) : (double)k / (double)N;
      hp.rowvar[k - 1] = r;
    }
    hp.r_true[k - 1] = r;
  }
  for (int64_t n = 1; n <= N; ++n) {
    if (o.task == HANKEL_SCHLOMILCH) {
      double w = (double)(n + o.gamma) * kPi;
      hp.om_true[n - 1] = w;
      hp.omt[n - 1] = w;
    } else {
      double wt = (n - 0.25) * kPi;
      double bn = hp.b[n - 1];
      hp.omt[n - 1] = wt;
      hp.om_true[n - 1] = wt + bn;
      hp.betan[n - 1] = bn / wt;
      if (o.task == HANKEL_DHT) hp.colpow[n - 1] = wt + bn;
    }
  }
}

// A thin block (few rows or few columns) does not need one transform as long as
// R + C: cutting the long side into segments of S gives short convolutions of
// length F >= thin + S - 1 whose results add up exactly (overlap-add over column
// segments when rows are few, overlap-save over row segments when columns are
// few). Pick the length with the fewest estimated FP64 operations per column:
// about 3.6 per point and radix-2 stage of each FFT plus 4 per point and segment
// for the spectrum products.
// In an FP64 plan, the radix-32 and radix-64 passes of a transform run on the tensor cores, at about
// 0.56 of the FP64 pipe's time per point (the autotuned splits against the built-in ones at 2^12,
// 2^18 and 2^21 points). A length's stages are costed by the share of its bits those radices can
// take in a split of 2-4 passes of radix 2^5..2^8 (below 2^12 points, the first pass only):
// 2^13 and 2^14 keep a radix-128 or radix-256 pass on the FP64 pipe, 2^19 one of radix 128.
constexpr double kStageOps = 3.6, kMacOps = 4.0, kTensorStageFrac = 0.56;

int tensor_bits(int logF) {
  if (logF < 10) return 0;
  if (logF < 12) return logF == 10 ? 5 : 6;
  if (logF == 13 || logF == 14) return 6;
  if (logF == 19) return 12;
  return logF;
}

double stage_ops(const HostPlan& hp, int logF) {
  if (hp.fp32 || hp.df64) return kStageOps;
  return kStageOps * (1.0 - (1.0 - kTensorStageFrac) * tensor_bits(logF) / (double)logF);
}

double full_column_cost(const HostPlan& hp, const Block& b) {
  return 2.0 * b.F * b.logF * stage_ops(hp, b.logF) + kMacOps * b.F;
}

void choose_segments(const HostPlan& hp, Block& b) {
  const int64_t thin = std::min(b.R, b.C), wide = std::max(b.R, b.C);
  const double kMac = kMacOps;
  double best = full_column_cost(hp, b);
  const int lfull = b.logF;  // b.logF changes when a shorter length wins
  for (int lf = 6; lf < lfull; ++lf) {
    const int64_t Fs = int64_t(1) << lf;
    if (Fs < 2 * thin) continue;
    const int64_t S = Fs - thin + 1;
    const int64_t nseg = (wide + S - 1) / S;
    const double cost = (double)(nseg + 1) * Fs * lf * stage_ops(hp, lf) + kMac * (double)nseg * Fs;
    if (cost < best) {
      best = cost;
      b.mode = (b.R <= b.C) ? kBlockRowSeg : kBlockColSeg;
      b.F = Fs;
      b.logF = lf;
      b.S = S;
      b.nseg = nseg;
    }
  }
}

// Estimated FP64 operations per stacked column of a block (the model of choose_segments).
double column_cost(const HostPlan& hp, const Block& b) {
  if (b.mode == kBlockFull) return full_column_cost(hp, b);
  return (double)(b.nseg + 1) * b.F * b.logF * stage_ops(hp, b.logF) + kMacOps * (double)b.nseg * b.F;
}

// A far block on rows k0..k1 and columns n0..n1 with its transform length and segmenting.
Block make_block(const HostPlan& hp, int64_t k0, int64_t k1, int64_t n0, int64_t n1) {
  Block b;
  b.k0 = k0; b.k1 = k1; b.n0 = n0; b.n1 = n1;
  b.R = k1 - k0 + 1;
  b.C = n1 - n0 + 1;
  int lf = 6;  // at least 64 points
  while ((int64_t(1) << lf) < b.R + b.C - 1) ++lf;
  b.logF = lf;
  b.F = int64_t(1) << lf;
  b.mode = kBlockFull;
  b.S = b.C;
  b.nseg = 1;
  if (!(hp.opt.flags & HANKEL_FLAG_NO_SEGMENT)) choose_segments(hp, b);
  return b;
}

void build_partition(HostPlan& hp) {
  const int64_t N = hp.opt.N;
  const double sq = std::sqrt(hp.D);
  auto tau = [&](int p) { return hp.alpha * std::pow(hp.beta, (double)p) * sq; };
  auto kidx = [&](double t) { return ceil_index(t, -hp.x0); };  // k - x0 >= t
  auto nidx = [&](double t) { return ceil_index(t, hp.y0); };   // n + y0 >= t
  std::vector<Block> raw;
  auto add = [&](int64_t k0, int64_t k1, int64_t n0, int64_t n1) {
    k0 = std::max(k0, hp.nrd + 1);
    n0 = std::max(n0, hp.ncd + 1);
    k1 = std::min(k1, N);
    n1 = std::min(n1, N);
    if (k0 > k1 || n0 > n1) return;
    raw.push_back(make_block(hp, k0, k1, n0, n1));
  };
  // Eq. (19): Q1 J Q1 and, for p = 1..P, Q_{2p+1} J Q_{2p} and Q_{2p} J Q_{2p+1}, with the
  // row band of Q_{2p+1} read as [alpha beta^p sqrt(N), alpha beta^{p-1} sqrt(N)).
  add(kidx(tau(0)), N, nidx(tau(0)), N);
  for (int p = 1; p <= hp.P; ++p) {
    add(kidx(tau(p)), kidx(tau(p - 1)) - 1, nidx(tau(-p)), N);
    add(kidx(tau(-p)), N, nidx(tau(p)), nidx(tau(p - 1)) - 1);
  }
  hp.blocks = raw;
  // Near set: per row, the columns not covered by a block; always a prefix 1..nend(k).
  std::vector<int64_t> fstart(N + 2, N + 1), covered(N + 2, 0);
  hp.far_count = 0;
  for (const Block& b : hp.blocks) {
    for (int64_t k = b.k0; k <= b.k1; ++k) {
      fstart[k] = std::min(fstart[k], b.n0);
      covered[k] += b.C;
    }
    hp.far_count += b.R * b.C;
  }
  hp.nend.assign(N, 0);
  hp.near_count = 0;
  hp.zmax = 0.0;
  for (int64_t k = 1; k <= N; ++k) {
    int64_t ne = fstart[k] - 1;
    // the far columns of row k must be exactly fstart..N
    if (covered[k] != N - ne) { hp.nend.clear(); return; }
    hp.nend[k - 1] = ne;
    hp.near_count += ne;
    if (ne > 0) hp.zmax = std::max(hp.zmax, hp.r_true[k - 1] * hp.om_true[ne - 1]);
  }
}

void build_columns(HostPlan& hp) {
  const hankel_options& o = hp.opt;
  const int M = hp.M;
  const int U1 = hp.U1, U2 = hp.U2;
  const int nd = 2 * M + U2 - 1;  // delta = u2 - j in [-(2M-1), U2-1]
  std::vector<cplx> G((size_t)U1 * nd * U2, cplx(0.0, 0.0));
  auto at = [&](int u1, int delta, int u2) -> cplx& { return G[((size_t)u1 * nd + (delta + 2 * M - 1)) * U2 + u2]; };
  cplx c[128];
  if (o.task == HANKEL_SCHLOMILCH) {
    hankel_c(o.nu, M, c);
    for (int j = 0; j < 2 * M; ++j) at(0, -j, 0) += c[j];
  } else if (o.task == HANKEL_FOURIER_BESSEL) {
    // Section 5.1: J_nu(r j_{0,n}) ~ sum_u (r b_n)^u sum_lam g_{u,lam} J_lam(r omega~_n) (Eq. 22 rearranged)
    for (int u = 0; u < U2; ++u)
      for (auto& t : neumann_terms(o.nu, hp.K, hp.T, u)) {
        hankel_c(t.first, M, c);
        for (int j = 0; j < 2 * M; ++j) at(0, u - j, u) += t.second * c[j];
      }
  } else {
    // Section 6, Eq. (26): rows perturbed by e_k (outer sum over u1, truncation K, T), then each
    // J_lam(r~_k j_{0,n}) expanded in b_n as in Section 5 (inner sum over u2, truncation K2, T2).
    for (int u1 = 0; u1 < U1; ++u1)
      for (auto& t1 : neumann_terms(0, hp.K, hp.T, u1))
        for (int u2 = 0; u2 < U2; ++u2)
          for (auto& t2 : neumann_terms(t1.first, hp.K2, hp.T2, u2)) {
            hankel_c(t2.first, M, c);
            for (int j = 0; j < 2 * M; ++j) at(u1, u2 - j, u2) += (t1.second * t2.second) * c[j];
          }
  }
  hp.cols.clear();
  for (int u1 = 0; u1 < U1; ++u1)
    for (int d = -(2 * M - 1); d <= U2 - 1; ++d) {
      ColSpec cs;
      cs.u1 = u1;
      cs.delta = d;
      cs.nterm = U2;
      for (int u2 = 0; u2 < kMaxU; ++u2) cs.G[u2] = u2 < U2 ? at(u1, d, u2) : cplx(0.0, 0.0);
      hp.cols.push_back(cs);
    }
}

// Per-block choice of stacked columns. Column l contributes W_l(k) T_l(n) to entry (k, n) of
// a block (times a unimodular chirp), with W_l(k) = rowpert^u1 rowvar^(delta-1/2) and
// |T_l(n)| <= |colpow^u1| omt^(delta-1/2) sum_u2 |G_l[u2]| |beta|^u2. Written as
//   |W_l(k)| = (|rowpert| rowvar)^u1 rowvar^(delta-1/2-u1),
//   |colpow^u1 omt^(delta-1/2)| = (|colpow|/omt)^u1 omt^(delta-1/2+u1),
// each is a slowly varying factor (e_k r~_k and omega_n/omega~_n change little over a
// block) times a power of a monotone node value, so the block maxima of the slowly varying
// factors (found by a scan) and of the powers (at the block's end nodes) bound max|W_l| and
// max|T_l| closely, and A_l = max|W_l| max|T_l| bounds the column's share of every entry.
// The truncations K, T, K2, T2 and M are fixed for the worst block (Sections 5.2, 6.1); far
// from the near field the perturbations e_k omega_n and r b_n are tiny and many columns
// contribute less than eps. A block drops its columns in increasing order of A_l while their
// sum stays within its share of a budget of kDropFrac * eps per entry (split evenly between
// the blocks that meet in one row); every entry then moves by at most that sum, so
// |f_k - f'_k| <= kDropFrac * eps * sum_n |c_n|. With kDropFrac = 1 an entry keeps the
// expansion's own eps (the truncations above) plus at most eps from the dropped columns,
// and f stays within O(eps ||c||_1) (Sections 5.2, 6.1).
constexpr double kDropFrac = 1.0;
// Blocks that may meet in one row while a block's budget is kDropFrac * eps / kRowBlocks.
constexpr int kRowBlocks = 16;

// Range maxima of a node sequence over index ranges, from maxima of chunks of 1024.
struct RangeMax {
  std::vector<double> v, chunk;
  static constexpr int64_t kChunk = 1024;
  explicit RangeMax(std::vector<double> x) : v(std::move(x)) {
    chunk.assign((v.size() + kChunk - 1) / kChunk, -INFINITY);
    for (size_t i = 0; i < v.size(); ++i) chunk[i / kChunk] = std::max(chunk[i / kChunk], v[i]);
  }
  double max(int64_t a, int64_t b) const {  // 0-based inclusive
    double m = -INFINITY;
    while (a <= b && a % kChunk) m = std::max(m, v[a++]);
    while (a + kChunk - 1 <= b) m = std::max(m, chunk[a / kChunk]), a += kChunk;
    while (a <= b) m = std::max(m, v[a++]);
    return m;
  }
};

struct NodeRanges {
  RangeMax rp, rv, nrv, cp, om, nom, bt;  // maxima of |e_k| r~_k, rowvar, -rowvar, colpow/omt, omt, -omt, |beta|
  explicit NodeRanges(const HostPlan& hp)
      : rp(map(hp.rowpert, hp.rowvar, [](double e, double r) { return std::fabs(e) * r; })),
        rv(hp.rowvar),
        nrv(map(hp.rowvar, hp.rowvar, [](double r, double) { return -r; })),
        cp(map(hp.colpow, hp.omt, [](double c, double w) { return std::fabs(c) / w; })),
        om(hp.omt),
        nom(map(hp.omt, hp.omt, [](double w, double) { return -w; })),
        bt(map(hp.betan, hp.betan, [](double b, double) { return std::fabs(b); })) {}
  template <class Fn>
  static std::vector<double> map(const std::vector<double>& a, const std::vector<double>& b, Fn fn) {
    std::vector<double> o(a.size());
    for (size_t i = 0; i < a.size(); ++i) o[i] = fn(a[i], b[i]);
    return o;
  }
};

void block_columns(const HostPlan& hp, const NodeRanges& nr, Block& b, double budget) {
  const int ncols = (int)hp.cols.size();
  b.lcols.clear();
  b.dropped = 0.0;
  if (hp.opt.flags & HANKEL_FLAG_ALL_COLUMNS) {
    for (int l = 0; l < ncols; ++l) b.lcols.push_back(l);
    return;
  }
  const double rp = nr.rp.max(b.k0 - 1, b.k1 - 1), rv0 = -nr.nrv.max(b.k0 - 1, b.k1 - 1),
               rv1 = nr.rv.max(b.k0 - 1, b.k1 - 1);
  const double cp = nr.cp.max(b.n0 - 1, b.n1 - 1), om0 = -nr.nom.max(b.n0 - 1, b.n1 - 1),
               om1 = nr.om.max(b.n0 - 1, b.n1 - 1), bt = nr.bt.max(b.n0 - 1, b.n1 - 1);
  auto pw = [](double x, double e) { return std::pow(x, e); };
  std::vector<std::pair<double, int>> bound(ncols);
  for (int l = 0; l < ncols; ++l) {
    const ColSpec& cs = hp.cols[l];
    const double er = cs.delta - 0.5 - cs.u1, ec = cs.delta - 0.5 + cs.u1;
    double poly = 0.0, bp = 1.0;
    for (int u = 0; u < cs.nterm; ++u, bp *= bt) poly += std::abs(cs.G[u]) * bp;
    double a = std::max(pw(rv0, er), pw(rv1, er)) * std::max(pw(om0, ec), pw(om1, ec)) * poly;
    if (cs.u1) a *= pw(rp, cs.u1) * pw(cp, cs.u1);
    bound[l] = {std::isfinite(a) ? a : INFINITY, l};
  }
  std::sort(bound.begin(), bound.end());
  std::vector<char> keep(ncols, 1);
  double sum = 0.0;
  for (const auto& x : bound) {
    if (sum + x.first > budget) break;
    sum += x.first;
    keep[x.second] = 0;
  }
  b.dropped = sum;
  for (int l = 0; l < ncols; ++l)
    if (keep[l]) b.lcols.push_back(l);
  if (b.lcols.empty()) b.lcols.push_back(bound.back().second);  // every block keeps one column
}

// ---------------------------------------------------------------------------
// Low-rank form of a block (beyond the paper). Within a far block the kernel
// K(k, n) = sum_l rowfun_l(k) colfun_l(n) -- the smooth envelope that multiplies the chirp
// exp(i theta~_kn) -- is an analytic function of log k and log n of small numerical rank: its
// singular values fall by orders of magnitude per term, because the Hankel tail and the
// perturbation terms are smooth in z = r omega. It is sampled on a P x P Chebyshev grid in
// (log k, log n), using the node functions at real k and n (their closed forms, and b(n) from
// the root-offset fixed point), and factored there by cross approximation with complete
// pivoting (Gaussian elimination stopped when the largest residual is below tol):
// K_grid ~ sum_a u_a v_a^T. U_a and V_a interpolate u_a and v_a at any k and n. The form is
// kept when it is exact to kLowRankFrac * eps on a validation set of entries of the block
// (its corners, edges and pseudo-random entries, against the expansion at the integer nodes)
// and has fewer terms than the block's kept columns; the block then runs rank transforms per
// vector instead of lcols.size(). Entries carry at most eps (expansion) + eps (dropped
// columns) + kLowRankFrac * eps (low-rank form).
// ---------------------------------------------------------------------------
constexpr double kLowRankFrac = 0.5;
constexpr int kChebP0 = 32, kChebPMax = 64;

void node_row(const HostPlan& hp, double k, double* rv, double* rp) {
  const int64_t N = hp.opt.N;
  if (hp.opt.task == HANKEL_DHT) {
    const double bN1 = hp.b[N], jN1 = (N + 0.75) * kPi + bN1;
    *rv = (4.0 * k - 1.0) / (4.0 * N + 3.0);
    *rp = (root_offset_large(k) * (N + 0.75) - bN1 * (k - 0.25)) / (jN1 * (N + 0.75));
  } else {
    *rv = hp.opt.grid == HANKEL_GRID_UNIT ? (k - 1.0) / (double)(N - 1) : k / (double)N;
    *rp = 0.0;
  }
}

void node_col(const HostPlan& hp, double n, double* om, double* bt, double* cp) {
  if (hp.opt.task == HANKEL_SCHLOMILCH) {
    *om = (n + hp.opt.gamma) * kPi;
    *bt = 0.0;
    *cp = 1.0;
  } else {
    const double w = (n - 0.25) * kPi, bn = root_offset_large(n);
    *om = w;
    *bt = bn / w;
    *cp = hp.opt.task == HANKEL_DHT ? w + bn : 1.0;
  }
}

cplx kernel_sum(const HostPlan& hp, const std::vector<int>& lcols, double rv, double rp, double om, double bt,
                double cp) {
  cplx acc(0.0, 0.0);
  for (int l : lcols) {
    const ColSpec& cs = hp.cols[l];
    cplx poly(0.0, 0.0);
    for (int u = cs.nterm - 1; u >= 0; --u) poly = poly * bt + cs.G[u];
    const double row = std::pow(rv, cs.delta - 0.5) * (cs.u1 ? std::pow(rp, cs.u1) : 1.0);
    const double col = std::pow(om, cs.delta - 0.5) * (cs.u1 ? std::pow(cp, cs.u1) : 1.0);
    acc += row * col * poly;
  }
  return acc;
}

double cheb_node(int i, int P) { return std::cos(kPi * (i + 0.5) / P); }

bool try_lowrank(const HostPlan& hp, Block& b, int P, double tol) {
  const int nl = (int)b.lcols.size();
  const double lk0 = std::log((double)b.k0), lk1 = std::log((double)b.k1);
  const double ln0 = std::log((double)b.n0), ln1 = std::log((double)b.n1);
  std::vector<double> rv(P), rp(P), om(P), bt(P), cp(P);
  for (int i = 0; i < P; ++i) {
    const double x = cheb_node(i, P);
    node_row(hp, std::exp(0.5 * (lk0 + lk1) + 0.5 * (lk1 - lk0) * x), &rv[i], &rp[i]);
    node_col(hp, std::exp(0.5 * (ln0 + ln1) + 0.5 * (ln1 - ln0) * x), &om[i], &bt[i], &cp[i]);
  }
  std::vector<cplx> R((size_t)P * P);
  for (int i = 0; i < P; ++i)
    for (int j = 0; j < P; ++j) R[(size_t)i * P + j] = kernel_sum(hp, b.lcols, rv[i], rp[i], om[j], bt[j], cp[j]);
  // cross approximation with complete pivoting
  std::vector<cplx> u, v;
  int rank = 0;
  for (;;) {
    size_t best = 0;
    double m = -1.0;
    for (size_t e = 0; e < R.size(); ++e)
      if (std::abs(R[e]) > m) { m = std::abs(R[e]); best = e; }
    if (m <= tol) break;
    if (rank + 1 >= nl) return false;  // no fewer terms than the kept columns
    const int is = (int)(best / P), js = (int)(best % P);
    const cplx piv = R[best];
    std::vector<cplx> ua(P), va(P);
    for (int i = 0; i < P; ++i) ua[i] = R[(size_t)i * P + js] / piv;
    for (int j = 0; j < P; ++j) va[j] = R[(size_t)is * P + j];
    for (int i = 0; i < P; ++i)
      for (int j = 0; j < P; ++j) R[(size_t)i * P + j] -= ua[i] * va[j];
    u.insert(u.end(), ua.begin(), ua.end());
    v.insert(v.end(), va.begin(), va.end());
    ++rank;
  }
  if (rank == 0) return false;
  // validation against the expansion at the integer nodes
  auto approx = [&](int64_t k, int64_t n) {
    const double x = log_coord((double)k, b.k0, b.k1), y = log_coord((double)n, b.n0, b.n1);
    cplx acc(0.0, 0.0);
    for (int a = 0; a < rank; ++a) acc += cheb_interp(&u[(size_t)a * P], P, x) * cheb_interp(&v[(size_t)a * P], P, y);
    return acc;
  };
  auto exact = [&](int64_t k, int64_t n) {
    return kernel_sum(hp, b.lcols, hp.rowvar[k - 1], hp.rowpert[k - 1], hp.omt[n - 1], hp.betan[n - 1],
                      hp.colpow[n - 1]);
  };
  std::vector<std::pair<int64_t, int64_t>> pts;
  const int64_t ks[3] = {b.k0, (b.k0 + b.k1) / 2, b.k1}, ns[3] = {b.n0, (b.n0 + b.n1) / 2, b.n1};
  for (int64_t k : ks)
    for (int64_t n : ns) pts.push_back({k, n});
  uint64_t st = 0x9e3779b97f4a7c15ull ^ (uint64_t)(b.k0 * 1315423911u + b.n0);
  auto rnd = [&]() {
    st = st * 6364136223846793005ull + 1442695040888963407ull;
    return (double)(st >> 11) * (1.0 / 9007199254740992.0);
  };
  for (int t = 0; t < 1536; ++t) {
    double fk = rnd(), fn = rnd();
    if (t & 1) {  // log-uniform: dense near the block's small-z corner
      fk = std::exp(lk0 + (lk1 - lk0) * fk);
      fn = std::exp(ln0 + (ln1 - ln0) * fn);
    } else {
      fk = b.k0 + (b.k1 - b.k0) * fk;
      fn = b.n0 + (b.n1 - b.n0) * fn;
    }
    pts.push_back({std::min(b.k1, std::max(b.k0, (int64_t)std::llround(fk))),
                   std::min(b.n1, std::max(b.n0, (int64_t)std::llround(fn)))});
  }
  double err = 0.0;
  for (const auto& q : pts) err = std::max(err, std::abs(approx(q.first, q.second) - exact(q.first, q.second)));
  if (err > kLowRankFrac * hp.opt.eps) return false;
  b.rank = rank;
  b.P = P;
  b.ucheb = u;
  b.vcheb = v;
  b.lowrank_err = err;
  return true;
}

// Terms of the block's low-rank form on a coarse grid (no validation): the cost estimate of
// the subdivision. Returns the kept columns when the form would not be shorter.
int estimate_rank(const HostPlan& hp, const Block& b) {
  const int nl = (int)b.lcols.size();
  if (b.R < 8 || b.C < 8 || nl < 3) return nl;
  constexpr int P = 24;
  const double lk0 = std::log((double)b.k0), lk1 = std::log((double)b.k1);
  const double ln0 = std::log((double)b.n0), ln1 = std::log((double)b.n1);
  double rv[P], rp[P], om[P], bt[P], cp[P];
  for (int i = 0; i < P; ++i) {
    const double x = cheb_node(i, P);
    node_row(hp, std::exp(0.5 * (lk0 + lk1) + 0.5 * (lk1 - lk0) * x), &rv[i], &rp[i]);
    node_col(hp, std::exp(0.5 * (ln0 + ln1) + 0.5 * (ln1 - ln0) * x), &om[i], &bt[i], &cp[i]);
  }
  std::vector<cplx> R((size_t)P * P);
  for (int i = 0; i < P; ++i)
    for (int j = 0; j < P; ++j) R[(size_t)i * P + j] = kernel_sum(hp, b.lcols, rv[i], rp[i], om[j], bt[j], cp[j]);
  const double tol = 0.15 * hp.opt.eps;
  for (int rank = 0; rank < nl; ++rank) {
    size_t best = 0;
    double m = -1.0;
    for (size_t e = 0; e < R.size(); ++e)
      if (std::abs(R[e]) > m) { m = std::abs(R[e]); best = e; }
    if (m <= tol) return std::max(rank, 1);
    const int is = (int)(best / P), js = (int)(best % P);
    const cplx piv = R[best];
    for (int i = 0; i < P; ++i) {
      const cplx ui = R[(size_t)i * P + js] / piv;
      for (int j = 0; j < P; ++j) R[(size_t)i * P + j] -= ui * R[(size_t)is * P + j] * (i == is ? 0.0 : 1.0);
    }
    for (int j = 0; j < P; ++j) R[(size_t)is * P + j] = 0.0;
  }
  return nl;
}

void compress_blocks(HostPlan& hp) {
  for (Block& b : hp.blocks) {
    b.rank = 0;
    if (hp.opt.flags & (HANKEL_FLAG_NO_LOWRANK | HANKEL_FLAG_ALL_COLUMNS)) continue;
    if (b.R < 8 || b.C < 8 || b.lcols.size() < 3) continue;
    double tol = 0.15 * hp.opt.eps;
    for (int P = kChebP0; P <= kChebPMax; P += 16, tol *= 0.25)
      if (try_lowrank(hp, b, P, tol)) break;
  }
}

// Precision of each transform of a block. The rounding error of a term computed in precision
// u grows with u times the size of its contribution, max_k |U_l(k)| max_n |V_l(n)| (per unit of
// ||c||_1). Each factor is a polynomial interpolant p = sum_j a_j T_j in the Chebyshev
// variable, so max |p| <= sum_j |a_j| bounds it above, and the largest value at the Chebyshev
// points bounds it below. In MIXED plans of FP64 or DF64 precision a term takes the lowest
// precision whose upper bound stays within
//   max(u_plan / 4, eps / 200) x (the largest grid size of the block's terms),
// i.e. a quarter of the rounding bound of the block's leading term in the plan precision, or
// a two-hundredth of the requested accuracy; the terms of a low-rank form shrink geometrically
// (about 1e-4 per term for the DHT), so only the leading ones keep the plan precision. Direct
// blocks (no low-rank form) and FP32 plans keep one precision for every transform.
constexpr double kUnitFP64 = 1.1102230246251565e-16;  // 2^-53
constexpr double kUnitDF64 = 1.4210854715202004e-14;  // 2^-46: double-float with sloppy sums
constexpr double kUnitFP32 = 5.9604644775390625e-08;  // 2^-24

void assign_term_precision(HostPlan& hp) {
  const int base = hp.fp32 ? kTermFP32 : hp.df64 ? kTermDF64 : kTermFP64;
  const bool mixed =
      hp.opt.precision == HANKEL_PREC_MIXED && !hp.fp32 && !(hp.opt.flags & HANKEL_FLAG_UNIFORM_TERMS);
  for (Block& b : hp.blocks) {
    const int nl = b.rank ? b.rank : (int)b.lcols.size();
    b.tprec.assign((size_t)nl, (int8_t)base);
    if (!mixed || !b.rank) continue;
    std::vector<double> lo(nl), hi(nl);
    // sum_j |a_j| of the interpolant through values f_i at the points cos(pi (i + 1/2) / P):
    // a_j = (2 - [j = 0]) / P sum_i f_i cos(pi j (i + 1/2) / P)
    auto coef_sum = [&](const std::vector<cplx>& vals, int li) {
      double tot = 0.0;
      for (int j = 0; j < b.P; ++j) {
        cplx aj(0.0, 0.0);
        for (int i = 0; i < b.P; ++i) aj += vals[(size_t)li * b.P + i] * std::cos(kPi * j * (i + 0.5) / b.P);
        tot += std::abs(aj) * (j == 0 ? 1.0 : 2.0) / b.P;
      }
      return tot;
    };
    double A = 0.0;
    for (int li = 0; li < nl; ++li) {
      double mu = 0.0, mv = 0.0;
      for (int j = 0; j < b.P; ++j) {
        mu = std::max(mu, std::abs(b.ucheb[(size_t)li * b.P + j]));
        mv = std::max(mv, std::abs(b.vcheb[(size_t)li * b.P + j]));
      }
      lo[li] = mu * mv;
      // slightly above the coefficient sums, for their own rounding
      hi[li] = (1.0 + 1e-12) * coef_sum(b.ucheb, li) * coef_sum(b.vcheb, li);
      A = std::max(A, lo[li]);
    }
    const double ub = base == kTermFP64 ? kUnitFP64 : kUnitDF64;
    const double tau = std::max(0.25 * ub, hp.opt.eps / 200.0) * A;
    for (int li = 0; li < nl; ++li) {
      int p = base;
      if (base == kTermFP64 && kUnitDF64 * hi[li] <= tau) p = kTermDF64;
      if (kUnitFP32 * hi[li] <= tau) p = kTermFP32;
      b.tprec[li] = (int8_t)p;
    }
  }
}

// Subdivision of the far blocks (an addition to the partition of Eq. 19). The blocks of
// Eq. (19) touch the near field at one corner, where z~ ~ s and every stacked column is
// needed, but stretch to z~ ~ N: away from that corner the Hankel tail and the perturbation
// terms shrink and far fewer columns pass the drop bound. A block is cut in two, across its
// rows or its columns at one of a few geometric points, when the cut lowers the estimated
// work (transforms x column_cost, plus a fixed cost per block execution spread over max_nrhs
// vectors; transforms = the low-rank form's terms on a coarse grid, or the kept columns when
// low-rank forms are off); the halves are refined again. The union of the blocks, hence the
// near set, does not change.
constexpr double kBlockLaunchOps = 1e7;  // FP64-operation equivalent of the launches of one block
constexpr int64_t kMinSide = 64;

double block_work(const HostPlan& hp, const Block& b) {
  const bool lowrank = !(hp.opt.flags & (HANKEL_FLAG_NO_LOWRANK | HANKEL_FLAG_ALL_COLUMNS));
  const int terms = lowrank ? estimate_rank(hp, b) : (int)b.lcols.size();
  return (double)terms * column_cost(hp, b) + kBlockLaunchOps / hp.opt.max_nrhs;
}

void refine(const HostPlan& hp, const NodeRanges& nr, Block b, double budget, int depth, std::vector<Block>& out) {
  block_columns(hp, nr, b, budget);
  const double w0 = block_work(hp, b);
  double best = 0.97 * w0;
  Block bl1, bl2;
  bool found = false;
  auto consider = [&](Block c1, Block c2) {
    block_columns(hp, nr, c1, budget);
    block_columns(hp, nr, c2, budget);
    const double w = block_work(hp, c1) + block_work(hp, c2);
    if (w < best) {
      best = w;
      bl1 = c1;
      bl2 = c2;
      found = true;
    }
  };
  if (depth < 24) {
    for (double t : {0.25, 0.5, 0.75}) {
      if (b.R >= 2 * kMinSide) {
        int64_t km = (int64_t)std::llround(std::exp((1 - t) * std::log((double)b.k0) + t * std::log((double)b.k1)));
        km = std::min(std::max(km, b.k0 + kMinSide), b.k1 - kMinSide + 1);
        consider(make_block(hp, b.k0, km - 1, b.n0, b.n1), make_block(hp, km, b.k1, b.n0, b.n1));
      }
      if (b.C >= 2 * kMinSide) {
        int64_t nm = (int64_t)std::llround(std::exp((1 - t) * std::log((double)b.n0) + t * std::log((double)b.n1)));
        nm = std::min(std::max(nm, b.n0 + kMinSide), b.n1 - kMinSide + 1);
        consider(make_block(hp, b.k0, b.k1, b.n0, nm - 1), make_block(hp, b.k0, b.k1, nm, b.n1));
      }
    }
  }
  if (!found) {
    out.push_back(b);
    return;
  }
  refine(hp, nr, bl1, budget, depth + 1, out);
  refine(hp, nr, bl2, budget, depth + 1, out);
}

void select_columns(HostPlan& hp) {
  const int64_t N = hp.opt.N;
  NodeRanges nr(hp);
  double budget = kDropFrac * hp.opt.eps / kRowBlocks;
  const bool subdivide = !(hp.opt.flags & (HANKEL_FLAG_NO_REFINE | HANKEL_FLAG_ALL_COLUMNS));
  if (subdivide) {
    std::vector<Block> out;
    for (const Block& b : hp.blocks) refine(hp, nr, b, budget, 0, out);
    hp.blocks = out;
  }
  // blocks meeting in one row; the budget must cover all of them
  std::vector<int> per_row(N + 2, 0);
  for (const Block& b : hp.blocks) {
    per_row[b.k0] += 1;
    per_row[b.k1 + 1] -= 1;
  }
  int maxrow = 1, run = 0;
  for (int64_t k = 1; k <= N; ++k) maxrow = std::max(maxrow, run += per_row[k]);
  budget = kDropFrac * hp.opt.eps / std::max(maxrow, subdivide ? kRowBlocks : 1);
  for (Block& b : hp.blocks) block_columns(hp, nr, b, budget);
}

// Taylor polynomials of J_nu about z_c = (i + 1/2)/sub on [i/sub, (i+1)/sub). The coefficients
// follow from the Neumann addition formula (Eq. 8) with each J_s(delta) expanded in its Taylor
// series (Eq. 6) -- the same rearrangement as Section 5.1 with K and T unbounded:
// t_d = 2^{-d} sum_t (-1)^t / (t!(d-t)!) [J_{nu-s}(z_c) + (-1)^s J_{nu+s}(z_c)], s = d-2t,
// the s = 0 term counted once. Every derivative of J_nu is at most 1 in size, so degree d on
// half-width h = 1/(2 sub) errs by at most h^{d+1}/(d+1)!; the degree is the smallest that
// keeps this below eps/100 (at most kJTabDegMax).
void build_jtable(HostPlan& hp) {
  const int nu = hp.opt.nu;
  const int sub = kJTabSub;
  const double h = 0.5 / sub;
  int deg = 2;
  for (double b = h * h * h / 6.0; deg < kJTabDegMax && b > 0.01 * hp.opt.eps; b *= h / (deg + 2)) ++deg;
  hp.jt_deg = deg;
  hp.jt_sub = sub;
  hp.jt_n = (int64_t)std::ceil(hp.zmax * sub) + 2;
  hp.jtab.assign((size_t)hp.jt_n * (deg + 1), 0.0);
  hp.jtabq.assign((size_t)hp.jt_n * (deg + 1), 0);
  std::vector<DD> J;
  const int L = nu + deg + 1;
  for (int64_t i = 0; i < hp.jt_n; ++i) {
    const DD zc = dd_scale(ddv(i + 0.5), 1.0 / sub);  // sub is a power of two
    miller_all(zc, L, J);
    auto jl = [&](int lam) -> DD {  // J_lam for any integer lam (DLMF 10.4.1)
      if (lam >= 0) return J[lam];
      return ((-lam) & 1) ? dd_neg(J[-lam]) : J[-lam];
    };
    for (int d = 0; d <= deg; ++d) {
      DD acc = ddv(0.0);
      for (int t = 0; 2 * t <= d; ++t) {
        int s = d - 2 * t;
        double coef = std::ldexp((t & 1) ? -1.0 : 1.0, -d) / (factorial(t) * factorial(d - t));
        DD term = (s == 0) ? jl(nu) : dd_add(jl(nu - s), (s & 1) ? dd_neg(jl(nu + s)) : jl(nu + s));
        acc = dd_add(acc, dd_mul(ddv(coef), term));
      }
      hp.jtab[(size_t)i * (deg + 1) + d] = acc.h + acc.l;
      // |t_d sub^-d| < 2: the scaled value fits a signed 64-bit integer; x - rint(x) is exact
      const double x = std::ldexp(acc.h, 62 - kJTabLog * d), y = std::ldexp(acc.l, 62 - kJTabLog * d);
      hp.jtabq[(size_t)i * (deg + 1) + d] = std::llrint(x) + std::llrint((x - std::rint(x)) + y);
    }
  }
}

}  // namespace

int build_host_plan(const hankel_options& opt, HostPlan& hp) {
  int st = choose_params(opt, hp);
  if (st != HANKEL_OK) return st;
  build_nodes(hp);
  build_partition(hp);
  if (hp.nend.empty()) return HANKEL_EINVAL;  // partition invariant violated
  build_columns(hp);
  select_columns(hp);
  compress_blocks(hp);
  assign_term_precision(hp);
  build_jtable(hp);
  return HANKEL_OK;
}

double table_j(const HostPlan& hp, double z) {
  int64_t i = (int64_t)(z * hp.jt_sub);
  if (i < 0) i = 0;
  if (i >= hp.jt_n) i = hp.jt_n - 1;
  double d = z - ((double)i + 0.5) / hp.jt_sub;
  const double* t = &hp.jtab[(size_t)i * (hp.jt_deg + 1)];
  double v = t[hp.jt_deg];
  for (int j = hp.jt_deg - 1; j >= 0; --j) v = v * d + t[j];
  return v;
}

// The fixed-point evaluation FP64 near fields use on the device, restated on the host: the
// interval i = floor(z sub) and U = (z sub - i - 1/2) 2^64 from the bits of z (z >= 0), Horner's
// rule in Q62 with the floor of each signed 128-bit product over 2^64, one rounding to double.
double table_j_q62(const HostPlan& hp, double z) {
  uint64_t bits;
  memcpy(&bits, &z, sizeof bits);
  const int E = (int)(bits >> 52) & 0x7ff;
  const uint64_t M = (bits & 0xfffffffffffffULL) | (E ? (1ULL << 52) : 0ULL);
  const int sh = 52 + 1023 - kJTabLog - E;
  int64_t i;
  uint64_t F;
  if (sh <= 0) {
    i = hp.jt_n;
    F = 0;
  } else if (sh <= 52) {
    i = (int64_t)(M >> sh);
    F = M << (64 - sh);
  } else {
    i = 0;
    F = sh - 53 < 64 ? (M << 11) >> (sh - 53) : 0ULL;
  }
  if (i >= hp.jt_n) {
    i = hp.jt_n - 1;
    F = ~0ULL;
  }
  const int64_t U = (int64_t)(F ^ (1ULL << 63));
  const long long* t = &hp.jtabq[(size_t)i * (hp.jt_deg + 1)];
  int64_t v = t[hp.jt_deg];
  for (int j = hp.jt_deg - 1; j >= 0; --j) v = (int64_t)(((__int128)v * U) >> 64) + t[j];
  return std::ldexp((double)v, -62);
}

// The far-field representation of entry (k, n) summed over the given stacked columns:
// Re[ exp(i theta~_kn) sum_l rowfun_l(k) colfun_l(n) ].
double expansion_entry(const HostPlan& hp, int64_t k, int64_t n, const std::vector<int>* lcols) {
  // exp(i theta~_kn), theta~ = pi U_k V_n / E reduced exactly
  __int128 U = (__int128)hp.Ua * k + hp.Ub, V = (__int128)hp.Va * n + hp.Vb;
  __int128 num = (U * V) % ((__int128)2 * hp.E);
  double s, c;
  sincospi_ratio((int64_t)num, hp.E, &s, &c);
  cplx ph(c, s), acc(0.0, 0.0);
  double rv = hp.rowvar[k - 1], rp = hp.rowpert[k - 1];
  double w = hp.omt[n - 1], bt = hp.betan[n - 1], cp = hp.colpow[n - 1];
  const size_t count = lcols ? lcols->size() : hp.cols.size();
  for (size_t j = 0; j < count; ++j) {
    const ColSpec& cs = hp.cols[lcols ? (*lcols)[j] : (int)j];
    cplx poly(0.0, 0.0);
    for (int u2 = cs.nterm - 1; u2 >= 0; --u2) poly = poly * bt + cs.G[u2];
    double row = std::pow(rv, cs.delta - 0.5) * (cs.u1 ? std::pow(rp, cs.u1) : 1.0);
    double col = std::pow(w, cs.delta - 0.5) * (cs.u1 ? std::pow(cp, cs.u1) : 1.0);
    acc += row * col * poly;
  }
  return (ph * acc).real();
}

double log_coord(double k, int64_t k0, int64_t k1) {
  if (k1 <= k0) return 0.0;
  const double l0 = std::log((double)k0), l1 = std::log((double)k1);
  return (2.0 * std::log(k) - l0 - l1) / (l1 - l0);
}

cplx cheb_interp(const cplx* vals, int P, double x) {
  cplx num(0.0, 0.0);
  double den = 0.0;
  for (int i = 0; i < P; ++i) {
    const double d = x - cheb_node(i, P);
    if (d == 0.0) return vals[i];
    const double w = ((i & 1) ? -1.0 : 1.0) * std::sin(kPi * (i + 0.5) / P) / d;
    num += w * vals[i];
    den += w;
  }
  return num / den;
}

double host_entry(const HostPlan& hp, int64_t k, int64_t n, int* is_far) {
  *is_far = 0;
  if (n > hp.nend[k - 1]) {
    *is_far = 1;
    const Block* blk = nullptr;
    for (const Block& b : hp.blocks)
      if (k >= b.k0 && k <= b.k1 && n >= b.n0 && n <= b.n1) blk = &b;
    if (blk->rank == 0) return expansion_entry(hp, k, n, &blk->lcols);
    // low-rank form: Re[exp(i theta~_kn) sum_a U_a(k) V_a(n)]
    __int128 U = (__int128)hp.Ua * k + hp.Ub, V = (__int128)hp.Va * n + hp.Vb;
    __int128 num = (U * V) % ((__int128)2 * hp.E);
    double s, c;
    sincospi_ratio((int64_t)num, hp.E, &s, &c);
    const double x = log_coord((double)k, blk->k0, blk->k1), y = log_coord((double)n, blk->n0, blk->n1);
    cplx acc(0.0, 0.0);
    for (int a = 0; a < blk->rank; ++a)
      acc += cheb_interp(&blk->ucheb[(size_t)a * blk->P], blk->P, x) *
             cheb_interp(&blk->vcheb[(size_t)a * blk->P], blk->P, y);
    return (cplx(c, s) * acc).real();
  }
  // FP64 plans evaluate near-field J in fixed point on the device; FP32 and DF64 plans (whose
  // small batches use their own float tables) are represented by the FP64 table
  const double z = hp.r_true[k - 1] * hp.om_true[n - 1];
  return (hp.fp32 || hp.df64) ? table_j(hp, z) : table_j_q62(hp, z);
}

}  // namespace hk
