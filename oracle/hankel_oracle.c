/*
 * TEST INFRASTRUCTURE -- NOT PART OF THE PRODUCT PATH.
 *
 * A plain, slow, CPU-only oracle for the discrete Hankel-type sums of the
 * paper (Townsend, "A fast analysis-based discrete Hankel transform using
 * asymptotic expansions", arXiv:1501.01652), Eq. (2):
 *
 *     f_k = sum_{n=1}^{N} c_n J_nu(r_k omega_n),   1 <= k <= N.
 *
 * It evaluates that definition directly, O(N^2), in FP64 with Kahan
 * summation over n, using its own Bessel evaluator. It shares no code with
 * the CUDA library. Only the test-suite, the smoke check and the benchmark's
 * CPU-baseline leg may load it.
 *
 * Tasks (Section 1, items (1)-(3)):
 *   task 0  Schlomilch expansion (Section 4, Eq. 11): omega_n = (n+gamma)pi,
 *           integer gamma (Remark 4.1 shift).
 *   task 1  Fourier-Bessel expansion (Section 5, Eq. 20): omega_n = j_{0,n}.
 *   task 2  Discrete Hankel transform of order 0 (Section 6, Eq. 25):
 *           r_k = j_{0,k}/j_{0,N+1}, omega_n = j_{0,n}, nu = 0.
 * Sample points for tasks 0 and 1: grid 0 gives r_k = (k-1)/(N-1)
 * (so that r spans [0,1] as in Eq. 3's DCT-I nodes), grid 1 gives the
 * paper's r_k = k/N (Sections 4 and 5).
 *
 * Every argument is represented as z = pi*P/Q + delta with integers P, Q
 * (the exact equispaced part, Lemma 3.2's "perturbed equally-spaced grid")
 * and a small FP64 perturbation delta. For large z the phase
 * mu = z - (2nu+1)pi/4 of the Hankel expansion (Eq. 4) is then reduced
 * exactly in integer arithmetic, so no digits are lost at z ~ 1e7.
 *
 * Bessel evaluator (Section 2.1 lists the three regimes):
 *   z <= 2       power series, Eq. (6) (DLMF 10.2.2)
 *   2 < z < 25   Miller's backward recurrence (DLMF 3.6(vi)) normalised by
 *                J_0 + 2 sum_{k>=1} J_{2k} = 1 (DLMF 10.12.4)
 *   z >= 25      Hankel asymptotic expansion, Eq. (4), summed until the
 *                terms stop decreasing (DLMF 10.17(iii)); if the smallest
 *                term is not below 1e-17 (large order), Miller instead
 *
 * Nodes (Lemma 3.2): j_{0,n} = (n-1/4)pi + b_n with b_n kept as its own
 * FP64 number. b_n starts from McMahon's expansion (DLMF 10.21.19) and is
 * refined by Newton's method on J_0 with the argument formed as
 * pi*(4n-1)/4 + b, never as a rounded sum (in double-double for the few
 * zeros below 30, where the FP64 Miller recurrence limits the accuracy).
 *
 * A second, independent implementation in double-double arithmetic
 * (nodes by Newton, J by Miller's recurrence for every z, plain summation)
 * serves as a brute-force cross-check for N <= 64.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define ORC_TASK_SCHLOMILCH 0
#define ORC_TASK_FOURIER_BESSEL 1
#define ORC_TASK_DHT 2

static const double ORC_PI = 3.14159265358979323846;

/* ------------------------------------------------------------------ */
/* J_nu(z) in FP64                                                     */
/* ------------------------------------------------------------------ */

/* Eq. (6): J_nu(z) = sum_t (-1)^t (z/2)^(2t+nu) / (t! (t+nu)!), nu >= 0. */
static double orc_series(int nu, double z) {
  double half = 0.5 * z;
  double term = 1.0;
  for (int i = 1; i <= nu; ++i) term *= half / i;
  double sum = term;
  for (int t = 1; t < 200; ++t) {
    term *= -(half * half) / ((double)t * (double)(t + nu));
    sum += term;
    if (fabs(term) <= 1e-18 * fabs(sum)) break;
  }
  return sum;
}

/* Miller's backward recurrence J_{k-1} = (2k/z) J_k - J_{k+1}, started far
 * above max(nu, z) and normalised with J_0 + 2 sum J_{2k} = 1. nu >= 0. */
static double orc_miller(int nu, double z) {
  int start = (int)z + 60 + nu;
  if (start & 1) start += 1;
  double jp1 = 0.0, j = 1e-30, norm = 0.0, jnu = 0.0;
  for (int k = start; k >= 1; --k) {
    /* here j = J_k (unnormalised), jp1 = J_{k+1} */
    if (k == nu) jnu = j;
    if ((k & 1) == 0) norm += 2.0 * j;
    double jm1 = (2.0 * k / z) * j - jp1;
    jp1 = j;
    j = jm1;
    if (fabs(j) > 1e250) { /* rescale everything tracked so far */
      j *= 1e-250; jp1 *= 1e-250; norm *= 1e-250; jnu *= 1e-250;
    }
  }
  /* now j = J_0 */
  if (nu == 0) jnu = j;
  norm += j;
  return jnu / norm;
}

/* Eq. (4) summed until its terms stop decreasing. The coefficients are
 * a_m(nu) = prod_{i=1}^m (4nu^2-(2i-1)^2) / (m! 8^m). *ok is cleared when the
 * smallest term is not below 1e-17, i.e. z is too small for this order. */
static double orc_hankel_sum(int nu, double z, double cos_mu, double sin_mu, int* ok) {
  double mu4 = 4.0 * (double)nu * (double)nu;
  double a = 1.0;        /* a_m(nu) / z^m */
  double p = 0.0, q = 0.0;
  double prev = INFINITY;
  *ok = 0;
  for (int m = 0; m < 400; ++m) {
    double mag = fabs(a);
    if (m > 0 && (mag > prev || mag < 1e-19)) { *ok = (mag < 1e-17 || prev < 1e-17); break; } /* smallest term reached */
    prev = mag;
    /* term m contributes (-1)^(m/2) to P for even m, (-1)^((m-1)/2) to Q for odd m */
    int r = m & 3;
    if (r == 0) p += a; else if (r == 1) q += a; else if (r == 2) p -= a; else q -= a;
    double f = (mu4 - (2.0 * m + 1.0) * (2.0 * m + 1.0)) / (8.0 * (m + 1.0));
    a *= f / z;
  }
  return sqrt(2.0 / (ORC_PI * z)) * (cos_mu * p - sin_mu * q);
}

/* sin(pi*A/B) and cos(pi*A/B) for integers A and B > 0. The angle is
 * reduced in integer arithmetic to pi*y + q*pi/2 with |y| <= 1/4, so the
 * result keeps full relative accuracy even where it is zero or tiny. */
static void orc_sincospi_rational(int64_t A, int64_t B, double* s, double* c) {
  int64_t a = A % (2 * B);
  if (a < 0) a += 2 * B;                      /* angle pi*a/B, a in [0, 2B) */
  int64_t q = (4 * a + B) / (2 * B);          /* nearest multiple of pi/2: round(2a/B) */
  int64_t ynum = 2 * a - q * B;               /* y = ynum / (2B), |y| <= 1/4 */
  double y = ORC_PI * ((double)ynum / (double)(2 * B));
  double cy = cos(y), sy = sin(y);
  switch (q & 3) {
    case 0: *c = cy; *s = sy; break;
    case 1: *c = -sy; *s = cy; break;
    case 2: *c = -cy; *s = -sy; break;
    default: *c = sy; *s = -cy; break;
  }
}

/* J_nu(z) for z = pi*P/Q + delta, Q > 0, P >= 0, integer nu (any sign). */
double orc_besselj_pi(int nu, int64_t P, int64_t Q, double delta) {
  int sgn = 1;
  if (nu < 0) { nu = -nu; if (nu & 1) sgn = -1; }
  double z = ORC_PI * ((double)P / (double)Q) + delta;
  if (z <= 0.0) return (nu == 0) ? (double)sgn : 0.0;
  double v;
  if (z <= 2.0) {
    v = orc_series(nu, z);
  } else if (z < 25.0) {
    v = orc_miller(nu, z);
  } else {
    /* mu = z - (2nu+1)pi/4 = pi*(4P - (2nu+1)Q)/(4Q) + delta */
    double cx, sx;
    orc_sincospi_rational(4 * P - (int64_t)(2 * nu + 1) * Q, 4 * Q, &sx, &cx);
    double cd = cos(delta), sd = sin(delta);
    int ok;
    v = orc_hankel_sum(nu, z, cx * cd - sx * sd, sx * cd + cx * sd, &ok);
    if (!ok) v = orc_miller(nu, z); /* large order: the expansion is not yet accurate */
  }
  return sgn * v;
}

/* J_nu(z) for a plain FP64 argument. */
double orc_besselj(int nu, double z) {
  int sgn = 1;
  if (nu < 0) { nu = -nu; if (nu & 1) sgn = -1; }
  if (z <= 0.0) return (nu == 0) ? (double)sgn : 0.0;
  double v;
  if (z <= 2.0) v = orc_series(nu, z);
  else if (z < 25.0) v = orc_miller(nu, z);
  else {
    /* cos/sin of mu = z - c by the addition formula: libm reduces z itself
     * exactly, whereas the rounded difference z - c would lose ulp(z)/2. */
    double c = (2.0 * nu + 1.0) * ORC_PI / 4.0;
    double cz = cos(z), sz = sin(z), cc = cos(c), sc = sin(c);
    int ok;
    v = orc_hankel_sum(nu, z, cz * cc + sz * sc, sz * cc - cz * sc, &ok);
    if (!ok) v = orc_miller(nu, z);
  }
  return sgn * v;
}

/* ------------------------------------------------------------------ */
/* Nodes: b_n = j_{0,n} - (n-1/4)pi (Lemma 3.2)                        */
/* ------------------------------------------------------------------ */

static double orc_j0_offset_dd(int64_t n, double guess); /* double-double Newton, below */

/* b[n-1] for n = 1..count. Returns 0 on success. */
int orc_j0_zero_offsets(int64_t count, double* b) {
  for (int64_t n = 1; n <= count; ++n) {
    double beta = (n - 0.25) * ORC_PI;
    double ib = 1.0 / beta, ib2 = ib * ib;
    /* McMahon (DLMF 10.21.19) with mu = 4 nu^2 = 0 */
    double g = ib * (1.0 / 8.0 + ib2 * (-31.0 / 384.0 + ib2 * (3779.0 / 15360.0 - ib2 * (6277237.0 / 3440640.0))));
    for (int it = 0; it < 20; ++it) {
      /* z = pi*(4n-1)/4 + g */
      double j0 = orc_besselj_pi(0, 4 * n - 1, 4, g);
      double j1 = orc_besselj_pi(1, 4 * n - 1, 4, g);
      double step = j0 / j1; /* Newton: J_0' = -J_1 */
      g += step;
      if (fabs(step) <= 1e-17 * fabs(g)) break;
    }
    if (beta < 30.0) g = orc_j0_offset_dd(n, g); /* Miller's J_0 limits the FP64 Newton here */
    b[n - 1] = g;
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* The direct O(N^2) sum                                               */
/* ------------------------------------------------------------------ */

typedef struct {
  int task, nu, grid;
  int64_t gamma, N;
  int nrhs;
  const double* c;
  int64_t ldc;
  const int64_t* rows;
  int64_t nrows;
  double* f;
  int64_t ldf;
  const double* b; /* b_n, n = 1..N+1 (tasks 1, 2) */
  int64_t next;    /* work counter */
  pthread_mutex_t lock;
} orc_job;

/* Phase of entry (k, n), 1-based: z = pi*P/Q + delta. */
static void orc_phase(const orc_job* J, int64_t k, int64_t n, int64_t* P, int64_t* Q, double* delta) {
  int64_t N = J->N;
  if (J->task == ORC_TASK_SCHLOMILCH) {
    if (J->grid == 0) { *P = (k - 1) * (n + J->gamma); *Q = N - 1; }
    else { *P = k * (n + J->gamma); *Q = N; }
    *delta = 0.0;
  } else if (J->task == ORC_TASK_FOURIER_BESSEL) {
    double r;
    if (J->grid == 0) { *P = (k - 1) * (4 * n - 1); *Q = 4 * (N - 1); r = (double)(k - 1) / (double)(N - 1); }
    else { *P = k * (4 * n - 1); *Q = 4 * N; r = (double)k / (double)N; }
    *delta = r * J->b[n - 1];
  } else {
    /* r_k = j_{0,k}/j_{0,N+1} = rt_k + e_k with rt_k = (4k-1)/(4N+3) and
     * e_k = (b_k (N+3/4) - b_{N+1} (k-1/4)) / (j_{0,N+1} (N+3/4))  (proof of Lemma 3.2) */
    double bk = J->b[k - 1], bN1 = J->b[N];
    double jN1 = (N + 0.75) * ORC_PI + bN1;
    double ek = (bk * (N + 0.75) - bN1 * (k - 0.25)) / (jN1 * (N + 0.75));
    double rt = (double)(4 * k - 1) / (double)(4 * N + 3);
    double jn = (n - 0.25) * ORC_PI + J->b[n - 1];
    *P = (4 * k - 1) * (4 * n - 1);
    *Q = 4 * (4 * N + 3);
    *delta = rt * J->b[n - 1] + ek * jn;
  }
}

static void* orc_worker(void* arg) {
  orc_job* J = (orc_job*)arg;
  double* acc = (double*)malloc(sizeof(double) * 2 * (size_t)J->nrhs);
  for (;;) {
    pthread_mutex_lock(&J->lock);
    int64_t i = J->next++;
    pthread_mutex_unlock(&J->lock);
    if (i >= J->nrows) break;
    int64_t k = J->rows[i] + 1;
    for (int r = 0; r < J->nrhs; ++r) { acc[2 * r] = 0.0; acc[2 * r + 1] = 0.0; }
    for (int64_t n = 1; n <= J->N; ++n) {
      int64_t P, Q; double delta;
      orc_phase(J, k, n, &P, &Q, &delta);
      double jv = orc_besselj_pi(J->nu, P, Q, delta);
      for (int r = 0; r < J->nrhs; ++r) {
        /* Kahan-compensated accumulation */
        double y = J->c[r * J->ldc + (n - 1)] * jv - acc[2 * r + 1];
        double t = acc[2 * r] + y;
        acc[2 * r + 1] = (t - acc[2 * r]) - y;
        acc[2 * r] = t;
      }
    }
    for (int r = 0; r < J->nrhs; ++r) J->f[r * J->ldf + i] = acc[2 * r];
  }
  free(acc);
  return NULL;
}

/*
 * f[r*ldf + i] = sum_n c[r*ldc + n-1] J_nu(r_k omega_n) with k = rows[i]+1,
 * for r < nrhs, i < nrows. nthreads <= 0 uses every online core.
 * Returns 0, or -1 on invalid arguments.
 */
int orc_transform(int task, int nu, int grid, int64_t gamma, int64_t N, int nrhs,
                  const double* c, int64_t ldc, const int64_t* rows, int64_t nrows,
                  double* f, int64_t ldf, int nthreads) {
  if (N < 2 || nrhs < 1 || task < 0 || task > 2) return -1;
  if (task == ORC_TASK_DHT && nu != 0) return -1;
  for (int64_t i = 0; i < nrows; ++i) if (rows[i] < 0 || rows[i] >= N) return -1;
  orc_job J;
  memset(&J, 0, sizeof J);
  J.task = task; J.nu = nu; J.grid = grid; J.gamma = gamma; J.N = N; J.nrhs = nrhs;
  J.c = c; J.ldc = ldc; J.rows = rows; J.nrows = nrows; J.f = f; J.ldf = ldf;
  double* b = NULL;
  if (task != ORC_TASK_SCHLOMILCH) {
    b = (double*)malloc(sizeof(double) * (size_t)(N + 1));
    orc_j0_zero_offsets(N + 1, b);
  }
  J.b = b;
  pthread_mutex_init(&J.lock, NULL);
  if (nthreads <= 0) nthreads = (int)sysconf(_SC_NPROCESSORS_ONLN);
  if (nthreads < 1) nthreads = 1;
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nthreads);
  for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, orc_worker, &J);
  for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
  free(th);
  pthread_mutex_destroy(&J.lock);
  free(b);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Double-double brute force (N <= 64)                                 */
/* ------------------------------------------------------------------ */

typedef struct { double hi, lo; } dd;

static dd dd_two_sum(double a, double b) {
  double s = a + b, bb = s - a;
  dd r = { s, (a - (s - bb)) + (b - bb) };
  return r;
}
static dd dd_quick(double a, double b) { double s = a + b; dd r = { s, b - (s - a) }; return r; }
static dd dd_d(double a) { dd r = { a, 0.0 }; return r; }
static dd dd_add(dd a, dd b) {
  dd s = dd_two_sum(a.hi, b.hi), t = dd_two_sum(a.lo, b.lo);
  s.lo += t.hi; s = dd_quick(s.hi, s.lo); s.lo += t.lo; return dd_quick(s.hi, s.lo);
}
static dd dd_neg(dd a) { dd r = { -a.hi, -a.lo }; return r; }
static dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }
static dd dd_mul(dd a, dd b) {
  double p = a.hi * b.hi;
  double e = fma(a.hi, b.hi, -p);
  e += a.hi * b.lo + a.lo * b.hi;
  return dd_quick(p, e);
}
static dd dd_div(dd a, dd b) {
  double q1 = a.hi / b.hi;
  dd r = dd_sub(a, dd_mul(dd_d(q1), b));
  double q2 = r.hi / b.hi;
  r = dd_sub(r, dd_mul(dd_d(q2), b));
  double q3 = r.hi / b.hi;
  dd q = dd_quick(q1, q2);
  return dd_add(q, dd_d(q3));
}
static dd dd_scale(dd a, double s) { dd r = { a.hi * s, a.lo * s }; return r; } /* s a power of two */
static const dd DD_PI = { 3.141592653589793116, 1.2246467991473532072e-16 };

/* J_nu(z) in double-double, nu >= 0, z >= 0: series for z <= 2, Miller otherwise. */
static dd dd_besselj(int nu, dd z) {
  if (z.hi <= 0.0) return dd_d(nu == 0 ? 1.0 : 0.0);
  if (z.hi <= 2.0) {
    dd half = dd_scale(z, 0.5), h2 = dd_mul(half, half);
    dd term = dd_d(1.0);
    for (int i = 1; i <= nu; ++i) term = dd_div(dd_mul(term, half), dd_d((double)i));
    dd sum = term;
    for (int t = 1; t < 200; ++t) {
      term = dd_div(dd_neg(dd_mul(term, h2)), dd_d((double)t * (double)(t + nu)));
      sum = dd_add(sum, term);
      if (fabs(term.hi) <= 1e-34 * fabs(sum.hi)) break;
    }
    return sum;
  }
  int start = (int)z.hi + 80 + nu;
  if (start & 1) start += 1;
  dd jp1 = dd_d(0.0), j = dd_d(1e-30), norm = dd_d(0.0), jnu = dd_d(0.0);
  for (int k = start; k >= 1; --k) {
    if (k == nu) jnu = j;
    if ((k & 1) == 0) norm = dd_add(norm, dd_scale(j, 2.0));
    dd jm1 = dd_sub(dd_mul(dd_div(dd_d(2.0 * k), z), j), jp1);
    jp1 = j; j = jm1;
    if (fabs(j.hi) > 1e250) {
      j = dd_scale(j, 0x1p-830); jp1 = dd_scale(jp1, 0x1p-830);
      norm = dd_scale(norm, 0x1p-830); jnu = dd_scale(jnu, 0x1p-830);
    }
  }
  if (nu == 0) jnu = j;
  norm = dd_add(norm, j);
  return dd_div(jnu, norm);
}

/* b_n = j_{0,n} - (n-1/4)pi by Newton's method in double-double from a guess. */
static double orc_j0_offset_dd(int64_t n, double guess) {
  dd base = dd_mul(DD_PI, dd_d(n - 0.25));
  dd g = dd_d(guess);
  for (int it = 0; it < 8; ++it) {
    dd z = dd_add(base, g);
    dd step = dd_div(dd_besselj(0, z), dd_besselj(1, z));
    g = dd_add(g, step);
    if (fabs(step.hi) < 1e-33 * fabs(g.hi)) break;
  }
  return g.hi + g.lo;
}

/* j_{0,n} in double-double for n = 1..count, by Newton from the FP64 offsets. */
static void dd_j0_zeros(int64_t count, dd* out) {
  double* b = (double*)malloc(sizeof(double) * (size_t)count);
  orc_j0_zero_offsets(count, b);
  for (int64_t n = 1; n <= count; ++n) {
    dd base = dd_mul(DD_PI, dd_d(n - 0.25));
    dd g = dd_d(b[n - 1]);
    for (int it = 0; it < 8; ++it) {
      dd z = dd_add(base, g);
      dd step = dd_div(dd_besselj(0, z), dd_besselj(1, z));
      g = dd_add(g, step);
      if (fabs(step.hi) < 1e-33 * fabs(g.hi)) break;
    }
    out[n - 1] = dd_add(base, g);
  }
  free(b);
}

/* Same contract as orc_transform, all rows, in double-double; N <= 64, nu >= 0. */
int orc_transform_dd(int task, int nu, int grid, int64_t gamma, int64_t N, int nrhs,
                     const double* c, int64_t ldc, double* f, int64_t ldf) {
  if (N < 2 || N > 64 || nrhs < 1 || nu < 0 || task < 0 || task > 2) return -1;
  if (task == ORC_TASK_DHT && nu != 0) return -1;
  dd jz[66];
  if (task != ORC_TASK_SCHLOMILCH) dd_j0_zeros(N + 1, jz);
  for (int64_t k = 1; k <= N; ++k) {
    dd r;
    if (task == ORC_TASK_DHT) r = dd_div(jz[k - 1], jz[N]);
    else if (grid == 0) r = dd_div(dd_d((double)(k - 1)), dd_d((double)(N - 1)));
    else r = dd_div(dd_d((double)k), dd_d((double)N));
    for (int rr = 0; rr < nrhs; ++rr) {
      dd acc = dd_d(0.0);
      for (int64_t n = 1; n <= N; ++n) {
        dd w = (task == ORC_TASK_SCHLOMILCH) ? dd_mul(DD_PI, dd_d((double)(n + gamma))) : jz[n - 1];
        dd v = dd_besselj(nu, dd_mul(r, w));
        acc = dd_add(acc, dd_mul(dd_d(c[rr * ldc + (n - 1)]), v));
      }
      f[rr * ldf + (k - 1)] = acc.hi + acc.lo;
    }
  }
  return 0;
}

/* J_nu(z) evaluated in double-double, rounded to FP64 (test access). */
double orc_besselj_dd(int nu, double z) {
  int sgn = 1;
  if (nu < 0) { nu = -nu; if (nu & 1) sgn = -1; }
  dd v = dd_besselj(nu, dd_d(z));
  return sgn * (v.hi + v.lo);
}

/* j_{0,n} - (n-1/4)pi in double-double, rounded to FP64, n = 1..count (count <= 4096). */
int orc_j0_zero_offsets_dd(int64_t count, double* b) {
  if (count < 1 || count > 4096) return -1;
  dd* z = (dd*)malloc(sizeof(dd) * (size_t)count);
  dd_j0_zeros(count, z);
  for (int64_t n = 1; n <= count; ++n) {
    dd off = dd_sub(z[n - 1], dd_mul(DD_PI, dd_d(n - 0.25)));
    b[n - 1] = off.hi + off.lo;
  }
  free(z);
  return 0;
}
