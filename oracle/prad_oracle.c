/*
 * prad oracle: a plain, slow FP64 CPU restatement of the per-timestep
 * synchrotron-emission particle step of Wallin, Gonoskov & Marklund,
 * "Effects of high energy photon emissions in laser generated
 * ultra-relativistic plasmas: real-time synchrotron simulations"
 * (arXiv:1409.5574).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the CPU
 * baseline of the benchmark load this library. The GPU library never calls
 * it, includes none of its code and shares no header, table or constant
 * generator with it. Every function below cites the passage of the paper it
 * follows; readings where the paper is silent are marked READING.
 *
 * Pins (tests/test_oracle_*.py) fix each function against something other
 * than itself: the curand host Philox generator, scipy's K_nu quadrature,
 * the closed-form integrals of F and S, Boris invariants and closed-form
 * rotations, and Monte-Carlo expectations with computed sigma.
 *
 * Units.  SI at the interface for the problem description (dt in s, fields in
 * V/m and T, wavelength in m).  Particle state is normalised: time in
 * 1/omega_ref, length in c/omega_ref, momentum u = p/(m_e c), fields
 * E/(m_e c omega_ref/e) and B/(m_e omega_ref/e).  Energies are in m_e c^2.
 *
 * Build: gcc -O2 -std=c11 -fopenmp -ffp-contract=off -fPIC -shared.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- physical constants (CODATA 2018, exact where defined) ------------- */
#define ORC_C 299792458.0
#define ORC_QE 1.602176634e-19
#define ORC_ME 9.1093837015e-31
#define ORC_HBAR 1.054571817e-34
#define ORC_EPS0 8.8541878128e-12
#define ORC_PI 3.14159265358979323846

/* fine-structure constant alpha = e^2 / (4 pi eps0 hbar c), evaluated here */
double orc_alpha(void) {
  return ORC_QE * ORC_QE / (4.0 * ORC_PI * ORC_EPS0 * ORC_HBAR * ORC_C);
}

/* ======================================================================
 * Philox4x32-10 (Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11): ten rounds of the Philox S-box/P-box network on
 * a 128-bit counter, with the 64-bit key bumped by the Weyl constants
 * between rounds.  Written from the published definition.
 * ====================================================================== */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u; /* golden-ratio Weyl increment */
      k1 += 0xBB67AE85u; /* sqrt(3)-1 Weyl increment */
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ======================================================================
 * The synchrotron function, Eq. (8):  F(x) = x * int_x^inf K_{5/3}(y) dy.
 * With K_nu(y) = int_0^inf exp(-y cosh s) cosh(nu s) ds and the y-integral
 * taken first,  F(x) = x * int_0^inf exp(-x cosh s) cosh(5s/3)/cosh(s) ds.
 * The integrand is even and analytic in the strip |Im s| < pi/2, so the
 * trapezoid rule converges geometrically; step 1/16 leaves an error far
 * below double rounding.
 * ====================================================================== */
double orc_F_exact(double x) {
  if (!(x > 0.0)) return 0.0;
  const double h = 1.0 / 16.0;
  double sum = 0.5; /* s = 0: exp(-x) * 1 / 1, factored below */
  double s0 = exp(-x);
  double acc = 0.5 * s0;
  for (int k = 1; k < 4000; ++k) {
    double s = k * h;
    double ch = cosh(s);
    double arg = x * ch;
    if (arg > 800.0) break;
    double term = exp(-arg) * cosh(5.0 * s / 3.0) / ch;
    acc += term;
    if (arg > 50.0 && term < 1e-30 * acc) break;
  }
  (void)sum;
  return x * h * acc;
}

/* K_{5/3}(x) by the same representation (used for F'(x) = F/x - x K53). */
static double orc_K53(double x) {
  const double h = 1.0 / 16.0;
  double acc = 0.5 * exp(-x);
  for (int k = 1; k < 4000; ++k) {
    double s = k * h;
    double arg = x * cosh(s);
    if (arg > 800.0) break;
    double term = exp(-arg) * cosh(5.0 * s / 3.0);
    acc += term;
    if (arg > 50.0 && term < 1e-30 * acc) break;
  }
  return h * acc;
}

/* ---- interpolated F:  cubic Hermite in (ln x, ln F) on log-spaced nodes --
 * Nodes 1e-17 .. ~68, 600 per decade.  Values and slopes come from the
 * quadrature above (slope d ln F / d ln x = 1 - x^2 K53(x) / F(x)).  Below
 * the first node the leading small-x asymptote of F is used; above the last node, F is
 * taken as 0 (F(68) ~ 3e-29).  Nodes and interpolation deliberately differ
 * from the GPU library's table. */
#define ORC_NT 11300
static double orc_lx0, orc_dlx;
static double orc_lnF[ORC_NT], orc_slope[ORC_NT];
/* cumulative tables on the same nodes: int_0^x F(t)/t dt and int_0^x F dt */
static double orc_cumN[ORC_NT], orc_cumE[ORC_NT];
static double orc_a_val, orc_A_val;
static uint64_t orc_A_int;
static int orc_ready = 0;

static double orc_F_small(double x) {
  /* F(x) -> 4 pi / (sqrt(3) Gamma(1/3)) (x/2)^(1/3) as x -> 0 */
  const double c = 4.0 * ORC_PI / (sqrt(3.0) * tgamma(1.0 / 3.0));
  return c * cbrt(0.5 * x);
}

double orc_F(double x) {
  if (!(x > 0.0)) return 0.0;
  double lx = log(x);
  double u = (lx - orc_lx0) / orc_dlx;
  if (u < 0.0) return orc_F_small(x);
  if (u >= (double)(ORC_NT - 1)) return 0.0;
  int i = (int)u;
  double t = u - i;
  double h = orc_dlx;
  double y0 = orc_lnF[i], y1 = orc_lnF[i + 1];
  double m0 = orc_slope[i] * h, m1 = orc_slope[i + 1] * h;
  double t2 = t * t, t3 = t2 * t;
  double y = (2 * t3 - 3 * t2 + 1) * y0 + (t3 - 2 * t2 + t) * m0 +
             (-2 * t3 + 3 * t2) * y1 + (t3 - t2) * m1;
  return exp(y);
}

/* ======================================================================
 * Proposal density of the noise-reduction scheme, Eq. (11):
 *   S(x) = (4/3) x^(1/3) for x < a,   (7/9) e^(-x) for x > a,
 * with a fixed by int_0^inf S = 1, i.e.  a^(4/3) + (7/9) e^(-a) = 1.
 * READING: the paper prints a ~ 0.69021 (rounded); the exact root is solved
 * here by Newton in FP64.  At x == a the exponential branch is taken.
 * ====================================================================== */
static long double orc_solve_a(void) {
  /* long double (>= 64-bit mantissa on x86-64 and aarch64) so that the
   * integer branch threshold below is exact */
  long double a = 0.69L;
  for (int it = 0; it < 80; ++it) {
    long double f = powl(a, 4.0L / 3.0L) + (7.0L / 9.0L) * expl(-a) - 1.0L;
    long double df = (4.0L / 3.0L) * cbrtl(a) - (7.0L / 9.0L) * expl(-a);
    long double step = f / df;
    a -= step;
    if (fabsl(step) < 1e-19L) break;
  }
  return a;
}

double orc_const_a(void) { return orc_a_val; }

double orc_S(double x) {
  if (x < 0.0) return 0.0;
  if (x < orc_a_val) return (4.0 / 3.0) * cbrt(x);
  return (7.0 / 9.0) * exp(-x);
}

/* P(x) = int_0^x S, Eq. (12) */
double orc_P(double x) {
  if (x <= 0.0) return 0.0;
  if (x < orc_a_val) return pow(x, 4.0 / 3.0);
  return 1.0 - (7.0 / 9.0) * exp(-x);
}

/* Inverse of P for a real R' in (0,1) (tests only). */
double orc_Pinv(double R) {
  if (R < orc_A_val) return pow(R, 0.75);
  return -log((9.0 / 7.0) * (1.0 - R));
}

/* ======================================================================
 * Uniforms from one Philox block (READING; the paper only says R', R are
 * uniform on [0:1]):
 *   W  = w1 * 2^32 + w0  (64 bits),  R' = (W + 1/2) / 2^64,
 *   1 - R' = (~W + 1/2) / 2^64  (integer complement, exact),
 *   R  = (w2 + 1/2) / 2^32.
 * The branch R' < a^(4/3) is decided on the integer W against
 * T = round(a^(4/3) 2^64) (W < T), so every precision takes the same branch.
 * Returns x = P^-1(R') and stores R.
 * ====================================================================== */
uint64_t orc_branch_threshold(void) { return orc_A_int; }

static double orc_sample_x_branch(const uint32_t w[4], double* R_out,
                                  int* low_out) {
  uint64_t W = ((uint64_t)w[1] << 32) | (uint64_t)w[0];
  double x;
  *low_out = W < orc_A_int;
  if (W < orc_A_int) {
    double Rp = ((double)W + 0.5) * 0x1p-64;
    x = pow(Rp, 0.75);
  } else {
    uint64_t C = ~W;
    double one_minus = ((double)C + 0.5) * 0x1p-64;
    x = -log((9.0 / 7.0) * one_minus);
  }
  if (R_out) *R_out = ((double)w[2] + 0.5) * 0x1p-32;
  return x;
}

double orc_sample_x(const uint32_t w[4], double* R_out) {
  int low;
  return orc_sample_x_branch(w, R_out, &low);
}

/* S on the branch the sample was drawn from (READING: S is discontinuous at
 * x = a, and rounding can put a high-branch x a hair below a, so the branch,
 * not the rounded x, selects the formula of Eq. (11)). */
static double orc_S_branch(double x, int low) {
  return low ? (4.0 / 3.0) * cbrt(x) : (7.0 / 9.0) * exp(-x);
}

double orc_S_of_words(const uint32_t w[4]) {
  int low;
  double x = orc_sample_x_branch(w, 0, &low);
  return orc_S_branch(x, low);
}

/* ======================================================================
 * Spectral CDFs used by the statistical pins and the learned sampler's
 * error metric:
 *   number CDF  G(x) = int_0^x F(t)/t dt / (5 pi / 3)
 *   energy CDF  Q(x) = int_0^x F(t) dt  / (8 pi / (9 sqrt 3))   [Eq. (10)]
 * Both normalisers are the closed-form Mellin moments of F.  Cumulative
 * integrals are taken on the node grid in ln x with composite Simpson on
 * the Hermite interpolant (8 panels per node interval), plus the exact
 * integral of the small-x asymptote below the first node.
 * ====================================================================== */
static void orc_build_cums(void) {
  double x0 = exp(orc_lx0);
  double c = 4.0 * ORC_PI / (sqrt(3.0) * tgamma(1.0 / 3.0)) * cbrt(0.5);
  /* int_0^x0 c t^(1/3) / t dt = 3 c x0^(1/3); int_0^x0 c t^(1/3) dt = (3/4) c x0^(4/3) */
  orc_cumN[0] = 3.0 * c * cbrt(x0);
  orc_cumE[0] = 0.75 * c * pow(x0, 4.0 / 3.0);
  const int M = 8;
  for (int i = 0; i + 1 < ORC_NT; ++i) {
    double sN = 0.0, sE = 0.0;
    double h = orc_dlx / M;
    for (int k = 0; k <= M; ++k) {
      double ly = orc_lx0 + i * orc_dlx + k * h;
      double y = exp(ly);
      double f = orc_F(y);
      double wgt = (k == 0 || k == M) ? 1.0 : ((k & 1) ? 4.0 : 2.0);
      sN += wgt * f;       /* dt/t = d ln t */
      sE += wgt * f * y;   /* dt = t d ln t */
    }
    orc_cumN[i + 1] = orc_cumN[i] + sN * h / 3.0;
    orc_cumE[i + 1] = orc_cumE[i] + sE * h / 3.0;
  }
}

static double orc_cum_at(const double* cum, double x, int energy) {
  if (!(x > 0.0)) return 0.0;
  double lx = log(x);
  double u = (lx - orc_lx0) / orc_dlx;
  if (u < 0.0) {
    double c = 4.0 * ORC_PI / (sqrt(3.0) * tgamma(1.0 / 3.0)) * cbrt(0.5);
    return energy ? 0.75 * c * pow(x, 4.0 / 3.0) : 3.0 * c * cbrt(x);
  }
  if (u >= (double)(ORC_NT - 1)) return cum[ORC_NT - 1];
  int i = (int)u;
  /* Simpson from node i to x on the interpolant */
  double la = orc_lx0 + i * orc_dlx;
  const int M = 8;
  double h = (lx - la) / M;
  double s = 0.0;
  for (int k = 0; k <= M; ++k) {
    double y = exp(la + k * h);
    double f = orc_F(y) * (energy ? y : 1.0);
    double wgt = (k == 0 || k == M) ? 1.0 : ((k & 1) ? 4.0 : 2.0);
    s += wgt * f;
  }
  return cum[i] + s * h / 3.0;
}

double orc_int_F_over_x(double x) { return orc_cum_at(orc_cumN, x, 0); }
double orc_int_F(double x) { return orc_cum_at(orc_cumE, x, 1); }
double orc_G(double x) { return orc_int_F_over_x(x) / (5.0 * ORC_PI / 3.0); }
double orc_Q(double x) {
  return orc_int_F(x) / (8.0 * ORC_PI / (9.0 * sqrt(3.0)));
}

/* inverse number CDF by bisection in ln x (tests and sampler targets) */
double orc_Ginv(double r) {
  if (r <= 0.0) return 0.0;
  if (r >= 1.0) return INFINITY;
  /* ln x from -200: G(x) ~ 1.23 x^(1/3) reaches r = 1e-30 at ln x ~ -207,
   * so every r representable in the tests is bracketed */
  double lo = -230.0, hi = log(80.0);
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (orc_G(exp(mid)) < r) lo = mid; else hi = mid;
    if (hi - lo < 1e-15) break;
  }
  return exp(0.5 * (lo + hi));
}

void orc_G_batch(const double* x, double* out, int64_t n) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) out[i] = orc_G(x[i]);
}
void orc_Q_batch(const double* x, double* out, int64_t n) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) out[i] = orc_Q(x[i]);
}
void orc_Ginv_batch(const double* r, double* out, int64_t n) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) out[i] = orc_Ginv(r[i]);
}
void orc_F_batch(const double* x, double* out, int64_t n) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) out[i] = orc_F(x[i]);
}
void orc_F_exact_batch(const double* x, double* out, int64_t n) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) out[i] = orc_F_exact(x[i]);
}

/* ======================================================================
 * Angular spread of the emission about the particle's velocity (Eqs. (5)
 * and (6), the circular-motion spectrum by angle).  With x = omega/omega_c
 * (omega_c of Eq. (1), equal to (3/2) gamma^3 c / rho for the orbit radius
 * rho) and psi = gamma theta, theta the angle out of the plane of the orbit,
 * Eq. (6) gives xi = (x/2) (1 + psi^2)^(3/2) and Eq. (5)'s prefactor
 * (omega rho / c)^2 (1/gamma^2 + theta^2)^2 = (9/4) x^2 gamma^2 (1 + psi^2)^2,
 * so at fixed x the radiated energy per unit psi is proportional to
 *   sigma(x, psi) + pi(x, psi),
 *   sigma = (1 + psi^2)^2 K_2/3(xi)^2,  pi = (1 + psi^2) psi^2 K_1/3(xi)^2
 * (the two polarisation terms of Eq. (5)).  Integrated over all psi this
 * is (2 pi / sqrt 3) F(x) / x^2, F of Eq. (8); over x and psi the sigma
 * term carries 7/8 of the energy.  The paper's method emits along the
 * mean velocity (collinear); the optional spread turns each photon by
 * theta = psi / gamma out of the plane of the step's orbit, psi drawn
 * from this density (sign from a second Philox word).
 * ====================================================================== */

/* K_nu(z) = int_0^inf exp(-z cosh t) cosh(nu t) dt, trapezoid rule in t
 * (exponentially convergent for this integrand); the step shrinks as
 * 1/sqrt(z) where the peak at t = 0 narrows. */
static double orc_Knu(double nu, double z) {
  if (!(z > 0.0)) return INFINITY;
  const double h = 0.25 / (z > 5.0 ? sqrt(z / 5.0) : 1.0);
  double acc = 0.5 * exp(-z);
  for (int k = 1; k < 100000; ++k) {
    const double t = k * h;
    const double arg = z * cosh(t);
    if (arg > z + 745.0) break;
    acc += exp(-arg) * cosh(nu * t);
  }
  return h * acc;
}
double orc_K13(double z) { return orc_Knu(1.0 / 3.0, z); }
double orc_K23(double z) { return orc_Knu(2.0 / 3.0, z); }

void orc_ang_parts(double x, double psi, double* sig, double* pi) {
  const double q = 1.0 + psi * psi;
  const double xi = 0.5 * x * q * sqrt(q);
  const double k23 = orc_K23(xi), k13 = orc_K13(xi);
  *sig = q * q * k23 * k23;
  *pi = q * psi * psi * k13 * k13;
}

static double orc_ang_density(double x, double psi) {
  double s, p;
  orc_ang_parts(x, psi, &s, &p);
  return s + p;
}

/* psi where xi = xi(0) + 60: beyond it K^2(xi) has fallen by more than
 * e^-120 from its value at psi = 0 (K_nu(xi) ~ e^-xi) */
static double orc_ang_psimax(double x) {
  const double q = pow((x + 120.0) / x, 2.0 / 3.0);
  return sqrt(q - 1.0);
}

/* int_{sinh s0}^{sinh s1} density dpsi by composite Simpson in s = asinh psi
 * (dpsi = cosh s ds) with m (even) subintervals */
static double orc_ang_int(double x, double s0, double s1, int m) {
  const double h = (s1 - s0) / m;
  double acc = 0.0;
  for (int k = 0; k <= m; ++k) {
    const double s = s0 + k * h;
    const double wk = (k == 0 || k == m) ? 1.0 : ((k & 1) ? 4.0 : 2.0);
    acc += wk * orc_ang_density(x, sinh(s)) * cosh(s);
  }
  return acc * h / 3.0;
}

#define ORC_ANG_PANELS 256
#define ORC_ANG_SUB 4

/* int_0^inf density dpsi (one side; the density is even in psi) */
double orc_ang_norm(double x) {
  const double smax = asinh(orc_ang_psimax(x));
  return orc_ang_int(x, 0.0, smax, ORC_ANG_PANELS * ORC_ANG_SUB);
}

/* fraction of the one-sided integral below psi >= 0 */
double orc_ang_cdf(double x, double psi) {
  const double smax = asinh(orc_ang_psimax(x));
  const double s = asinh(fabs(psi));
  if (s >= smax) return 1.0;
  const int m = 2 * (int)ceil(0.5 * ORC_ANG_PANELS * ORC_ANG_SUB * s / smax) + 2;
  return orc_ang_int(x, 0.0, s, m) / orc_ang_norm(x);
}

/* psi >= 0 with cdf(psi) = u: cumulative Simpson panels in s, then
 * bisection on s inside the panel that holds u */
double orc_ang_sample(double x, double u) {
  const double smax = asinh(orc_ang_psimax(x));
  const double h = smax / ORC_ANG_PANELS;
  double cum[ORC_ANG_PANELS + 1];
  cum[0] = 0.0;
  for (int k = 0; k < ORC_ANG_PANELS; ++k)
    cum[k + 1] = cum[k] + orc_ang_int(x, k * h, (k + 1) * h, ORC_ANG_SUB);
  const double target = u * cum[ORC_ANG_PANELS];
  int k = 0;
  while (k < ORC_ANG_PANELS - 1 && cum[k + 1] < target) ++k;
  double a = k * h, b = (k + 1) * h;
  for (int it = 0; it < 60; ++it) {
    const double m = 0.5 * (a + b);
    if (cum[k] + orc_ang_int(x, k * h, m, ORC_ANG_SUB) < target) a = m; else b = m;
  }
  return sinh(0.5 * (a + b));
}

void orc_K13_batch(const double* z, double* out, int64_t n) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) out[i] = orc_K13(z[i]);
}
void orc_K23_batch(const double* z, double* out, int64_t n) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) out[i] = orc_K23(z[i]);
}
void orc_ang_parts_batch(const double* x, const double* psi, double* sig, double* pi,
                         int64_t n) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) orc_ang_parts(x[i], psi[i], &sig[i], &pi[i]);
}
void orc_ang_norm_batch(const double* x, double* out, int64_t n) {
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < n; ++i) out[i] = orc_ang_norm(x[i]);
}
void orc_ang_cdf_batch(const double* x, const double* psi, double* out, int64_t n) {
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < n; ++i) out[i] = orc_ang_cdf(x[i], psi[i]);
}
void orc_ang_sample_batch(const double* x, const double* u, double* out, int64_t n) {
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < n; ++i) out[i] = orc_ang_sample(x[i], u[i]);
}

int orc_init(void) {
  if (orc_ready) return 0;
  long double a_ld = orc_solve_a();
  long double A_ld = powl(a_ld, 4.0L / 3.0L);
  orc_a_val = (double)a_ld;
  orc_A_val = (double)A_ld;
  /* number of 64-bit words W with (W + 1/2) / 2^64 < a^(4/3) */
  orc_A_int = (uint64_t)floorl(ldexpl(A_ld, 64) + 0.5L);
  orc_lx0 = log(1e-17);
  orc_dlx = log(10.0) / 600.0;
  for (int i = 0; i < ORC_NT; ++i) {
    double x = exp(orc_lx0 + i * orc_dlx);
    double F = orc_F_exact(x);
    orc_lnF[i] = log(F);
    orc_slope[i] = 1.0 - x * x * orc_K53(x) / F;
  }
  orc_build_cums();
  orc_ready = 1;
  return 0;
}

/* ======================================================================
 * Boris push (Boris 1970, as used in the paper's Numerical implementation
 * section): half electric kick, magnetic rotation, half electric kick.
 * Normalised units, charge q in units of e, unit mass (electron/positron):
 *   du/dt = q (E + u x B / gamma).
 * ====================================================================== */
void orc_boris(double u[3], const double E[3], const double B[3], double q,
               double dtn) {
  double h = 0.5 * q * dtn;
  double um[3] = {u[0] + h * E[0], u[1] + h * E[1], u[2] + h * E[2]};
  double gm = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
  double t[3] = {h * B[0] / gm, h * B[1] / gm, h * B[2] / gm};
  double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
  double s[3] = {2.0 * t[0] / (1.0 + t2), 2.0 * t[1] / (1.0 + t2),
                 2.0 * t[2] / (1.0 + t2)};
  double up[3] = {um[0] + (um[1] * t[2] - um[2] * t[1]),
                  um[1] + (um[2] * t[0] - um[0] * t[2]),
                  um[2] + (um[0] * t[1] - um[1] * t[0])};
  double uq[3] = {um[0] + (up[1] * s[2] - up[2] * s[1]),
                  um[1] + (up[2] * s[0] - up[0] * s[2]),
                  um[2] + (up[0] * s[1] - up[1] * s[0])};
  u[0] = uq[0] + h * E[0];
  u[1] = uq[1] + h * E[1];
  u[2] = uq[2] + h * E[2];
}

/* ======================================================================
 * Effective magnetic field (normalised, Omega = |q| H_eff in m omega_r / e).
 * Field form: the field that gives the same transverse force,
 *   H_eff^2 = |E + beta x B|^2 - (E . beta)^2          (Eq. (1) context;
 *   the invariant form of the "same transverse acceleration" definition).
 * Momentum form, Eq. (9):
 *   H_eff = (m c gamma / e)(1/dt) sqrt(p^2 dp^2 - (p.dp)^2) / p^2,
 * with p the average momentum and dp the change over the step.
 * READING: gamma in Eq. (9) is the mean of the two end-point Lorentz
 * factors (exact for a Boris step in a pure perpendicular B).
 * ====================================================================== */
double orc_heff_field(const double E[3], const double B[3],
                      const double beta[3]) {
  double f0 = E[0] + (beta[1] * B[2] - beta[2] * B[1]);
  double f1 = E[1] + (beta[2] * B[0] - beta[0] * B[2]);
  double f2 = E[2] + (beta[0] * B[1] - beta[1] * B[0]);
  double eb = E[0] * beta[0] + E[1] * beta[1] + E[2] * beta[2];
  double h2 = f0 * f0 + f1 * f1 + f2 * f2 - eb * eb;
  return h2 > 0.0 ? sqrt(h2) : 0.0;
}

double orc_heff_momentum(const double u_old[3], const double u_new[3],
                         double dtn) {
  double p[3] = {0.5 * (u_old[0] + u_new[0]), 0.5 * (u_old[1] + u_new[1]),
                 0.5 * (u_old[2] + u_new[2])};
  double dp[3] = {u_new[0] - u_old[0], u_new[1] - u_old[1],
                  u_new[2] - u_old[2]};
  double p2 = p[0] * p[0] + p[1] * p[1] + p[2] * p[2];
  double dp2 = dp[0] * dp[0] + dp[1] * dp[1] + dp[2] * dp[2];
  double pdp = p[0] * dp[0] + p[1] * dp[1] + p[2] * dp[2];
  if (!(p2 > 0.0)) return 0.0;
  double g0 = sqrt(1.0 + u_old[0] * u_old[0] + u_old[1] * u_old[1] +
                   u_old[2] * u_old[2]);
  double g1 = sqrt(1.0 + u_new[0] * u_new[0] + u_new[1] * u_new[1] +
                   u_new[2] * u_new[2]);
  double gam = 0.5 * (g0 + g1);
  double c2 = p2 * dp2 - pdp * pdp;
  if (c2 < 0.0) c2 = 0.0;
  return gam * sqrt(c2) / (p2 * dtn);
}

/* ======================================================================
 * Problem description (SI) and the full step.
 * ====================================================================== */
typedef struct orc_problem {
  double omega_ref; /* rad/s */
  double dt;        /* s */
  double charge;    /* units of e (+-1), unit electron mass */
  uint64_t seed;
  uint32_t ensemble;
  int32_t rr_mode;   /* 0 off, 1 ledger only, 2 ledger + LL momentum kick */
  int32_t heff_form; /* 0 field form, 1 momentum form (Eq. (9)) */
  int32_t field_kind;/* 0 constant E,B; 1 CP plane wave along +-x; 2 Yee 2D */
  int32_t dims;      /* 3: 3D3V; 2: 2D3V (z frozen) */
  int32_t pad0;
  double E[3], B[3]; /* constant field [V/m], [T] */
  double a0, lambda, phase0; /* plane wave: amplitude, wavelength [m], phase */
  int32_t dir, hand;         /* propagation +-x, handedness +-1 */
  const float* yee[6];       /* Ex Ey Ez Bx By Bz, normalised, [ny][nx] */
  int32_t nx, ny;
  double dx, dy, x0, y0;     /* normalised grid spacing and origin */
  /* super-photon control (Monte Carlo method section: super-photons per
   * particle and step, real photons per super-photon): n_try trials of
   * 1/n_try of dN each; a particle-step takes part with probability
   * select_prob and then carries weight k w / select_prob */
  int32_t n_try;
  /* 1: turn each photon by theta = psi / gamma out of the plane of the
   * step's orbit (angular spread of Eqs. (5)-(6); 0: collinear) */
  int32_t ang_spread;
  double select_prob;
} orc_problem;

typedef struct orc_photons {
  int64_t capacity;
  double *x, *y, *z, *nx, *ny, *nz, *eps, *weight;
  uint32_t *pid, *step;
} orc_photons;

/* stats[0] records, [1] dropped, [2] dN>1, [3] clamp, [4] chi>1,
 * [5] steps outside the synchrotron (wiggler) regime, plane wave only:
 *     Omega < omega_L |1 - dir beta_x| (Omega tau_EM < 1, tau_EM the field
 *     period the particle sees; Eq. (3) and the text before it) */

/* normalisation factors */
static double orc_Er(double w) { return ORC_ME * ORC_C * w / ORC_QE; }
static double orc_Br(double w) { return ORC_ME * w / ORC_QE; }

/* quadratic-spline (second-order) weights about the nearest node */
static void orc_qs_weights(double xi, long* i0, double w[3]) {
  double n = floor(xi + 0.5);
  double d = xi - n;
  *i0 = (long)n;
  w[0] = 0.5 * (0.5 - d) * (0.5 - d);
  w[1] = 0.75 - d * d;
  w[2] = 0.5 * (0.5 + d) * (0.5 + d);
}

static double orc_yee_component(const orc_problem* P, int comp, double px,
                                double py) {
  /* staggering of the 2D Yee cell (i along x, j along y):
   * Ex (i+1/2, j), Ey (i, j+1/2), Ez (i, j),
   * Bx (i, j+1/2), By (i+1/2, j), Bz (i+1/2, j+1/2) */
  static const double sx[6] = {0.5, 0.0, 0.0, 0.0, 0.5, 0.5};
  static const double sy[6] = {0.0, 0.5, 0.0, 0.5, 0.0, 0.5};
  double xi = (px - P->x0) / P->dx - sx[comp];
  double yi = (py - P->y0) / P->dy - sy[comp];
  long i0, j0;
  double wx[3], wy[3];
  orc_qs_weights(xi, &i0, wx);
  orc_qs_weights(yi, &j0, wy);
  const float* F = P->yee[comp];
  double v = 0.0;
  for (int b = 0; b < 3; ++b) {
    long j = j0 - 1 + b;
    j %= P->ny; if (j < 0) j += P->ny;
    for (int a = 0; a < 3; ++a) {
      long i = i0 - 1 + a;
      i %= P->nx; if (i < 0) i += P->nx;
      v += wx[a] * wy[b] * (double)F[(size_t)j * (size_t)P->nx + (size_t)i];
    }
  }
  return v;
}

/* field at normalised position and step index n (time n * dtn) */
void orc_fields(const orc_problem* P, double px, double py, double pz,
                int64_t n, double E[3], double B[3]) {
  double w = P->omega_ref;
  (void)pz;
  if (P->field_kind == 0) {
    for (int k = 0; k < 3; ++k) {
      E[k] = P->E[k] / orc_Er(w);
      B[k] = P->B[k] / orc_Br(w);
    }
  } else if (P->field_kind == 1) {
    double wn = (2.0 * ORC_PI * ORC_C / P->lambda) / w; /* omega_L/omega_r */
    double E0 = P->a0 * wn;
    double t = (double)n * P->dt * w;
    double phi = wn * t - (double)P->dir * wn * px + P->phase0;
    double c = cos(phi), s = sin(phi);
    E[0] = 0.0;
    E[1] = E0 * c;
    E[2] = (double)P->hand * E0 * s;
    /* B = dir * x_hat x E  (unit c) */
    B[0] = 0.0;
    B[1] = -(double)P->dir * E[2];
    B[2] = (double)P->dir * E[1];
  } else {
    E[0] = orc_yee_component(P, 0, px, py);
    E[1] = orc_yee_component(P, 1, px, py);
    E[2] = orc_yee_component(P, 2, px, py);
    B[0] = orc_yee_component(P, 3, px, py);
    B[1] = orc_yee_component(P, 4, px, py);
    B[2] = orc_yee_component(P, 5, px, py);
  }
}

/*
 * Advance n particles by nsteps steps starting at global step index t0.
 * Follows the step list of the paper's Monte Carlo method section:
 * effective field (with the dp_perp/p <= 1 limit), omega_c (Eq. (1)),
 * a proposal frequency omega(R') from Eqs. (11)-(12), the emission count of
 * Eq. (13) and the comparison with R; plus the Landau-Lifshitz loss of
 * Eq. (4) booked in a per-particle ledger for the comparison of Fig. 3.
 *
 * READINGS (see also the uniform mapping above):
 *  - u_avg = (u^{n-1/2} + u^{n+1/2})/2 gives gamma and beta for H_eff and
 *    the LL loss; fields are taken at x^n, t^n.
 *  - The limit dp_perp/p <= 1 reads Omega * dt <= gamma_avg.
 *  - Eq. (13) per unit x = omega/omega_c (the omega_c of Eq. (10) cancels):
 *    dN = (sqrt3 / 2pi) alpha Omega dt F(x) / (x S(x)).
 *  - dN >= 1 gives multiplicity k = floor(dN) + [R < frac(dN)], stored as one
 *    record of weight k w.
 *  - Photon energy x * hbar omega_c, direction u_avg/|u_avg| (the collinear
 *    approximation of the Modelling section), position x^{n+1}.
 *  - The emitting particle gets no photon recoil; the LL force acts only in
 *    rr_mode 2, as an exact-for-beta->1 implicit kick
 *    u <- u / (1 + K gamma dt), K = (2/3) alpha eps_r Omega^2.
 *  - LL ledger increment per step: (2/3) alpha eps_r Omega^2 |u_avg|^2 dt
 *    (Eq. (4) with chi = eps_r Omega gamma and v^2 = beta^2).
 */
int orc_run(const orc_problem* P, int64_t n, int32_t nsteps, int64_t t0,
            double* X, double* Y, double* Z, double* UX, double* UY,
            double* UZ, const double* Wt, const uint32_t* pid,
            double* led_emit, double* led_ll, orc_photons* ph,
            int64_t* cursor, double* trial_dN, double* trial_R,
            double* trial_x, int64_t* stats) {
  if (!orc_ready) orc_init();
  const double w = P->omega_ref;
  const double dtn = P->dt * w;
  const double q = P->charge;
  const double alpha = orc_alpha();
  const double eps_r = ORC_HBAR * w / (ORC_ME * ORC_C * ORC_C);
  const double Cn = sqrt(3.0) / (2.0 * ORC_PI) * alpha; /* times Omega dt */
  const uint32_t key[2] = {(uint32_t)(P->seed & 0xffffffffu),
                           (uint32_t)(P->seed >> 32)};
  const double Lx = P->nx * P->dx, Ly = P->ny * P->dy;
  int64_t s_dn1 = 0, s_clamp = 0, s_chi = 0, s_rec = 0, s_drop = 0, s_wig = 0;
  const int n_try = P->n_try > 0 ? P->n_try : 1;
  const double q_sel = P->select_prob > 0.0 ? P->select_prob : 1.0;
  const double wl = (2.0 * ORC_PI * ORC_C / P->lambda) / w; /* omega_L / omega_ref */

#pragma omp parallel for schedule(dynamic, 64) \
    reduction(+ : s_dn1, s_clamp, s_chi, s_rec, s_drop, s_wig)
  for (int64_t i = 0; i < n; ++i) {
    double x = X[i], y = Y[i], z = Z ? Z[i] : 0.0;
    double u[3] = {UX[i], UY[i], UZ[i]};
    double wt = Wt[i];
    double le = led_emit[i], ll = led_ll[i];
    for (int32_t s = 0; s < nsteps; ++s) {
      int64_t step = t0 + s;
      double E[3], B[3];
      orc_fields(P, x, y, z, step, E, B);
      double uo[3] = {u[0], u[1], u[2]};
      orc_boris(u, E, B, q, dtn);
      double ua[3] = {0.5 * (uo[0] + u[0]), 0.5 * (uo[1] + u[1]),
                      0.5 * (uo[2] + u[2])};
      double ua2 = ua[0] * ua[0] + ua[1] * ua[1] + ua[2] * ua[2];
      double ga = sqrt(1.0 + ua2);
      double beta[3] = {ua[0] / ga, ua[1] / ga, ua[2] / ga};
      double Om;
      if (P->heff_form == 0)
        Om = fabs(q) * orc_heff_field(E, B, beta);
      else
        Om = orc_heff_momentum(uo, u, dtn);
      if (P->field_kind == 1 && Om < wl * fabs(1.0 - P->dir * beta[0])) s_wig++;
      if (Om * dtn > ga) { Om = ga / dtn; s_clamp++; }
      double wc = 1.5 * Om * ga * ga;          /* Eq. (1), normalised */
      double epsc = eps_r * wc;                /* hbar omega_c / m c^2 */
      double chi = (2.0 / 3.0) * epsc / ga;    /* Eq. (4) context */
      if (chi > 1.0) s_chi++;
      if (P->rr_mode >= 1)
        ll += wt * (2.0 / 3.0) * alpha * eps_r * Om * Om * ua2 * dtn;
      if (P->rr_mode == 2) {
        double K = (2.0 / 3.0) * alpha * eps_r * Om * Om;
        double gL = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        double f = 1.0 / (1.0 + K * gL * dtn);
        u[0] *= f; u[1] *= f; u[2] *= f;
      }
      double gn = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
      x += dtn * u[0] / gn;
      y += dtn * u[1] / gn;
      if (P->dims == 3) z += dtn * u[2] / gn;
      if (P->field_kind == 2) {
        x -= Lx * floor((x - P->x0) / Lx);
        y -= Ly * floor((y - P->y0) / Ly);
      }
      /* Monte Carlo emission: n_try trials, trial 0 from the block with
       * tag 0, trial j >= 1 from tag 0x10000 + j; the particle-step takes
       * part with probability select_prob (word 3 of the trial-0 block) */
      uint32_t ctr[4] = {pid[i], (uint32_t)step, 0u, P->ensemble}, rnd[4];
      orc_philox4x32_10(ctr, key, rnd);
      const int part = q_sel >= 1.0 || ((double)rnd[3] + 0.5) * 0x1p-32 < q_sel;
      for (int j = 0; j < n_try; ++j) {
        if (j > 0) {
          uint32_t cj[4] = {pid[i], (uint32_t)step, 0x10000u + (uint32_t)j, P->ensemble};
          orc_philox4x32_10(cj, key, rnd);
        }
        double R;
        int low;
        double xs = orc_sample_x_branch(rnd, &R, &low);
        double dN = Cn * Om * dtn * orc_F(xs) / (xs * orc_S_branch(xs, low)) / n_try;
        double fl = floor(dN);
        double k = fl + ((R < dN - fl) ? 1.0 : 0.0);
        if (part && dN > 1.0) s_dn1++;
        if (trial_dN && j == 0) {
          size_t idx = (size_t)i * (size_t)nsteps + (size_t)s;
          trial_dN[idx] = dN;
          trial_R[idx] = R;
          trial_x[idx] = xs;
        }
        if (part && k > 0.0 && wt > 0.0) {
          double eps = xs * epsc;
          double kw = k * wt / q_sel;
          le += kw * eps;
          int64_t slot;
#pragma omp atomic capture
          slot = (*cursor)++;
          if (slot < ph->capacity) {
            double un = sqrt(ua2);
            double inv = un > 0.0 ? 1.0 / un : 0.0;
            double dir[3] = {ua[0] * inv, ua[1] * inv, ua[2] * inv};
            if (P->ang_spread) {
              /* psi from the angular density at this x (its own Philox
               * block, tag 0x20000 + trial), theta = psi / gamma, turned
               * toward the orbit normal n = u^n x u^(n+1) / |u^n x u^(n+1)|
               * (the plane of the step's orbit holds both momenta; the LL
               * kick only rescales u^(n+1)) */
              uint32_t ca[4] = {pid[i], (uint32_t)step, 0x20000u + (uint32_t)j,
                                P->ensemble}, ra[4];
              orc_philox4x32_10(ca, key, ra);
              double psi = orc_ang_sample(xs, ((double)ra[0] + 0.5) * 0x1p-32);
              if (ra[1] & 0x80000000u) psi = -psi;
              double th = psi / ga;
              double c[3] = {uo[1] * u[2] - uo[2] * u[1], uo[2] * u[0] - uo[0] * u[2],
                             uo[0] * u[1] - uo[1] * u[0]};
              double cn = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
              if (cn > 0.0 && un > 0.0) {
                double ct = cos(th), st = sin(th);
                for (int a = 0; a < 3; ++a) dir[a] = ct * dir[a] + st * c[a] / cn;
              }
            }
            ph->x[slot] = x; ph->y[slot] = y; ph->z[slot] = z;
            ph->nx[slot] = dir[0]; ph->ny[slot] = dir[1]; ph->nz[slot] = dir[2];
            ph->eps[slot] = eps; ph->weight[slot] = kw;
            ph->pid[slot] = pid[i]; ph->step[slot] = (uint32_t)step;
            s_rec++;
          } else {
            s_drop++;
          }
        }
      }
    }
    X[i] = x; Y[i] = y; if (Z) Z[i] = z;
    UX[i] = u[0]; UY[i] = u[1]; UZ[i] = u[2];
    led_emit[i] = le; led_ll[i] = ll;
  }
  if (*cursor > ph->capacity) *cursor = ph->capacity;
  stats[0] += s_rec; stats[1] += s_drop; stats[2] += s_dn1;
  stats[3] += s_clamp; stats[4] += s_chi; stats[5] += s_wig;
  return 0;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Threads of the later parallel loops (timing of the single-core rate). */
void orc_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
