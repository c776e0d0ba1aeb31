// Host side of the C ABI declared in include/prad.h: context management,
// argument checking, normalisation of the SI problem description, the
// sampling table, launches and read-back.  Compute happens only in kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include <cuda_bf16.h>

#include "prad_internal.h"

using namespace prad;

namespace {

// ---- physical constants (CODATA 2018) -------------------------------------
constexpr double kC = 299792458.0;
constexpr double kQe = 1.602176634e-19;
constexpr double kMe = 9.1093837015e-31;
constexpr double kHbar = 1.054571817e-34;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kPi = 3.14159265358979323846;

thread_local char g_init_err[512];

}  // namespace

struct prad_ctx {
  prad_config cfg{};
  cudaStream_t stream = nullptr;
  int device = 0;
  int num_sms = 1;
  char err[512] = {0};
  // normalised constants
  double dtn = 0, alpha = 0, eps_r = 0;
  // fields
  prad_fields fields{};
  bool fields_set = false;
  // sampling tables
  float4* d_tab32 = nullptr;
  Coef4d* d_tab64 = nullptr;
  // photon buffer (SoA)
  float* d_ph[8] = {nullptr};
  uint32_t* d_pid = nullptr;
  uint32_t* d_step = nullptr;
  float4* d_pend = nullptr;      // learned sampler: per-slot network inputs
  double* d_hist = nullptr;      // angular histogram scratch (on first use)
  int finish_grid = 0;           // blocks of the learned sampler's finishing kernel
  // counters, ledgers, reduction scratch
  unsigned long long* d_cnt = nullptr;
  double* d_led_emit = nullptr;
  double* d_led_ll = nullptr;
  double* d_partials = nullptr;
  double* d_sums = nullptr;
  int red_blocks = 0;
  // host-side totals folded in at each drain
  int64_t drained_records = 0;
  int64_t drained_dropped = 0;
  // tile sort scratch (allocated on first use)
  SortBuffers sort{};
  // learned sampler
  float* d_mlp = nullptr;        // FP32 master parameters
  float* d_mlp_m = nullptr;      // Adam moments
  float* d_mlp_v = nullptr;
  float* d_mlp_grad = nullptr;
  __nv_bfloat16* d_mlp_w2 = nullptr;
  float* d_ginv = nullptr;       // ln G^-1 on a logit grid
  float* d_ang = nullptr;        // angular-spread table (PRAD_DIAG_ANGLE_SPREAD)
  float* d_mlp_partial = nullptr;
  float* d_mlp_loss_part = nullptr;
  float* d_mlp_loss = nullptr;
  int mlp_partial_blocks = 0;
  int64_t mlp_t = 0;             // Adam step count
  // batched ensembles
  StepParams<float>* d_batch = nullptr;
  int64_t* d_batch_off = nullptr;
  unsigned long long* d_batch_next = nullptr;
  unsigned long long* d_batch_busy = nullptr;  // per-CTA busy clocks of the last call
  int batch_busy_n = 0;                        // its entries
  int batch_grid = 0;                          // CTAs of the last call's launches
  int batch_cap = 0;
  std::vector<StepParams<float>> h_batch;
  std::vector<int64_t> h_batch_off;
  // captured CUDA graph of the last batch call shape
  cudaGraphExec_t graph_exec = nullptr;
  uint64_t graph_key = 0;
  // run-time specialised step kernels (prad_config.specialize)
  SpecCache* spec = nullptr;
  int64_t spec_launches = 0;
};

namespace {

int fail(prad_ctx* c, int code, const char* fmt, ...) {
  char* dst = c ? c->err : g_init_err;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(dst, 512, fmt, ap);
  va_end(ap);
  return code;
}

#define CK(ctx, call)                                                        \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess)                                                   \
      return fail((ctx), PRAD_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// ---- F(x) of Eq. (8) for the table ------------------------------------------
// F(x) = x int_0^inf exp(-x cosh s) cosh(5 s / 3) / cosh(s) ds, by composite
// 16-point Gauss-Legendre panels of width 1/2 up to where x cosh s > 720.
struct GaussLegendre {
  double x[16], w[16];
  GaussLegendre() {
    const int n = 16;
    for (int i = 0; i < n; ++i) {
      double z = std::cos(kPi * (i + 0.75) / (n + 0.5)), pp = 1.0;
      for (int it = 0; it < 100; ++it) {
        double p1 = 1.0, p2 = 0.0;
        for (int j = 1; j <= n; ++j) {
          const double p3 = p2;
          p2 = p1;
          p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
        }
        pp = n * (z * p1 - p2) / (z * z - 1.0);
        const double dz = p1 / pp;
        z -= dz;
        if (std::fabs(dz) < 1e-16) break;
      }
      x[i] = z;
      w[i] = 2.0 / ((1.0 - z * z) * pp * pp);
    }
  }
};

double synchrotron_F(double x, const GaussLegendre& gl) {
  if (!(x > 0.0)) return 0.0;
  const double smax = std::acosh(720.0 / x + 1.0);
  const double width = 0.5;
  double acc = 0.0;
  for (double a = 0.0; a < smax; a += width) {
    const double mid = a + 0.5 * width, half = 0.5 * width;
    for (int k = 0; k < 16; ++k) {
      const double s = mid + half * gl.x[k];
      const double ch = std::cosh(s);
      acc += half * gl.w[k] * std::exp(-x * ch) * std::cosh(5.0 * s / 3.0) / ch;
    }
  }
  return x * acc;
}

// g = F / S on each branch of the proposal, Eq. (11).
double g_low(double t, const GaussLegendre& gl) {  // x = t^3 < a
  if (t <= 0.0) {
    // lim F(x) / ((4/3) x^(1/3)) = (3/4) 4 pi / (sqrt3 Gamma(1/3)) 2^(-1/3)
    return 0.75 * 4.0 * kPi / (std::sqrt(3.0) * std::tgamma(1.0 / 3.0)) *
           std::cbrt(0.5);
  }
  const double x = t * t * t;
  return synchrotron_F(x, gl) / ((4.0 / 3.0) * t);
}
double g_high(double x, const GaussLegendre& gl) {  // x >= a
  return synchrotron_F(x, gl) * std::exp(x) * (9.0 / 7.0);
}

// Per-interval cubic through g at s = 0, 1/3, 2/3, 1 (Newton forward form
// expanded to monomials in s).
void cubic_coefs(double f0, double f1, double f2, double f3, double c[4]) {
  const double d1 = f1 - f0;
  const double d2 = f2 - 2.0 * f1 + f0;
  const double d3 = f3 - 3.0 * f2 + 3.0 * f1 - f0;
  c[0] = f0;
  c[1] = 3.0 * d1 - 1.5 * d2 + d3;
  c[2] = 4.5 * d2 - 4.5 * d3;
  c[3] = 4.5 * d3;
}

void build_tables(std::vector<float4>& t32, std::vector<Coef4d>& t64) {
  GaussLegendre gl;
  t32.resize(kNTab);
  t64.resize(kNTab);
  const double T1 = kCbrtA;
  for (int i = 0; i < kNTab; ++i) {
    double v[4];
    for (int k = 0; k < 4; ++k) {
      if (i < kN1) {
        const double t = (i + k / 3.0) * T1 / kN1;
        v[k] = g_low(t, gl);
      } else {
        const int j = i - kN1;
        const double x = kA + (j + k / 3.0) * (kXmax - kA) / kN2;
        v[k] = g_high(x, gl);
      }
    }
    double c[4];
    cubic_coefs(v[0], v[1], v[2], v[3], c);
    t64[i] = Coef4d{c[0], c[1], c[2], c[3]};
    t32[i] = make_float4(static_cast<float>(c[0]), static_cast<float>(c[1]),
                         static_cast<float>(c[2]), static_cast<float>(c[3]));
  }
}

// ---- G^-1 table ------------------------------------------------------------
// G(x) = int_0^x F(t)/t dt / (5 pi/3): cumulative Simpson in ln t on
// [1e-8, 90] (F from the quadrature above), the exact integral of the small-x
// asymptote below, and the upper tail accumulated from the top so 1 - G keeps
// its relative accuracy.  The table holds ln G^-1(r) at kGiN nodes uniform in
// logit(r) on [-kGiL, kGiL], by interpolation in (ln t, ln G) / (ln t, ln T).
void build_ginv(std::vector<float>& out) {
  GaussLegendre gl;
  const double lt0 = std::log(1e-8), lt1 = std::log(90.0), h = 0.02;
  const int M = static_cast<int>((lt1 - lt0) / h) + 1;
  std::vector<double> lt(M + 1), lo(M + 1), hi(M + 1), seg(M);
  const double c = 4.0 * kPi / (std::sqrt(3.0) * std::tgamma(1.0 / 3.0)) * std::cbrt(0.5);
  const double norm = 5.0 * kPi / 3.0;
  for (int k = 0; k <= M; ++k) lt[k] = lt0 + k * h;
  for (int k = 0; k < M; ++k) {  // Simpson, 4 panels, integrand F(e^y) dy
    const int P = 4;
    double acc = 0.0;
    for (int q = 0; q <= P; ++q) {
      const double y = lt[k] + q * h / P;
      const double wq = (q == 0 || q == P) ? 1.0 : ((q & 1) ? 4.0 : 2.0);
      acc += wq * synchrotron_F(std::exp(y), gl);
    }
    seg[k] = acc * (h / P) / 3.0;
  }
  lo[0] = 3.0 * c * std::cbrt(std::exp(lt0));
  for (int k = 0; k < M; ++k) lo[k + 1] = lo[k] + seg[k];
  hi[M] = 0.0;
  for (int k = M - 1; k >= 0; --k) hi[k] = hi[k + 1] + seg[k];
  const double total = lo[0] + hi[0];
  out.resize(kGiN);
  for (int i = 0; i < kGiN; ++i) {
    const double l = -kGiL + 2.0 * kGiL * i / (kGiN - 1);
    double lnx;
    if (l <= 0.0) {
      const double r = 1.0 / (1.0 + std::exp(-l));
      const double target = r * total;  // normalise by the computed total
      if (target <= lo[0]) {
        lnx = 3.0 * std::log(target / (3.0 * c));
      } else {
        int a = 0, b = M;
        while (b - a > 1) {
          const int m = (a + b) / 2;
          (lo[m] <= target ? a : b) = m;
        }
        const double f = (std::log(target) - std::log(lo[a])) /
                         (std::log(lo[b]) - std::log(lo[a]));
        lnx = lt[a] + f * (lt[b] - lt[a]);
      }
    } else {
      const double t1 = 1.0 / (1.0 + std::exp(l)) * total;  // (1 - r) total
      int a = 0, b = M;
      if (t1 <= hi[M - 1]) {
        a = M - 1;
        b = M;
        lnx = lt[M - 1];
      } else {
        while (b - a > 1) {
          const int m = (a + b) / 2;
          (hi[m] >= t1 ? a : b) = m;
        }
        const double f = (std::log(t1) - std::log(hi[a])) / (std::log(hi[b]) - std::log(hi[a]));
        lnx = lt[a] + f * (lt[b] - lt[a]);
      }
    }
    out[i] = static_cast<float>(lnx);
  }
  (void)norm;
}

// ---- angular spread table (Eqs. (5)-(6)) -----------------------------------
// K_1/3 and K_2/3 on nodes uniform in ln z over [kKz0, kKz0 + (n - 1) kKh]:
// K_nu(z) = int_0^inf exp(-z cosh t) cosh(nu t) dt and its z-derivative
// -int_0^inf cosh t exp(-z cosh t) cosh(nu t) dt by 16-point Gauss-Legendre
// panels (scaled by e^z against underflow); between nodes cubic Hermite in
// (ln z, ln K).  The density needs z = xi in [x/2, x/2 + 50] for x in the
// table's range: [5e-9, 70].
struct BesselThirds {
  static constexpr double kKz0 = -21.0, kKh = 1.0 / 256.0;
  static constexpr int kN = 26 * 256 + 1;  // up to ln z = 5
  std::vector<double> l13, l23, d13, d23;  // ln K, d ln K / d ln z
  explicit BesselThirds(const GaussLegendre& gl)
      : l13(kN), l23(kN), d13(kN), d23(kN) {
    for (int k = 0; k < kN; ++k) {
      const double z = std::exp(kKz0 + k * kKh);
      const double tmax = std::acosh(1.0 + 745.0 / z);
      const double width = 0.5 / std::max(1.0, std::sqrt(z / 5.0));
      double a1 = 0, a2 = 0, b1 = 0, b2 = 0;
      for (double a = 0.0; a < tmax; a += width) {
        const double mid = a + 0.5 * width, half = 0.5 * width;
        for (int q = 0; q < 16; ++q) {
          const double t = mid + half * gl.x[q];
          const double ch = std::cosh(t);
          const double e = half * gl.w[q] * std::exp(-z * (ch - 1.0));
          const double c1 = std::cosh(t / 3.0), c2 = 2.0 * c1 * c1 - 1.0;  // cosh(2t/3)
          a1 += e * c1;
          a2 += e * c2;
          b1 += e * c1 * ch;
          b2 += e * c2 * ch;
        }
      }
      l13[k] = std::log(a1) - z;
      l23[k] = std::log(a2) - z;
      d13[k] = -z * b1 / a1;
      d23[k] = -z * b2 / a2;
    }
  }
  void eval(double z, double* k13, double* k23) const {
    double u = (std::log(z) - kKz0) / kKh;
    u = std::min(std::max(u, 0.0), static_cast<double>(kN - 1));
    const int i = std::min(static_cast<int>(u), kN - 2);
    const double t = u - i, t2 = t * t, t3 = t2 * t;
    const double h00 = 2 * t3 - 3 * t2 + 1, h10 = t3 - 2 * t2 + t, h01 = -2 * t3 + 3 * t2,
                 h11 = t3 - t2;
    *k13 = std::exp(h00 * l13[i] + h10 * kKh * d13[i] + h01 * l13[i + 1] + h11 * kKh * d13[i + 1]);
    *k23 = std::exp(h00 * l23[i] + h10 * kKh * d23[i] + h01 * l23[i + 1] + h11 * kKh * d23[i + 1]);
  }
};

// The table of y = psi / (v s(x)) (geometry in prad_internal.h): per row x,
// the one-sided integral of Eq. (5)'s density in psi, (1 + psi^2)^2
// K_2/3(xi)^2 + (1 + psi^2) psi^2 K_1/3(xi)^2 with xi = (x/2)(1 + psi^2)^(3/2),
// by 4-point Gauss-Legendre on 1024 equal steps in s = asinh psi up to
// xi = x/2 + 50; cumulative from below and tail from above (so 1 - u keeps
// its accuracy); psi for each column's u from the cubic Hermite form of the
// cumulative over the step that holds it (values and slopes at its ends).
void build_ang_table(std::vector<float>& out) {
  GaussLegendre gl16;
  const BesselThirds kb(gl16);
  static const double g4x[4] = {-0.8611363115940526, -0.3399810435848563, 0.3399810435848563,
                                0.8611363115940526};
  static const double g4w[4] = {0.3478548451374538, 0.6521451548625461, 0.6521451548625461,
                                0.3478548451374538};
  const int M = 1024;
  std::vector<double> seg(M), D(M + 1), lo(M + 1), hi(M + 1);
  out.assign(static_cast<size_t>(kAngNL) * kAngNV, 0.0f);
  for (int i = 0; i < kAngNL; ++i) {
    const double lx = kAngLx0 + i * (kAngLx1 - kAngLx0) / (kAngNL - 1);
    const double x = std::exp(lx);
    auto dens_s = [&](double sv) {  // density in s: (sigma + pi) dpsi/ds
      const double psi = std::sinh(sv), q = 1.0 + psi * psi;
      double k13, k23;
      kb.eval(0.5 * x * q * std::sqrt(q), &k13, &k23);
      return (q * q * k23 * k23 + q * psi * psi * k13 * k13) * std::cosh(sv);
    };
    const double qmax = std::pow((x + 100.0) / x, 2.0 / 3.0);
    const double hs = std::asinh(std::sqrt(qmax - 1.0)) / M;
    for (int k = 0; k <= M; ++k) D[k] = dens_s(k * hs);
    for (int k = 0; k < M; ++k) {
      double acc = 0.0;
      for (int q = 0; q < 4; ++q) acc += g4w[q] * dens_s((k + 0.5 + 0.5 * g4x[q]) * hs);
      seg[k] = 0.5 * hs * acc;
    }
    lo[0] = 0.0;
    for (int k = 0; k < M; ++k) lo[k + 1] = lo[k] + seg[k];
    hi[M] = 0.0;
    for (int k = M - 1; k >= 0; --k) hi[k] = hi[k + 1] + seg[k];
    const double total = lo[M];
    const double sc = std::cbrt(2.0 / x) * std::pow(1.0 + x, -1.0 / 6.0);
    for (int j = 1; j < kAngNV; ++j) {
      const double v = j * kAngVmax / (kAngNV - 1), w = v * v;
      int k;
      double m;  // mass below the target inside step k
      if (w <= std::log(2.0)) {  // u <= 1/2
        const double target = -std::expm1(-w) * total;
        int a = 0, b = M;
        while (b - a > 1) {
          const int mid = (a + b) / 2;
          (lo[mid] <= target ? a : b) = mid;
        }
        k = a;
        m = target - lo[k];
      } else {
        const double tail = std::exp(-w) * total;  // (1 - u) total
        int a = 0, b = M;
        while (b - a > 1) {
          const int mid = (a + b) / 2;
          (hi[mid] > tail ? a : b) = mid;
        }
        k = a;
        m = seg[k] - (tail - hi[k + 1]);
      }
      m = std::min(std::max(m, 0.0), seg[k]);
      // C(tau) = seg h01 + hs D_k h10 + hs D_k+1 h11 = m, by bisection
      double ta = 0.0, tb = 1.0;
      for (int it = 0; it < 60; ++it) {
        const double t = 0.5 * (ta + tb), t2 = t * t, t3 = t2 * t;
        const double c = seg[k] * (-2 * t3 + 3 * t2) + hs * D[k] * (t3 - 2 * t2 + t) +
                         hs * D[k + 1] * (t3 - t2);
        (c < m ? ta : tb) = t;
      }
      const double psi = std::sinh((k + 0.5 * (ta + tb)) * hs);
      out[static_cast<size_t>(i) * kAngNV + j] = static_cast<float>(psi / (v * sc));
    }
  }
}

static_assert(PRAD_ANG_NL == kAngNL && PRAD_ANG_NV == kAngNV &&
                  PRAD_ANG_LX0 == kAngLx0 && PRAD_ANG_LX1 == kAngLx1 &&
                  PRAD_ANG_VMAX == kAngVmax,
              "public and internal angular-table geometry agree");

// The table, built on first use in the process (~0.3 s), like the tables
// prad_init builds.
const std::vector<float>& ang_table_host() {
  static std::once_flag once;
  static std::vector<float> t;
  std::call_once(once, [] { build_ang_table(t); });
  return t;
}

uint16_t to_bf16(float f) {  // round to nearest even
  uint32_t u;
  std::memcpy(&u, &f, 4);
  const uint32_t rounding = 0x7FFFu + ((u >> 16) & 1u);
  return static_cast<uint16_t>((u + rounding) >> 16);
}

// Fixed Glorot-uniform initialisation (splitmix64 stream), biases zero
// except the output bias, which starts at the typical ln x / 10.
void init_mlp_params(std::vector<float>& p, uint64_t seed) {
  p.assign(kNumParams, 0.0f);
  uint64_t st = seed * 0x9E3779B97F4A7C15ull + 1;
  auto uni = [&]() {
    st += 0x9E3779B97F4A7C15ull;
    uint64_t z = st;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (static_cast<double>(z >> 11) + 0.5) * 0x1p-53 * 2.0 - 1.0;
  };
  const double a1 = std::sqrt(6.0 / (3 + kHid)), a2 = std::sqrt(6.0 / (2 * kHid)),
               a3 = std::sqrt(6.0 / (kHid + 1));
  for (int k = 0; k < kHid * 3; ++k) p[kOffW1 + k] = static_cast<float>(a1 * uni());
  for (int k = 0; k < kHid * kHid; ++k) p[kOffW2 + k] = static_cast<float>(a2 * uni());
  for (int k = 0; k < kHid; ++k) p[kOffW3 + k] = static_cast<float>(a3 * uni());
  p[kOffB3] = -0.1f;
}

int upload_mlp(prad_ctx* c, const float* host_params) {
  std::vector<uint16_t> w2(kHid * kHid);
  for (int k = 0; k < kHid * kHid; ++k) w2[k] = to_bf16(host_params[kOffW2 + k]);
  CK(c, cudaMemcpyAsync(c->d_mlp, host_params, sizeof(float) * kNumParams,
                        cudaMemcpyHostToDevice, c->stream));
  CK(c, cudaMemcpyAsync(c->d_mlp_w2, w2.data(), sizeof(uint16_t) * kHid * kHid,
                        cudaMemcpyHostToDevice, c->stream));
  CK(c, cudaMemsetAsync(c->d_mlp_m, 0, sizeof(float) * kNumParams, c->stream));
  CK(c, cudaMemsetAsync(c->d_mlp_v, 0, sizeof(float) * kNumParams, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  c->mlp_t = 0;
  return PRAD_OK;
}

// Super-photon control or diagnostics enabled: the kernels' CTRL variant.
bool ctrl_of(const prad_ctx* c) {
  return c->cfg.n_try > 1 || (c->cfg.select_prob > 0.0 && c->cfg.select_prob < 1.0) ||
         c->cfg.diagnostics != 0;
}

// The standard configuration of the batched kernel's ensembles (constant or
// plane-wave fields, so three dimensions): LL kick applied, field-form H_eff.
// the batched kernel's standard variant: as std_config of the step kernels
// (LL kick applied, field-form H_eff, unit charge)
bool std_of(const prad_ctx* c) {
  return c->cfg.rr_mode == PRAD_RR_APPLY && c->cfg.heff_form == PRAD_HEFF_FIELD &&
         std::fabs(c->cfg.charge) == 1.0;
}

MlpDev mlp_dev(const prad_ctx* c) {
  MlpDev d;
  d.params = c->d_mlp;
  d.w2 = c->d_mlp_w2;
  return d;
}

// Learned sampler: energies and ledger entries of the records appended
// since the last call (one launch after each push or batch call).
int mlp_finish(prad_ctx* c, double* led_base) {
  if (c->cfg.sampler == PRAD_SAMPLER_TABLE) return PRAD_OK;
  MlpFinishArgs a;
  a.mlp = mlp_dev(c);
  a.ginv = c->d_ginv;
  a.eps = c->d_ph[6];
  a.weight = c->d_ph[7];
  a.pend = c->d_pend;
  a.counters = c->d_cnt;
  a.led_emit = led_base;
  a.cap = c->cfg.photon_capacity;
  a.wdt_per_eps = static_cast<float>(c->dtn / c->eps_r);
  a.check_output = c->cfg.sampler == PRAD_SAMPLER_MLP_FALLBACK;
  CK(c, launch_mlp_finish(a, c->finish_grid, c->stream));
  return PRAD_OK;
}

template <typename R>
void fill_common(const prad_ctx* c, StepParams<R>& p, const prad_fields& f);

template <typename R>
void fill_common(const prad_ctx* c, StepParams<R>& p) {
  fill_common<R>(c, p, c->fields);
}

template <typename R>
void fill_common(const prad_ctx* c, StepParams<R>& p, const prad_fields& f) {
  const double q = c->cfg.charge;
  const double dtn = c->dtn;
  p.half_q_dtn = static_cast<R>(0.5 * q * dtn);
  p.dtn = static_cast<R>(dtn);
  p.inv_dtn = static_cast<R>(1.0 / dtn);
  p.abs_q = static_cast<R>(std::fabs(q));
  p.cn_dt = static_cast<R>(std::sqrt(3.0) / (2.0 * kPi) * c->alpha * dtn);
  p.eps_r = static_cast<R>(c->eps_r);
  p.eps_r15 = static_cast<R>(1.5 * c->eps_r);
  p.ll_coef = static_cast<R>(2.0 / 3.0 * c->alpha * c->eps_r * dtn);
  p.rr_mode = c->cfg.rr_mode;
  p.heff_form = c->cfg.heff_form;
  p.ensemble = c->cfg.ensemble;
  p.key0 = static_cast<uint32_t>(c->cfg.seed & 0xffffffffull);
  p.key1 = static_cast<uint32_t>(c->cfg.seed >> 32);
  philox_round_keys(c->cfg.seed, p.rkey);
  p.t_scale = static_cast<R>(kTScale);
  p.x_scale = static_cast<R>(kXScale);
  p.a = static_cast<R>(kA);
  p.thr = kThr;
  if constexpr (sizeof(R) == 4)
    p.tab = c->d_tab32;
  else
    p.tab = c->d_tab64;
  p.px = c->d_ph[0]; p.py = c->d_ph[1]; p.pz = c->d_ph[2];
  p.pnx = c->d_ph[3]; p.pny = c->d_ph[4]; p.pnz = c->d_ph[5];
  p.peps = c->d_ph[6]; p.pw = c->d_ph[7];
  p.ppid = c->d_pid; p.pstep = c->d_step;
  p.ppend = c->d_pend;
  p.cap = c->cfg.photon_capacity;
  p.counters = c->d_cnt;
  p.led_off = 0;
  p.led_base = c->d_led_emit;
  p.cp_dt = static_cast<R>(5.0 * std::sqrt(3.0) / 6.0 * c->alpha * dtn);
  p.ntry = c->cfg.n_try > 0 ? c->cfg.n_try : 1;
  p.diag = c->cfg.diagnostics;
  const double q_sel = c->cfg.select_prob > 0.0 ? c->cfg.select_prob : 1.0;
  p.inv_ntry = static_cast<R>(1.0 / p.ntry);
  p.sel_q = static_cast<R>(q_sel);
  p.inv_sel_q = static_cast<R>(1.0 / q_sel);
  p.wl = R(0);
  p.mlp = mlp_dev(c);
  p.ginv = c->d_ginv;
  p.ang = c->d_ang;
  // field, normalised: E by m c omega_ref / e, B by m omega_ref / e
  const double w = c->cfg.omega_ref;
  p.field_kind = f.kind;
  const double Er = kMe * kC * w / kQe, Br = kMe * w / kQe;
  for (int k = 0; k < 3; ++k) {
    p.E[k] = static_cast<R>(f.E[k] / Er);
    p.B[k] = static_cast<R>(f.B[k] / Br);
  }
  p.dims = 3;
  if (f.kind == PRAD_FIELD_PLANE_WAVE) {
    const double wn = (2.0 * kPi * kC / f.lambda) / w;  // omega_L / omega_ref
    p.wl = static_cast<R>(wn);
    p.E0 = static_cast<R>(f.a0 * wn);
    const double kcd = f.dir * wn / (2.0 * kPi);
    p.kc = static_cast<R>(kcd);
    p.kc_lo = static_cast<R>(kcd - static_cast<double>(p.kc));
    p.hand = static_cast<R>(f.hand);
    p.dir = static_cast<R>(f.dir);
    // hand, dir = +-1: these products are exact
    p.pw_ez = p.hand * p.E0;
    p.pw_by = -p.dir * p.hand * p.E0;
    p.pw_bz = p.dir * p.E0;
    // fixed-point cycles: phase0 / 2pi and omega_L dt / 2pi, modulo 1
    long double c0 = static_cast<long double>(f.phase0) / (2.0L * kPi);
    c0 -= std::floor(c0);
    long double cs = static_cast<long double>(wn) * dtn / (2.0L * kPi);
    cs -= std::floor(cs);
    p.phase_t0 = static_cast<uint64_t>(std::ldexp(c0, 64));
    p.phase_step = static_cast<uint64_t>(std::ldexp(cs, 64));
  } else {
    p.E0 = p.kc = p.kc_lo = p.hand = p.dir = R(0);
    p.pw_ez = p.pw_by = p.pw_bz = R(0);
    p.phase_t0 = p.phase_step = 0;
  }
  if (f.kind == PRAD_FIELD_YEE2D) {
    for (int k = 0; k < 6; ++k) p.yee[k] = f.yee[k];
    p.nx = f.nx; p.ny = f.ny;
    p.inv_dx = static_cast<R>(1.0 / f.dx);
    p.inv_dy = static_cast<R>(1.0 / f.dy);
    p.inv_dx_lo = static_cast<R>(1.0 / f.dx - static_cast<double>(p.inv_dx));
    p.inv_dy_lo = static_cast<R>(1.0 / f.dy - static_cast<double>(p.inv_dy));
    p.x0 = static_cast<R>(f.x0);
    p.y0 = static_cast<R>(f.y0);
    p.Lx = static_cast<R>(f.nx * f.dx);
    p.Ly = static_cast<R>(f.ny * f.dy);
    p.dims = 2;
  } else {
    for (int k = 0; k < 6; ++k) p.yee[k] = nullptr;
    p.nx = p.ny = 0;
    p.inv_dx = p.inv_dy = p.x0 = p.y0 = p.Lx = p.Ly = R(0);
    p.inv_dx_lo = p.inv_dy_lo = R(0);
  }
}

bool aligned(const void* p, size_t a) {
  return (reinterpret_cast<uintptr_t>(p) % a) == 0;
}

void free_sort(SortBuffers& b) {
  for (int k = 0; k < 7; ++k) cudaFree(b.tmp[k]);
  cudaFree(b.tmp_pid);
  cudaFree(b.counts);
  cudaFree(b.starts);
  cudaFree(b.cursor);
  cudaFree(b.work);
  cudaFree(b.work_count);
  b = SortBuffers{};
}

int tile_counts(const prad_fields& f, int* ntx, int* nty) {
  *ntx = (f.nx + kTile - 1) / kTile;
  *nty = (f.ny + kTile - 1) / kTile;
  return (*ntx) * (*nty);
}

int64_t max_work_items(int64_t n, int ntiles) {
  return n / kChunk + (n < ntiles ? n : ntiles) + 1;
}

// Scratch for the sort: max_particles copies of the 7 state arrays and the
// ids, per-tile counters and the work list.
int ensure_sort(prad_ctx* c, size_t elem) {
  int ntx, nty;
  const int ntiles = tile_counts(c->fields, &ntx, &nty);
  SortBuffers& b = c->sort;
  if (b.capacity >= c->cfg.max_particles && b.ntiles >= ntiles) return PRAD_OK;
  free_sort(b);
  const size_t np = static_cast<size_t>(c->cfg.max_particles);
  for (int k = 0; k < 7; ++k) CK(c, cudaMalloc(&b.tmp[k], np * elem));
  CK(c, cudaMalloc(&b.tmp_pid, np * sizeof(uint32_t)));
  CK(c, cudaMalloc(&b.counts, sizeof(unsigned int) * ntiles));
  CK(c, cudaMalloc(&b.starts, sizeof(unsigned int) * (ntiles + 1)));
  CK(c, cudaMalloc(&b.cursor, sizeof(unsigned int) * ntiles));
  const int64_t mw = max_work_items(c->cfg.max_particles, ntiles);
  CK(c, cudaMalloc(&b.work, sizeof(int4) * mw));
  CK(c, cudaMalloc(&b.work_count, sizeof(unsigned int)));
  b.capacity = c->cfg.max_particles;
  b.ntiles = ntiles;
  b.max_work = static_cast<int32_t>(mw);
  return PRAD_OK;
}

template <typename R>
int sort_t(prad_ctx* c, const prad_particles* pp, int64_t n) {
  int rc = ensure_sort(c, sizeof(R));
  if (rc != PRAD_OK) return rc;
  int ntx, nty;
  const int ntiles = tile_counts(c->fields, &ntx, &nty);
  SortBuffers b = c->sort;
  b.ntiles = ntiles;
  R* arr[7] = {static_cast<R*>(pp->x), static_cast<R*>(pp->y), static_cast<R*>(pp->z),
               static_cast<R*>(pp->ux), static_cast<R*>(pp->uy), static_cast<R*>(pp->uz),
               static_cast<R*>(pp->w)};
  const prad_fields& f = c->fields;
  CK(c, launch_tile_sort<R>(arr, pp->pid, n, b, f.nx, f.ny, f.x0, f.y0, 1.0 / f.dx,
                            1.0 / f.dy, c->stream));
  return PRAD_OK;
}

int check_sort_args(prad_ctx* c, const prad_particles* pp, int64_t n) {
  if (!c->fields_set || c->fields.kind != PRAD_FIELD_YEE2D)
    return fail(c, PRAD_ERR_STATE, "sort_by_tile: fields are not YEE2D");
  if (!pp->pid) return fail(c, PRAD_ERR_ARG, "sort_by_tile: a pid array is required");
  if (n > c->cfg.max_particles)
    return fail(c, PRAD_ERR_ARG, "sort_by_tile: n exceeds max_particles");
  if (!aligned(pp->pid, 4)) return fail(c, PRAD_ERR_ARG, "sort_by_tile: misaligned pid");
  return PRAD_OK;
}

// The run-time specialised kernel a float launch runs (*f = nullptr when the
// context does not ask for one or the launch is not of a specialisable
// variant); PRAD_ERR_CUDA when it cannot be compiled.
int spec_for(prad_ctx* c, const StepParams<float>& p, bool tiled, const SpecFn** f) {
  *f = nullptr;
  SpecVariant v;
  if (!c->cfg.specialize ||
      !push_emit_spec_variant(p, c->fields.kind, c->cfg.sampler, tiled, &v))
    return PRAD_OK;
  if (!c->spec) c->spec = spec_create();
  char msg[448] = {0};
  const cudaError_t e = spec_get(c->spec, c->device, p, v, f, msg, sizeof(msg));
  if (e != cudaSuccess)
    return fail(c, PRAD_ERR_CUDA, "push_emit: run-time specialisation: %s (%s)", msg,
                cudaGetErrorString(e));
  return PRAD_OK;
}

template <typename R>
int push_emit_t(prad_ctx* c, const prad_particles* pp, int64_t n,
                int32_t nsteps) {
  StepParams<R> p{};
  fill_common<R>(c, p);
  const void* arrs[6] = {pp->x, pp->y, pp->ux, pp->uy, pp->uz, pp->w};
  for (const void* a : arrs)
    if (!a || !aligned(a, sizeof(R)))
      return fail(c, PRAD_ERR_ARG, "push_emit: null or misaligned particle array");
  if (pp->z && !aligned(pp->z, sizeof(R)))
    return fail(c, PRAD_ERR_ARG, "push_emit: misaligned z");
  if (!pp->z && c->fields.kind != PRAD_FIELD_YEE2D)
    return fail(c, PRAD_ERR_ARG, "push_emit: z may be NULL only for YEE2D");
  p.x = static_cast<R*>(pp->x); p.y = static_cast<R*>(pp->y);
  p.z = static_cast<R*>(pp->z);
  p.ux = static_cast<R*>(pp->ux); p.uy = static_cast<R*>(pp->uy);
  p.uz = static_cast<R*>(pp->uz);
  p.w = static_cast<const R*>(pp->w);
  p.led_emit = c->d_led_emit + pp->ledger_offset;
  p.led_ll = c->d_led_ll + pp->ledger_offset;
  p.led_n = c->cfg.max_particles - pp->ledger_offset;
  p.led_off = pp->ledger_offset;
  p.pid = pp->pid;
  if (pp->pid && !aligned(pp->pid, 4))
    return fail(c, PRAD_ERR_ARG, "push_emit: misaligned pid array");
  p.n = n;
  p.pid0 = pp->pid0;
  const bool tiled = c->fields.kind == PRAD_FIELD_YEE2D && c->cfg.sort_interval > 0 &&
                     pp->pid != nullptr && c->cfg.sampler == PRAD_SAMPLER_TABLE;
  if (tiled) {
    if (n > c->cfg.max_particles)
      return fail(c, PRAD_ERR_ARG, "push_emit: n exceeds max_particles (sort scratch)");
    int ntx, nty;
    tile_counts(c->fields, &ntx, &nty);
    p.ntx = ntx;
    const int interval = c->cfg.sort_interval;
    for (int32_t done = 0; done < nsteps;) {
      const int32_t m = (nsteps - done) < interval ? (nsteps - done) : interval;
      int rc = sort_t<R>(c, pp, n);
      if (rc != PRAD_OK) return rc;
      p.work = c->sort.work;
      p.work_count = c->sort.work_count;
      p.t0 = pp->t0 + done;
      p.nsub = m;
      const int64_t mw = max_work_items(n, c->sort.ntiles);
      if constexpr (sizeof(R) == 4) {
        const SpecFn* spec = nullptr;
        rc = spec_for(c, p, true, &spec);
        if (rc != PRAD_OK) return rc;
        if (spec) {
          CK(c, spec_launch(spec, p, static_cast<int>(mw), 256, c->stream));
          ++c->spec_launches;
          done += m;
          continue;
        }
      }
      CK(c, launch_push_emit_tiled<R>(p, static_cast<int>(mw), 256, c->stream));
      done += m;
    }
    return PRAD_OK;
  }
  // default block: 256 threads, or, when that leaves SMs without a block
  // (n < 256 x SMs), the smallest multiple of 32 that spreads the particles
  // over every SM (FP64 on GB300 runs at a small fraction of the FP32 rate
  // per SM: 10^4 particles take half the time on 105 blocks of 96 threads
  // as on 40 of 256)
  int block = c->cfg.block_size > 0 ? c->cfg.block_size : 256;
  if (c->cfg.block_size <= 0 && n < static_cast<int64_t>(256) * c->num_sms) {
    const int64_t per_sm = (n + c->num_sms - 1) / c->num_sms;
    const int64_t b = (per_sm + 31) / 32 * 32;
    block = static_cast<int>(b < 32 ? 32 : (b > 256 ? 256 : b));
  }
  const int sub = c->cfg.steps_per_launch > 0 ? c->cfg.steps_per_launch : 1;
  const int sub_eff = sub < nsteps ? sub : nsteps;
  // persistent grid: at most the resident blocks of the kernel variant, so
  // no block waits for a second wave (blocks_per_sm = 0: all of them)
  const SpecFn* spec = nullptr;
  if constexpr (sizeof(R) == 4) {
    p.nsub = sub_eff;
    const int rc = spec_for(c, p, false, &spec);
    if (rc != PRAD_OK) return rc;
  }
  const int occ = spec ? spec_occupancy(spec, block)
                       : push_emit_occupancy<R>(p, c->fields.kind, c->cfg.sampler, sub_eff,
                                                block, ctrl_of(c));
  const int bps = c->cfg.blocks_per_sm > 0 && c->cfg.blocks_per_sm < occ ? c->cfg.blocks_per_sm
                                                                         : occ;
  const int64_t want = (n + block - 1) / block;
  const int64_t cap = static_cast<int64_t>(c->num_sms) * bps;
  const int grid = static_cast<int>(want < cap ? want : cap);
  const uint64_t phase0 = p.phase_t0;
  for (int32_t done = 0; done < nsteps;) {
    const int32_t m = (nsteps - done) < sub ? (nsteps - done) : sub;
    p.t0 = pp->t0 + done;
    p.nsub = m;
    // wave phase at the launch's first step (modulo one cycle)
    p.phase_t0 = phase0 + static_cast<uint64_t>(p.t0) * p.phase_step;
    if constexpr (sizeof(R) == 4) {
      if (spec) {
        const int rc = spec_for(c, p, false, &spec);  // the variant of this launch's nsub
        if (rc != PRAD_OK) return rc;
      }
      if (spec) {
        CK(c, spec_launch(spec, p, grid, block, c->stream));
        ++c->spec_launches;
        done += m;
        continue;
      }
    }
    CK(c, launch_push_emit<R>(p, c->fields.kind, c->cfg.sampler, grid, block, c->stream));
    done += m;
  }
  return mlp_finish(c, c->d_led_emit);
}

}  // namespace

extern "C" {

int prad_init(prad_ctx** out, const prad_config* cfg) {
  if (!out || !cfg) return fail(nullptr, PRAD_ERR_ARG, "prad_init: null argument");
  *out = nullptr;
  if (!(cfg->dt > 0.0) || !(cfg->omega_ref > 0.0))
    return fail(nullptr, PRAD_ERR_ARG, "prad_init: dt and omega_ref must be > 0");
  if (cfg->photon_capacity < 1 || cfg->max_particles < 1)
    return fail(nullptr, PRAD_ERR_ARG,
                "prad_init: photon_capacity and max_particles must be >= 1");
  if (cfg->precision != PRAD_FP32 && cfg->precision != PRAD_FP64)
    return fail(nullptr, PRAD_ERR_ARG, "prad_init: bad precision");
  if (cfg->sampler < PRAD_SAMPLER_TABLE || cfg->sampler > PRAD_SAMPLER_MLP_FALLBACK)
    return fail(nullptr, PRAD_ERR_ARG, "prad_init: bad sampler");
  if (cfg->sampler != PRAD_SAMPLER_TABLE && cfg->precision != PRAD_FP32)
    return fail(nullptr, PRAD_ERR_ARG, "prad_init: the learned sampler is FP32 only");
  if (cfg->rr_mode < PRAD_RR_OFF || cfg->rr_mode > PRAD_RR_APPLY)
    return fail(nullptr, PRAD_ERR_ARG, "prad_init: bad rr_mode");
  if (cfg->heff_form != PRAD_HEFF_FIELD && cfg->heff_form != PRAD_HEFF_MOMENTUM)
    return fail(nullptr, PRAD_ERR_ARG, "prad_init: bad heff_form");
  if (cfg->charge != 1.0 && cfg->charge != -1.0)
    return fail(nullptr, PRAD_ERR_ARG, "prad_init: charge must be +1 or -1");
  if (cfg->block_size < 0 || cfg->block_size > 256 || (cfg->block_size % 32) != 0)
    return fail(nullptr, PRAD_ERR_ARG, "prad_init: block_size must be a multiple of 32 <= 256");
  if (cfg->steps_per_launch < 0 || cfg->blocks_per_sm < 0 || cfg->sort_interval < 0)
    return fail(nullptr, PRAD_ERR_ARG, "prad_init: negative launch parameter");
  if (cfg->specialize != 0 && cfg->specialize != 1)
    return fail(nullptr, PRAD_ERR_ARG, "prad_init: specialize must be 0 or 1");
  if (cfg->n_try < 0 || cfg->n_try > 65535)
    return fail(nullptr, PRAD_ERR_ARG, "prad_init: n_try outside [0, 65535]");
  if (cfg->n_try > 1 && cfg->sampler != PRAD_SAMPLER_TABLE)
    return fail(nullptr, PRAD_ERR_ARG, "prad_init: n_try > 1 needs the table sampler");
  if (!(cfg->select_prob >= 0.0 && cfg->select_prob <= 1.0))
    return fail(nullptr, PRAD_ERR_ARG, "prad_init: select_prob outside [0, 1]");
  if (cfg->diagnostics & ~(PRAD_DIAG_WIGGLER | PRAD_DIAG_ANGLE_SPREAD))
    return fail(nullptr, PRAD_ERR_ARG, "prad_init: unknown diagnostics bit");
  if ((cfg->diagnostics & PRAD_DIAG_ANGLE_SPREAD) && cfg->sampler != PRAD_SAMPLER_TABLE)
    return fail(nullptr, PRAD_ERR_ARG,
                "prad_init: PRAD_DIAG_ANGLE_SPREAD needs the table sampler");

  prad_ctx* c = new (std::nothrow) prad_ctx();
  if (!c) return fail(nullptr, PRAD_ERR_ARG, "prad_init: out of host memory");
  c->cfg = *cfg;
  c->stream = static_cast<cudaStream_t>(cfg->stream);
  auto bail = [&](int code) {
    std::snprintf(g_init_err, sizeof(g_init_err), "%s", c->err);
    prad_destroy(c);
    return code;
  };
#define CKI(call)                                                         \
  do {                                                                    \
    cudaError_t e_ = (call);                                              \
    if (e_ != cudaSuccess) {                                              \
      fail(c, PRAD_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));    \
      return bail(PRAD_ERR_CUDA);                                         \
    }                                                                     \
  } while (0)
  CKI(cudaGetDevice(&c->device));
  CKI(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
  c->dtn = cfg->dt * cfg->omega_ref;
  c->alpha = kQe * kQe / (4.0 * kPi * kEps0 * kHbar * kC);
  c->eps_r = kHbar * cfg->omega_ref / (kMe * kC * kC);

  // host tables are built once per process (pure functions of the paper's
  // constants) and uploaded to every context
  static std::once_flag once;
  static std::vector<float4> t32;
  static std::vector<Coef4d> t64;
  static std::vector<float> ginv_host;
  std::call_once(once, [] {
    build_tables(t32, t64);
    build_ginv(ginv_host);
  });
  if (cfg->diagnostics & PRAD_DIAG_ANGLE_SPREAD) {
    const std::vector<float>& ang_host = ang_table_host();
    CKI(cudaMalloc(&c->d_ang, ang_host.size() * sizeof(float)));
    CKI(cudaMemcpy(c->d_ang, ang_host.data(), ang_host.size() * sizeof(float),
                   cudaMemcpyHostToDevice));
  }
  CKI(cudaMalloc(&c->d_tab32, kNTab * sizeof(float4)));
  CKI(cudaMalloc(&c->d_tab64, kNTab * sizeof(Coef4d)));
  CKI(cudaMemcpy(c->d_tab32, t32.data(), kNTab * sizeof(float4), cudaMemcpyHostToDevice));
  CKI(cudaMemcpy(c->d_tab64, t64.data(), kNTab * sizeof(Coef4d), cudaMemcpyHostToDevice));

  const size_t cap = static_cast<size_t>(cfg->photon_capacity);
  for (int k = 0; k < 8; ++k) CKI(cudaMalloc(&c->d_ph[k], cap * sizeof(float)));
  CKI(cudaMalloc(&c->d_pid, cap * sizeof(uint32_t)));
  CKI(cudaMalloc(&c->d_step, cap * sizeof(uint32_t)));
  if (cfg->sampler != PRAD_SAMPLER_TABLE) {
    CKI(cudaMalloc(&c->d_pend, cap * sizeof(float4)));
    c->finish_grid = c->num_sms * mlp_finish_blocks_per_sm();
  }
  // per-CTA busy clocks of batched calls: at most 2048 threads per SM in
  // CTAs of at least 32 threads
  c->batch_busy_n = c->num_sms * 64;
  CKI(cudaMalloc(&c->d_batch_busy, sizeof(unsigned long long) * c->batch_busy_n));
  CKI(cudaMalloc(&c->d_cnt, kNumCounters * sizeof(unsigned long long)));
  CKI(cudaMemset(c->d_cnt, 0, kNumCounters * sizeof(unsigned long long)));
  const size_t np = static_cast<size_t>(cfg->max_particles);
  CKI(cudaMalloc(&c->d_led_emit, np * sizeof(double)));
  CKI(cudaMalloc(&c->d_led_ll, np * sizeof(double)));
  CKI(cudaMemset(c->d_led_emit, 0, np * sizeof(double)));
  CKI(cudaMemset(c->d_led_ll, 0, np * sizeof(double)));
  c->red_blocks = 2 * c->num_sms;
  CKI(cudaMalloc(&c->d_partials, 4 * c->red_blocks * sizeof(double)));
  CKI(cudaMalloc(&c->d_sums, 2 * sizeof(double)));
  // learned sampler: network, optimiser state, G^-1 table
  CKI(cudaMalloc(&c->d_mlp, sizeof(float) * kNumParams));
  CKI(cudaMalloc(&c->d_mlp_m, sizeof(float) * kNumParams));
  CKI(cudaMalloc(&c->d_mlp_v, sizeof(float) * kNumParams));
  CKI(cudaMalloc(&c->d_mlp_grad, sizeof(float) * kNumParams));
  CKI(cudaMalloc(&c->d_mlp_w2, sizeof(uint16_t) * kHid * kHid));
  CKI(cudaMalloc(&c->d_mlp_loss, sizeof(float)));
  CKI(cudaMalloc(&c->d_ginv, sizeof(float) * kGiN));
  {
    CKI(cudaMemcpy(c->d_ginv, ginv_host.data(), sizeof(float) * kGiN, cudaMemcpyHostToDevice));
    std::vector<float> p0;
    init_mlp_params(p0, 0x5eed5eedull);
    if (upload_mlp(c, p0.data()) != PRAD_OK) return bail(PRAD_ERR_CUDA);
  }
  CKI(cudaDeviceSynchronize());
#undef CKI
  *out = c;
  return PRAD_OK;
}

int prad_destroy(prad_ctx* c) {
  if (!c) return PRAD_OK;
  free_sort(c->sort);
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  spec_destroy(c->spec);
  cudaFree(c->d_batch);
  cudaFree(c->d_batch_off);
  cudaFree(c->d_batch_next);
  cudaFree(c->d_batch_busy);
  cudaFree(c->d_tab32);
  cudaFree(c->d_tab64);
  for (int k = 0; k < 8; ++k) cudaFree(c->d_ph[k]);
  cudaFree(c->d_pid);
  cudaFree(c->d_step);
  cudaFree(c->d_pend);
  cudaFree(c->d_hist);
  cudaFree(c->d_cnt);
  cudaFree(c->d_led_emit);
  cudaFree(c->d_led_ll);
  cudaFree(c->d_partials);
  cudaFree(c->d_sums);
  cudaFree(c->d_mlp);
  cudaFree(c->d_mlp_m);
  cudaFree(c->d_mlp_v);
  cudaFree(c->d_mlp_grad);
  cudaFree(c->d_mlp_w2);
  cudaFree(c->d_mlp_loss);
  cudaFree(c->d_ginv);
  cudaFree(c->d_ang);
  cudaFree(c->d_mlp_partial);
  cudaFree(c->d_mlp_loss_part);
  delete c;
  return PRAD_OK;
}

const char* prad_last_error(const prad_ctx* c) { return c ? c->err : g_init_err; }

int prad_set_fields(prad_ctx* c, const prad_fields* f) {
  if (!c || !f) return fail(c, PRAD_ERR_ARG, "set_fields: null argument");
  if (f->kind == PRAD_FIELD_CONST) {
    // nothing to check
  } else if (f->kind == PRAD_FIELD_PLANE_WAVE) {
    if (!(f->lambda > 0.0) || (f->dir != 1 && f->dir != -1) ||
        (f->hand != 1 && f->hand != -1))
      return fail(c, PRAD_ERR_ARG, "set_fields: plane wave needs lambda > 0, dir and hand = +-1");
  } else if (f->kind == PRAD_FIELD_YEE2D) {
    if (f->nx < 4 || f->ny < 4 || !(f->dx > 0.0) || !(f->dy > 0.0))
      return fail(c, PRAD_ERR_ARG, "set_fields: Yee grid needs nx, ny >= 4 and dx, dy > 0");
    if (static_cast<int64_t>(f->nx) * f->ny > (int64_t(1) << 31))
      return fail(c, PRAD_ERR_ARG, "set_fields: Yee grid larger than 2^31 cells");
    for (int k = 0; k < 6; ++k)
      if (!f->yee[k] || !aligned(f->yee[k], 4))
        return fail(c, PRAD_ERR_ARG, "set_fields: null or misaligned Yee plane %d", k);
  } else {
    return fail(c, PRAD_ERR_ARG, "set_fields: bad kind %d", f->kind);
  }
  c->fields = *f;
  c->fields_set = true;
  return PRAD_OK;
}

int prad_push_emit(prad_ctx* c, const prad_particles* p, int64_t n, int32_t nsteps) {
  if (!c || !p) return fail(c, PRAD_ERR_ARG, "push_emit: null argument");
  if (n < 0 || nsteps < 0) return fail(c, PRAD_ERR_ARG, "push_emit: negative size");
  if (!c->fields_set) return fail(c, PRAD_ERR_STATE, "push_emit: fields not set");
  if (n == 0 || nsteps == 0) return PRAD_OK;
  if (n > (int64_t(1) << 32))
    return fail(c, PRAD_ERR_ARG, "push_emit: more than 2^32 particles in one call");
  if (p->ledger_offset < 0 || p->ledger_offset + n > c->cfg.max_particles)
    return fail(c, PRAD_ERR_ARG, "push_emit: ledger range [%lld, %lld) outside max_particles %lld",
                (long long)p->ledger_offset, (long long)(p->ledger_offset + n),
                (long long)c->cfg.max_particles);
  if (p->t0 < 0 || p->t0 + nsteps > (int64_t(1) << 32))
    return fail(c, PRAD_ERR_ARG, "push_emit: step index outside [0, 2^32)");
  if (c->cfg.precision == PRAD_FP32) return push_emit_t<float>(c, p, n, nsteps);
  return push_emit_t<double>(c, p, n, nsteps);
}

int prad_sort_by_tile(prad_ctx* c, const prad_particles* p, int64_t n) {
  if (!c || !p) return fail(c, PRAD_ERR_ARG, "sort_by_tile: null argument");
  if (n < 0) return fail(c, PRAD_ERR_ARG, "sort_by_tile: negative n");
  int rc = check_sort_args(c, p, n);
  if (rc != PRAD_OK) return rc;
  if (n == 0) return PRAD_OK;
  if (c->cfg.precision == PRAD_FP32) return sort_t<float>(c, p, n);
  return sort_t<double>(c, p, n);
}

int prad_get_photons(prad_ctx* c, prad_photons* out, int64_t cap, int64_t* n_out,
                     int64_t* n_dropped, int32_t drain, int32_t out_on_device) {
  if (!c) return fail(c, PRAD_ERR_ARG, "get_photons: null context");
  if (cap < 0) return fail(c, PRAD_ERR_ARG, "get_photons: negative cap");
  if (cap > 0 && !out) return fail(c, PRAD_ERR_ARG, "get_photons: null output");
  unsigned long long cursor = 0;
  CK(c, cudaMemcpyAsync(&cursor, c->d_cnt + kCursor, sizeof(cursor),
                        cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  const int64_t capd = c->cfg.photon_capacity;
  const int64_t held = static_cast<int64_t>(cursor) < capd ? static_cast<int64_t>(cursor) : capd;
  const int64_t dropped = static_cast<int64_t>(cursor) > capd ? static_cast<int64_t>(cursor) - capd : 0;
  const int64_t m = held < cap ? held : cap;
  if (m > 0) {
    const cudaMemcpyKind kind = out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    float* dst[8] = {out->x, out->y, out->z, out->nx, out->ny, out->nz, out->eps, out->weight};
    for (int k = 0; k < 8; ++k)
      if (dst[k]) CK(c, cudaMemcpyAsync(dst[k], c->d_ph[k], m * sizeof(float), kind, c->stream));
    if (out->pid) CK(c, cudaMemcpyAsync(out->pid, c->d_pid, m * sizeof(uint32_t), kind, c->stream));
    if (out->step) CK(c, cudaMemcpyAsync(out->step, c->d_step, m * sizeof(uint32_t), kind, c->stream));
  }
  if (drain) {
    CK(c, cudaMemsetAsync(c->d_cnt + kCursor, 0, sizeof(unsigned long long), c->stream));
    CK(c, cudaMemsetAsync(c->d_cnt + kMlpDone, 0, sizeof(unsigned long long), c->stream));
    c->drained_records += held;
    c->drained_dropped += dropped;
  }
  CK(c, cudaStreamSynchronize(c->stream));
  if (n_out) *n_out = held;
  if (n_dropped) *n_dropped = dropped;
  return PRAD_OK;
}

int prad_angular_histogram(prad_ctx* c, const double axis[3], const double ref[3],
                           int32_t ntheta, int32_t nphi, double theta_max, double* out) {
  if (!c) return fail(c, PRAD_ERR_ARG, "angular_histogram: null context");
  if (!axis || !ref || !out) return fail(c, PRAD_ERR_ARG, "angular_histogram: null pointer");
  if (ntheta < 1 || nphi < 1 || static_cast<int64_t>(ntheta) * nphi > kMaxAngularBins)
    return fail(c, PRAD_ERR_ARG, "angular_histogram: need 1 <= ntheta, nphi and ntheta x nphi <= %d",
                kMaxAngularBins);
  if (!(theta_max > 0.0 && theta_max <= kPi))
    return fail(c, PRAD_ERR_ARG, "angular_histogram: theta_max outside (0, pi]");
  AngularArgs a;
  const double na = std::sqrt(axis[0] * axis[0] + axis[1] * axis[1] + axis[2] * axis[2]);
  if (!(na > 0.0)) return fail(c, PRAD_ERR_ARG, "angular_histogram: zero axis");
  for (int k = 0; k < 3; ++k) a.axis[k] = axis[k] / na;
  const double ra = ref[0] * a.axis[0] + ref[1] * a.axis[1] + ref[2] * a.axis[2];
  double e1[3] = {ref[0] - ra * a.axis[0], ref[1] - ra * a.axis[1], ref[2] - ra * a.axis[2]};
  const double n1 = std::sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
  const double nr = std::sqrt(ref[0] * ref[0] + ref[1] * ref[1] + ref[2] * ref[2]);
  if (!(n1 > 1e-9 * nr)) return fail(c, PRAD_ERR_ARG, "angular_histogram: ref parallel to axis");
  for (int k = 0; k < 3; ++k) a.e1[k] = e1[k] / n1;
  a.e2[0] = a.axis[1] * a.e1[2] - a.axis[2] * a.e1[1];
  a.e2[1] = a.axis[2] * a.e1[0] - a.axis[0] * a.e1[2];
  a.e2[2] = a.axis[0] * a.e1[1] - a.axis[1] * a.e1[0];
  a.theta_max = theta_max;
  a.ntheta = ntheta;
  a.nphi = nphi;
  a.nx = c->d_ph[3]; a.ny = c->d_ph[4]; a.nz = c->d_ph[5];
  a.eps = c->d_ph[6]; a.weight = c->d_ph[7];
  a.cursor = c->d_cnt + kCursor;
  a.cap = c->cfg.photon_capacity;
  if (!c->d_hist) CK(c, cudaMalloc(&c->d_hist, sizeof(double) * kMaxAngularBins));
  a.out = c->d_hist;
  CK(c, launch_angular_hist(a, c->num_sms * 2, c->stream));
  const size_t nb = static_cast<size_t>(ntheta) * nphi;
  CK(c, cudaMemcpyAsync(out, c->d_hist, sizeof(double) * nb, cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  return PRAD_OK;
}

int prad_energy_budget(prad_ctx* c, double* emitted, double* rr_loss, prad_stats* s) {
  if (!c) return fail(c, PRAD_ERR_ARG, "energy_budget: null context");
  CK(c, launch_ledger_reduce(c->d_led_emit, c->d_led_ll, c->cfg.max_particles,
                             c->d_partials, c->red_blocks, c->d_sums, c->stream));
  double sums[2];
  unsigned long long cnt[kNumCounters];
  CK(c, cudaMemcpyAsync(sums, c->d_sums, sizeof(sums), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaMemcpyAsync(cnt, c->d_cnt, sizeof(cnt), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  if (emitted) *emitted = sums[0];
  if (rr_loss) *rr_loss = sums[1];
  if (s) {
    const int64_t capd = c->cfg.photon_capacity;
    const int64_t cur = static_cast<int64_t>(cnt[kCursor]);
    s->records = c->drained_records + (cur < capd ? cur : capd);
    s->dropped = c->drained_dropped + (cur > capd ? cur - capd : 0);
    s->dn_gt1 = static_cast<int64_t>(cnt[kDnGt1]);
    s->clamped = static_cast<int64_t>(cnt[kClamp]);
    s->chi_gt1 = static_cast<int64_t>(cnt[kChiGt1]);
    s->nan_frozen = static_cast<int64_t>(cnt[kNan]);
    s->mlp_fallback = static_cast<int64_t>(cnt[kMlpFallback]);
    s->wiggler_invalid = static_cast<int64_t>(cnt[kWiggler]);
    s->status = static_cast<int32_t>(cnt[kStatus]);
    s->spec_launches = c->spec_launches < INT32_MAX ? static_cast<int32_t>(c->spec_launches)
                                                    : INT32_MAX;
  }
  return s && s->nan_frozen > 0 ? PRAD_WARN_NAN : PRAD_OK;
}

int prad_get_ledger(prad_ctx* c, double* emit, double* ll, int64_t offset, int64_t n,
                    int32_t out_on_device) {
  if (!c) return fail(c, PRAD_ERR_ARG, "get_ledger: null context");
  if (offset < 0 || n < 0 || offset + n > c->cfg.max_particles)
    return fail(c, PRAD_ERR_ARG, "get_ledger: range outside max_particles");
  const cudaMemcpyKind kind = out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (emit && n) CK(c, cudaMemcpyAsync(emit, c->d_led_emit + offset, n * sizeof(double), kind, c->stream));
  if (ll && n) CK(c, cudaMemcpyAsync(ll, c->d_led_ll + offset, n * sizeof(double), kind, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  return PRAD_OK;
}

int prad_reset(prad_ctx* c) {
  if (!c) return fail(c, PRAD_ERR_ARG, "reset: null context");
  const size_t np = static_cast<size_t>(c->cfg.max_particles);
  CK(c, cudaMemsetAsync(c->d_led_emit, 0, np * sizeof(double), c->stream));
  CK(c, cudaMemsetAsync(c->d_led_ll, 0, np * sizeof(double), c->stream));
  CK(c, cudaMemsetAsync(c->d_cnt, 0, kNumCounters * sizeof(unsigned long long), c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  c->drained_records = c->drained_dropped = 0;
  return PRAD_OK;
}

int prad_philox(prad_ctx* c, const uint32_t* ctr, uint32_t k0, uint32_t k1, uint32_t* out,
                int64_t n) {
  if (!c || (n > 0 && (!ctr || !out)) || n < 0) return fail(c, PRAD_ERR_ARG, "philox: bad argument");
  if (n == 0) return PRAD_OK;
  CK(c, launch_philox(ctr, k0, k1, out, n, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  return PRAD_OK;
}

int prad_eval_sampler(prad_ctx* c, const uint32_t* words, void* x_out, void* g_out, int64_t n) {
  if (!c || (n > 0 && (!words || !x_out || !g_out)) || n < 0)
    return fail(c, PRAD_ERR_ARG, "eval_sampler: bad argument");
  if (n == 0) return PRAD_OK;
  if (c->cfg.precision == PRAD_FP32) {
    StepParams<float> p{};
    fill_common<float>(c, p);
    CK(c, launch_eval_sampler<float>(p, words, static_cast<float*>(x_out),
                                     static_cast<float*>(g_out), n, c->stream));
  } else {
    StepParams<double> p{};
    fill_common<double>(c, p);
    CK(c, launch_eval_sampler<double>(p, words, static_cast<double*>(x_out),
                                      static_cast<double*>(g_out), n, c->stream));
  }
  CK(c, cudaStreamSynchronize(c->stream));
  return PRAD_OK;
}

namespace {

uint64_t mix64(uint64_t h, uint64_t v) {
  h ^= v + 0x9E3779B97F4A7C15ull + (h << 6) + (h >> 2);
  return h * 0xBF58476D1CE4E5B9ull;
}

int check_ensemble(prad_ctx* c, const prad_ensemble& e, int k) {
  if (e.n < 0) return fail(c, PRAD_ERR_ARG, "batch: ensemble %d has n < 0", k);
  if (e.field.kind != PRAD_FIELD_CONST && e.field.kind != PRAD_FIELD_PLANE_WAVE)
    return fail(c, PRAD_ERR_ARG, "batch: ensemble %d: only CONST and PLANE_WAVE fields", k);
  if (e.field.kind == PRAD_FIELD_PLANE_WAVE &&
      (!(e.field.lambda > 0.0) || (e.field.dir != 1 && e.field.dir != -1) ||
       (e.field.hand != 1 && e.field.hand != -1)))
    return fail(c, PRAD_ERR_ARG, "batch: ensemble %d: bad plane wave", k);
  if (e.n == 0) return PRAD_OK;
  const prad_particles& p = e.p;
  const void* arrs[7] = {p.x, p.y, p.z, p.ux, p.uy, p.uz, p.w};
  for (const void* a : arrs)
    if (!a || !aligned(a, 4)) return fail(c, PRAD_ERR_ARG, "batch: ensemble %d: null array", k);
  if (p.ledger_offset < 0 || p.ledger_offset + e.n > c->cfg.max_particles)
    return fail(c, PRAD_ERR_ARG, "batch: ensemble %d: ledger range outside max_particles", k);
  if (p.t0 < 0 || e.n > (int64_t(1) << 32)) return fail(c, PRAD_ERR_ARG, "batch: ensemble %d: bad t0/n", k);
  return PRAD_OK;
}

// Fill the per-ensemble parameters and the work-item prefix sums; returns
// the total number of work items.  `led` (optional) replaces the context's
// ledgers (the autotuner books into scratch).
int64_t build_batch(prad_ctx* c, const prad_ensemble* ens, int n_ens, int chunk,
                    std::vector<StepParams<float>>& hp, std::vector<int64_t>& off,
                    double* led_emit = nullptr, double* led_ll = nullptr) {
  hp.resize(n_ens);
  off.resize(n_ens + 1);
  off[0] = 0;
  for (int k = 0; k < n_ens; ++k) {
    const prad_ensemble& e = ens[k];
    StepParams<float>& p = hp[k];
    p = StepParams<float>{};
    fill_common<float>(c, p, e.field);
    p.x = static_cast<float*>(e.p.x); p.y = static_cast<float*>(e.p.y);
    p.z = static_cast<float*>(e.p.z);
    p.ux = static_cast<float*>(e.p.ux); p.uy = static_cast<float*>(e.p.uy);
    p.uz = static_cast<float*>(e.p.uz);
    p.w = static_cast<const float*>(e.p.w);
    p.pid = e.p.pid;
    p.led_base = led_emit ? led_emit : c->d_led_emit;
    p.led_emit = p.led_base + e.p.ledger_offset;
    p.led_ll = (led_ll ? led_ll : c->d_led_ll) + e.p.ledger_offset;
    p.led_n = c->cfg.max_particles - e.p.ledger_offset;
    p.led_off = e.p.ledger_offset;
    p.n = e.n;
    p.pid0 = e.p.pid0;
    p.ensemble = e.ensemble;
    p.t0 = e.p.t0;
    p.phase_t0 = p.phase_t0 + static_cast<uint64_t>(p.t0) * p.phase_step;
    off[k + 1] = off[k] + (e.n + chunk - 1) / chunk;
  }
  return off[n_ens];
}

int upload_batch(prad_ctx* c, const std::vector<StepParams<float>>& hp,
                 const std::vector<int64_t>& off) {
  const int n = static_cast<int>(hp.size());
  if (n > c->batch_cap) {
    cudaFree(c->d_batch);
    cudaFree(c->d_batch_off);
    c->d_batch = nullptr;
    c->d_batch_off = nullptr;
    c->batch_cap = 0;
    CK(c, cudaMalloc(&c->d_batch, sizeof(StepParams<float>) * n));
    CK(c, cudaMalloc(&c->d_batch_off, sizeof(int64_t) * (n + 1)));
    c->batch_cap = n;
  }
  if (!c->d_batch_next) CK(c, cudaMalloc(&c->d_batch_next, sizeof(unsigned long long)));
  c->h_batch = hp;  // keep the host copy alive until the copies complete
  c->h_batch_off = off;
  CK(c, cudaMemcpyAsync(c->d_batch, c->h_batch.data(), sizeof(StepParams<float>) * n,
                        cudaMemcpyHostToDevice, c->stream));
  CK(c, cudaMemcpyAsync(c->d_batch_off, c->h_batch_off.data(), sizeof(int64_t) * (n + 1),
                        cudaMemcpyHostToDevice, c->stream));
  return PRAD_OK;
}

// Issue the launches of one batch call on the stream (memset of the work
// counter + one persistent kernel per steps_per_launch chunk).
int issue_batch(prad_ctx* c, int n_ens, int64_t items, int32_t nsteps, int chunk, int nsub,
                int block, int bps) {
  BatchParams bp;
  bp.ens = c->d_batch;
  bp.item_off = c->d_batch_off;
  bp.next_item = c->d_batch_next;
  bp.total_items = items;
  bp.n_ens = n_ens;
  bp.chunk = chunk;
  bp.pad = 0;
  philox_round_keys(c->cfg.seed, bp.rkey);
  const int cap = batch_max_blocks_per_sm(block, c->cfg.sampler, ctrl_of(c), std_of(c));
  const int64_t g = static_cast<int64_t>(c->num_sms) * (bps < cap ? bps : cap);
  const int grid = static_cast<int>(g < items ? g : (items > 0 ? items : 1));
  // per-CTA busy clocks of this call (load balance), zeroed per call; the
  // array is allocated at init for the largest possible grid, so nothing
  // is allocated here (this may run inside a graph capture)
  bp.busy = nullptr;
  c->batch_grid = 0;
  if (c->d_batch_busy && grid <= c->batch_busy_n) {
    CK(c, cudaMemsetAsync(c->d_batch_busy, 0, sizeof(unsigned long long) * grid, c->stream));
    bp.busy = c->d_batch_busy;
    c->batch_grid = grid;
  }
  for (int32_t done = 0; done < nsteps;) {
    const int32_t m = (nsteps - done) < nsub ? (nsteps - done) : nsub;
    bp.step_base = done;
    bp.nsub = m;
    CK(c, cudaMemsetAsync(c->d_batch_next, 0, sizeof(unsigned long long), c->stream));
    CK(c, launch_push_emit_batch(bp, c->cfg.sampler, ctrl_of(c), std_of(c), grid, block,
                                 c->stream));
    done += m;
  }
  return mlp_finish(c, c->h_batch.empty() ? c->d_led_emit : c->h_batch[0].led_base);
}

int batch_chunk_of(const prad_ctx* c) { return c->cfg.batch_chunk > 0 ? c->cfg.batch_chunk : 2048; }
int batch_nsub_of(const prad_ctx* c, int32_t nsteps) {
  const int s = c->cfg.steps_per_launch > 0 ? c->cfg.steps_per_launch : nsteps;
  return s > 0 ? s : 1;
}

// process-wide cache of tuning results: (GPU, sizes, kinds, probe) -> tuning
std::mutex g_tune_mu;
std::vector<std::pair<uint64_t, prad_tuning>> g_tune_cache;

}  // namespace

int prad_push_emit_batch(prad_ctx* c, const prad_ensemble* ens, int32_t n_ens, int32_t nsteps) {
  if (!c || !ens || n_ens < 1 || nsteps < 0)
    return fail(c, PRAD_ERR_ARG, "push_emit_batch: bad argument");
  if (c->cfg.precision != PRAD_FP32)
    return fail(c, PRAD_ERR_ARG, "push_emit_batch: FP32 only");
  if (c->d_ang)
    return fail(c, PRAD_ERR_ARG, "push_emit_batch: no angular spread in batched calls");
  for (int k = 0; k < n_ens; ++k) {
    int rc = check_ensemble(c, ens[k], k);
    if (rc != PRAD_OK) return rc;
  }
  if (nsteps == 0) return PRAD_OK;
  const int chunk = batch_chunk_of(c);
  const int nsub = batch_nsub_of(c, nsteps);
  const int block = c->cfg.block_size > 0 ? c->cfg.block_size : 256;
  const int bps = c->cfg.blocks_per_sm > 0 ? c->cfg.blocks_per_sm : 3;
  std::vector<StepParams<float>> hp;
  std::vector<int64_t> off;
  const int64_t items = build_batch(c, ens, n_ens, chunk, hp, off);
  int rc = upload_batch(c, hp, off);
  if (rc != PRAD_OK) return rc;
  if (items == 0) return PRAD_OK;
  if (!c->cfg.use_graph) return issue_batch(c, n_ens, items, nsteps, chunk, nsub, block, bps);
  if (c->stream == nullptr)
    return fail(c, PRAD_ERR_ARG, "push_emit_batch: graph capture needs a non-default stream");
  uint64_t key = 0x1234;
  key = mix64(key, static_cast<uint64_t>(n_ens));
  key = mix64(key, static_cast<uint64_t>(items));
  for (int k = 0; k <= n_ens; ++k) key = mix64(key, static_cast<uint64_t>(off[k]));
  key = mix64(key, static_cast<uint64_t>(nsteps));
  key = mix64(key, (static_cast<uint64_t>(chunk) << 32) | static_cast<uint64_t>(nsub));
  key = mix64(key, (static_cast<uint64_t>(block) << 32) | static_cast<uint64_t>(bps));
  key = mix64(key, static_cast<uint64_t>(c->cfg.sampler));
  if (!c->graph_exec || c->graph_key != key) {
    if (c->graph_exec) {
      cudaGraphExecDestroy(c->graph_exec);
      c->graph_exec = nullptr;
    }
    CK(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    rc = issue_batch(c, n_ens, items, nsteps, chunk, nsub, block, bps);
    cudaGraph_t graph = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(c->stream, &graph);
    if (rc != PRAD_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (ee != cudaSuccess) return fail(c, PRAD_ERR_CUDA, "graph capture: %s", cudaGetErrorString(ee));
    const cudaError_t ei = cudaGraphInstantiate(&c->graph_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) return fail(c, PRAD_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ei));
    c->graph_key = key;
  }
  CK(c, cudaGraphLaunch(c->graph_exec, c->stream));
  return PRAD_OK;
}

int prad_autotune_batch(prad_ctx* c, const prad_ensemble* ens, int32_t n_ens, int32_t probe_steps,
                        int64_t sample, prad_tuning* out) {
  if (!c || !ens || n_ens < 1 || probe_steps < 1 || sample < 32)
    return fail(c, PRAD_ERR_ARG, "autotune_batch: bad argument");
  if (c->cfg.precision != PRAD_FP32)
    return fail(c, PRAD_ERR_ARG, "autotune_batch: FP32 only");
  if (c->d_ang)
    return fail(c, PRAD_ERR_ARG, "autotune_batch: no angular spread in batched calls");
  for (int k = 0; k < n_ens; ++k) {
    int rc = check_ensemble(c, ens[k], k);
    if (rc != PRAD_OK) return rc;
  }
  cudaDeviceProp prop;
  CK(c, cudaGetDeviceProperties(&prop, c->device));
  uint64_t key = 0xC0FFEE;
  for (const char* q = prop.name; *q; ++q) key = mix64(key, static_cast<uint64_t>(*q));
  key = mix64(key, static_cast<uint64_t>(probe_steps));
  key = mix64(key, static_cast<uint64_t>(sample));
  key = mix64(key, static_cast<uint64_t>(c->cfg.sampler));
  for (int k = 0; k < n_ens; ++k)
    key = mix64(key, (static_cast<uint64_t>(ens[k].n) << 2) | static_cast<uint64_t>(ens[k].field.kind));
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (const auto& kv : g_tune_cache)
      if (kv.first == key) {
        prad_tuning t = kv.second;
        t.candidates = 0;  // served from the cache
        c->cfg.block_size = t.block_size;
        c->cfg.blocks_per_sm = t.blocks_per_sm;
        c->cfg.batch_chunk = t.batch_chunk;
        c->cfg.steps_per_launch = t.steps_per_launch;
        if (out) *out = t;
        return PRAD_OK;
      }
  }
  // scratch copies of the first min(n, sample) particles of every ensemble
  std::vector<prad_ensemble> se(ens, ens + n_ens);
  int64_t tot = 0;
  std::vector<int64_t> m(n_ens);
  for (int k = 0; k < n_ens; ++k) {
    m[k] = ens[k].n < sample ? ens[k].n : sample;
    tot += m[k];
  }
  float *pristine = nullptr, *work = nullptr;
  double *le = nullptr, *ll = nullptr;
  uint32_t* pids = nullptr;
  auto cleanup = [&]() {
    cudaFree(pristine); cudaFree(work); cudaFree(le); cudaFree(ll); cudaFree(pids);
  };
  const size_t tb = static_cast<size_t>(tot > 0 ? tot : 1);
  if (cudaMalloc(&pristine, 7 * tb * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&work, 7 * tb * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&le, tb * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&ll, tb * sizeof(double)) != cudaSuccess) {
    cleanup();
    return fail(c, PRAD_ERR_CUDA, "autotune_batch: scratch allocation failed");
  }
  int64_t o = 0;
  for (int k = 0; k < n_ens; ++k) {
    void* src[7] = {ens[k].p.x, ens[k].p.y, ens[k].p.z, ens[k].p.ux, ens[k].p.uy, ens[k].p.uz,
                    ens[k].p.w};
    for (int a = 0; a < 7; ++a)
      if (m[k] > 0 && cudaMemcpyAsync(pristine + a * tb + o, src[a], m[k] * sizeof(float),
                                      cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess) {
        cleanup();
        return fail(c, PRAD_ERR_CUDA, "autotune_batch: copy failed");
      }
    prad_ensemble& s = se[k];
    s.n = m[k];
    s.p.x = work + 0 * tb + o; s.p.y = work + 1 * tb + o; s.p.z = work + 2 * tb + o;
    s.p.ux = work + 3 * tb + o; s.p.uy = work + 4 * tb + o; s.p.uz = work + 5 * tb + o;
    s.p.w = work + 6 * tb + o;
    s.p.pid = nullptr;
    s.p.ledger_offset = o;
    o += m[k];
  }
  unsigned long long cursor0 = 0;
  CK(c, cudaMemcpyAsync(&cursor0, c->d_cnt + kCursor, sizeof(cursor0), cudaMemcpyDeviceToHost,
                        c->stream));
  unsigned long long cnt_save[kNumCounters];
  CK(c, cudaMemcpyAsync(cnt_save, c->d_cnt, sizeof(cnt_save), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  prad_tuning best{};
  best.particle_steps_per_s = -1.0;
  int ncand = 0;
  const int blocks[2] = {128, 256};
  const int chunks[4] = {512, 1024, 2048, 4096};
  int rc_all = PRAD_OK;
  for (int bi = 0; bi < 2 && rc_all == PRAD_OK; ++bi) {
    const int block = blocks[bi];
    const int cap = batch_max_blocks_per_sm(block, c->cfg.sampler, ctrl_of(c), std_of(c));
    for (int bps = 2; bps <= cap && bps <= 2 * (256 / block) * 3 && rc_all == PRAD_OK; ++bps) {
      for (int ci = 0; ci < 4 && rc_all == PRAD_OK; ++ci) {
        const int chunk = chunks[ci];
        std::vector<StepParams<float>> hp;
        std::vector<int64_t> off;
        const int64_t items = build_batch(c, se.data(), n_ens, chunk, hp, off, le, ll);
        if ((rc_all = upload_batch(c, hp, off)) != PRAD_OK) break;
        float best_ms = 0.0f;
        for (int rep = 0; rep < 2; ++rep) {  // warm-up, then timed
          cudaMemcpyAsync(work, pristine, 7 * tb * sizeof(float), cudaMemcpyDeviceToDevice,
                          c->stream);
          cudaEventRecord(e0, c->stream);
          if ((rc_all = issue_batch(c, n_ens, items, probe_steps, chunk, probe_steps, block,
                                    bps)) != PRAD_OK)
            break;
          cudaEventRecord(e1, c->stream);
          cudaEventSynchronize(e1);
          cudaEventElapsedTime(&best_ms, e0, e1);
        }
        ++ncand;
        const double rate = tot * static_cast<double>(probe_steps) / (best_ms * 1e-3);
        if (rate > best.particle_steps_per_s) {
          best.block_size = block;
          best.blocks_per_sm = bps;
          best.batch_chunk = chunk;
          best.steps_per_launch = 0;
          best.particle_steps_per_s = rate;
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // restore the counters (photon cursor included: tuning records are
  // overwritten by later appends)
  cudaMemcpyAsync(c->d_cnt, cnt_save, sizeof(cnt_save), cudaMemcpyHostToDevice, c->stream);
  cudaStreamSynchronize(c->stream);
  cleanup();
  (void)cursor0;
  if (rc_all != PRAD_OK) return rc_all;
  best.candidates = ncand;
  c->cfg.block_size = best.block_size;
  c->cfg.blocks_per_sm = best.blocks_per_sm;
  c->cfg.batch_chunk = best.batch_chunk;
  c->cfg.steps_per_launch = best.steps_per_launch;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache.emplace_back(key, best);
  }
  if (out) *out = best;
  return PRAD_OK;
}

int prad_mlp_set_weights(prad_ctx* c, const float* params, int64_t n) {
  if (!c || !params || n != kNumParams)
    return fail(c, PRAD_ERR_ARG, "mlp_set_weights: need %d host floats", kNumParams);
  return upload_mlp(c, params);
}

int prad_mlp_get_weights(prad_ctx* c, float* params, int64_t n) {
  if (!c || !params || n != kNumParams)
    return fail(c, PRAD_ERR_ARG, "mlp_get_weights: need %d host floats", kNumParams);
  CK(c, cudaMemcpyAsync(params, c->d_mlp, sizeof(float) * kNumParams, cudaMemcpyDeviceToHost,
                        c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  return PRAD_OK;
}

namespace {
int ensure_mlp_partials(prad_ctx* c, int nblocks) {
  if (c->mlp_partial_blocks >= nblocks) return PRAD_OK;
  cudaFree(c->d_mlp_partial);
  cudaFree(c->d_mlp_loss_part);
  c->d_mlp_partial = nullptr;
  c->d_mlp_loss_part = nullptr;
  c->mlp_partial_blocks = 0;
  CK(c, cudaMalloc(&c->d_mlp_partial, sizeof(float) * kNumParams * nblocks));
  CK(c, cudaMalloc(&c->d_mlp_loss_part, sizeof(float) * nblocks));
  c->mlp_partial_blocks = nblocks;
  return PRAD_OK;
}

// training-sample ranges (log-uniform gamma and H_eff) and omega_c dt / (H gamma^2)
void mlp_ranges(const prad_ctx* c, float* lng_lo, float* lng_span, float* lnh_lo,
                float* lnh_span, float* wdt_per) {
  *lng_lo = static_cast<float>(std::log(10.0));
  *lng_span = static_cast<float>(std::log(1e4) - std::log(10.0));
  *lnh_lo = static_cast<float>(std::log(1e2));
  *lnh_span = static_cast<float>(std::log(1e6) - std::log(1e2));
  *wdt_per = static_cast<float>(1.5 * kQe / kMe * c->cfg.dt);
}
}  // namespace

int prad_mlp_train(prad_ctx* c, int64_t steps, int32_t batch, float lr, uint64_t seed,
                   float* final_loss) {
  if (!c || steps < 0 || batch < 1 || !(lr > 0.0f))
    return fail(c, PRAD_ERR_ARG, "mlp_train: bad argument");
  const int nblocks = (batch + 127) / 128;
  int rc = ensure_mlp_partials(c, nblocks);
  if (rc != PRAD_OK) return rc;
  float lng_lo, lng_span, lnh_lo, lnh_span, wdt;
  mlp_ranges(c, &lng_lo, &lng_span, &lnh_lo, &lnh_span, &wdt);
  const MlpDev dev = mlp_dev(c);
  for (int64_t s = 0; s < steps; ++s) {
    CK(c, launch_mlp_train_block(dev, static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32),
                                 static_cast<uint64_t>(s) * batch, batch, batch, nullptr,
                                 c->d_ginv, lng_lo, lng_span, lnh_lo, lnh_span, wdt,
                                 c->d_mlp_partial, c->d_mlp_loss_part, nblocks,
                                 c->d_cnt + kStatus, c->stream));
    c->mlp_t += 1;
    const double lr_s = lr * 0.5 * (1.0 + std::cos(kPi * static_cast<double>(s) / steps));
    const float b1t = static_cast<float>(std::pow(0.9, static_cast<double>(c->mlp_t)));
    const float b2t = static_cast<float>(std::pow(0.999, static_cast<double>(c->mlp_t)));
    CK(c, launch_mlp_reduce_adam(c->d_mlp_partial, nblocks, c->d_mlp_loss_part, c->d_mlp_grad,
                                 c->d_mlp, c->d_mlp_m, c->d_mlp_v, c->d_mlp_w2,
                                 static_cast<float>(lr_s), b1t, b2t, 1, c->d_mlp_loss,
                                 1.0f / static_cast<float>(batch), c->stream));
  }
  float loss = 0.0f;
  unsigned long long st = 0;
  CK(c, cudaMemcpyAsync(&loss, c->d_mlp_loss, sizeof(float), cudaMemcpyDeviceToHost,
                        c->stream));
  CK(c, cudaMemcpyAsync(&st, c->d_cnt + kStatus, sizeof(st), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  if (final_loss) *final_loss = loss;
  if (st & 4ull) return fail(c, PRAD_ERR_TIMEOUT, "mlp_train: a tensor-core wait timed out");
  return PRAD_OK;
}

int prad_mlp_grad(prad_ctx* c, const float* samples, int64_t n, float* grad, double* loss) {
  if (!c || !samples || n < 1 || n > (int64_t(1) << 24) || !grad)
    return fail(c, PRAD_ERR_ARG, "mlp_grad: bad argument");
  if (!aligned(samples, 16)) return fail(c, PRAD_ERR_ARG, "mlp_grad: samples not 16-B aligned");
  const int nblocks = static_cast<int>((n + 127) / 128);
  int rc = ensure_mlp_partials(c, nblocks);
  if (rc != PRAD_OK) return rc;
  float lng_lo, lng_span, lnh_lo, lnh_span, wdt;
  mlp_ranges(c, &lng_lo, &lng_span, &lnh_lo, &lnh_span, &wdt);
  CK(c, launch_mlp_train_block(mlp_dev(c), 0, 0, 0, n, n, reinterpret_cast<const float4*>(samples),
                               c->d_ginv, lng_lo, lng_span, lnh_lo, lnh_span, wdt,
                               c->d_mlp_partial, c->d_mlp_loss_part, nblocks,
                               c->d_cnt + kStatus, c->stream));
  CK(c, launch_mlp_reduce_adam(c->d_mlp_partial, nblocks, c->d_mlp_loss_part, c->d_mlp_grad,
                               c->d_mlp, c->d_mlp_m, c->d_mlp_v, c->d_mlp_w2, 0.0f, 0.0f, 0.0f,
                               0, c->d_mlp_loss, 1.0f / static_cast<float>(n), c->stream));
  float l = 0.0f;
  unsigned long long st = 0;
  CK(c, cudaMemcpyAsync(grad, c->d_mlp_grad, sizeof(float) * kNumParams,
                        cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaMemcpyAsync(&l, c->d_mlp_loss, sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaMemcpyAsync(&st, c->d_cnt + kStatus, sizeof(st), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  if (loss) *loss = l;
  if (st & 4ull) return fail(c, PRAD_ERR_TIMEOUT, "mlp_grad: a tensor-core wait timed out");
  return PRAD_OK;
}

int prad_mlp_eval(prad_ctx* c, const float* in, float* lnx, int64_t n) {
  if (!c || n < 0 || (n > 0 && (!in || !lnx))) return fail(c, PRAD_ERR_ARG, "mlp_eval: bad argument");
  if (n == 0) return PRAD_OK;
  CK(c, launch_mlp_eval(mlp_dev(c), in, lnx, n, c->d_cnt + kStatus, 0, c->stream));
  unsigned long long st = 0;
  CK(c, cudaMemcpyAsync(&st, c->d_cnt + kStatus, sizeof(st), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  if (st & 4ull) return fail(c, PRAD_ERR_TIMEOUT, "mlp_eval: a tensor-core wait timed out");
  return PRAD_OK;
}

int prad_mlp_wait_selftest(prad_ctx* c) {
  if (!c) return fail(c, PRAD_ERR_ARG, "mlp_wait_selftest: null context");
  // one tile of inputs and a status word of its own (the context's status
  // is not touched)
  constexpr int64_t n = 128;
  float* buf = nullptr;
  unsigned long long* st_d = nullptr;
  CK(c, cudaMalloc(&buf, sizeof(float) * 4 * n));
  cudaError_t e = cudaMalloc(&st_d, sizeof(unsigned long long));
  if (e != cudaSuccess) {
    cudaFree(buf);
    return fail(c, PRAD_ERR_CUDA, cudaGetErrorString(e));
  }
  std::vector<float> in(3 * n);
  for (int64_t i = 0; i < n; ++i) {
    in[3 * i] = (static_cast<float>(i) + 0.5f) / n;
    in[3 * i + 1] = 100.0f;
    in[3 * i + 2] = 1.0f;
  }
  unsigned long long st = 0;
  e = cudaMemcpyAsync(buf, in.data(), sizeof(float) * 3 * n, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(st_d, 0, sizeof(unsigned long long), c->stream);
  if (e == cudaSuccess) e = launch_mlp_eval(mlp_dev(c), buf, buf + 3 * n, n, st_d, 1, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&st, st_d, sizeof(st), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(buf);
  cudaFree(st_d);
  if (e != cudaSuccess) return fail(c, PRAD_ERR_CUDA, cudaGetErrorString(e));
  if (st & 4ull) return fail(c, PRAD_ERR_TIMEOUT, "mlp_wait_selftest: the bounded waits ran out");
  return fail(c, PRAD_ERR_STATE, "mlp_wait_selftest: the withheld waits did not report");
}

int prad_batch_balance(prad_ctx* c, double* efficiency, int32_t* ctas) {
  if (!c || !efficiency) return fail(c, PRAD_ERR_ARG, "batch_balance: null argument");
  if (c->batch_grid < 1 || !c->d_batch_busy)
    return fail(c, PRAD_ERR_STATE, "batch_balance: no batched call yet");
  std::vector<unsigned long long> busy(static_cast<size_t>(c->batch_grid));
  CK(c, cudaMemcpyAsync(busy.data(), c->d_batch_busy, sizeof(unsigned long long) * busy.size(),
                        cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  double sum = 0.0, mx = 0.0;
  for (unsigned long long b : busy) {
    sum += static_cast<double>(b);
    mx = static_cast<double>(b) > mx ? static_cast<double>(b) : mx;
  }
  *efficiency = mx > 0.0 ? sum / (mx * static_cast<double>(busy.size())) : 0.0;
  if (ctas) *ctas = c->batch_grid;
  return PRAD_OK;
}

int prad_angle_eval(prad_ctx* c, const float* x, const uint32_t* words, float* psi, int64_t n) {
  if (!c || n < 0 || (n > 0 && (!x || !words || !psi)))
    return fail(c, PRAD_ERR_ARG, "angle_eval: bad argument");
  if (!c->d_ang)
    return fail(c, PRAD_ERR_STATE, "angle_eval: context created without PRAD_DIAG_ANGLE_SPREAD");
  if (n == 0) return PRAD_OK;
  CK(c, launch_angle_eval(c->d_ang, x, words, psi, n, c->stream));
  return PRAD_OK;
}

int prad_angle_table(float* out, int64_t n) {
  if (!out || n < static_cast<int64_t>(kAngNL) * kAngNV)
    return fail(nullptr, PRAD_ERR_ARG, "angle_table: need %d floats", kAngNL * kAngNV);
  const std::vector<float>& t = ang_table_host();
  std::memcpy(out, t.data(), t.size() * sizeof(float));
  return PRAD_OK;
}

int prad_ginv_eval(prad_ctx* c, const float* r, float* lnx, int64_t n) {
  if (!c || n < 0 || (n > 0 && (!r || !lnx))) return fail(c, PRAD_ERR_ARG, "ginv_eval: bad argument");
  if (n == 0) return PRAD_OK;
  CK(c, launch_ginv_eval(c->d_ginv, r, lnx, n, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  return PRAD_OK;
}

}  // extern "C"
