// Fused per-step particle kernel: field gather, Boris push, effective field,
// omega_c, Monte Carlo synchrotron emission with the S(x) proposal, photon
// append and the FP64 emitted-energy / Landau-Lifshitz ledger
// (arXiv:1409.5574, Numerical implementation section, Eqs. (1), (4), (7)-(13)).
//
// One thread owns one particle for `nsub` consecutive steps; its state stays
// in registers between substeps and is read and written once per launch
// (SoA, fully coalesced 4- or 8-byte accesses).  The grid is a multiple of the
// SM count and strides over the particles.
#ifndef __CUDACC_RTC__
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>
#endif


#include "mlp_device.cuh"
#include "prad_internal.h"

namespace prad {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11), written from the published
// definition: ten rounds of two 32x32->64 multiplies and xors, key bumped by
// the Weyl constants after every round.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// The same generator with the ten round keys given (rk[2r], rk[2r + 1]):
// with rk in the kernel's parameter space each round's XOR with the key
// reads it from there instead of carrying the key schedule in registers, and
// each product is one 32 x 32 -> 64-bit multiply (hi and lo words at once).
// ZeroTag: counter word 2 is 0, and so is word 2 after the first round; the
// products of those words are left to the compiler, which folds them (the
// table-sampler kernels gain from it, the learned sampler's does not).
template <bool ZeroTag = false>
__device__ __forceinline__ uint4 philox10_rk(uint4 c, const uint32_t* rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint64_t p0, p1;
    asm("mul.wide.u32 %0, %1, %2;" : "=l"(p0) : "r"(c.x), "r"(0xD2511F53u));
    if (ZeroTag && r < 2)
      p1 = static_cast<uint64_t>(c.z) * 0xCD9E8D57ull;
    else
      asm("mul.wide.u32 %0, %1, %2;" : "=l"(p1) : "r"(c.z), "r"(0xCD9E8D57u));
    const uint32_t lo0 = static_cast<uint32_t>(p0), hi0 = static_cast<uint32_t>(p0 >> 32);
    const uint32_t lo1 = static_cast<uint32_t>(p1), hi1 = static_cast<uint32_t>(p1 >> 32);
    c = make_uint4(hi1 ^ c.y ^ rk[2 * r], lo1, hi0 ^ c.w ^ rk[2 * r + 1], lo0);
  }
  return c;
}

// The same generator for the counter (pid, step, 0, ens) of the table
// sampler, in two parts.  With word 2 zero, round 0's second product is 0
// and its first depends on pid only; after round 1, words 0 and 1 depend on
// (pid, ens) only, and so does round 2's first product.  philox_pre computes
// those four words once per particle; philox10_pre finishes the block for a
// step (two products fewer than philox10_rk), with the same result.
struct PhiloxPre {
  uint32_t w0, y1, h2, l2;
};
__device__ __forceinline__ PhiloxPre philox_pre(uint32_t pid, uint32_t ens, const uint32_t* rk) {
  uint64_t p;
  PhiloxPre q;
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(p) : "r"(pid), "r"(0xD2511F53u));
  const uint32_t z0 = static_cast<uint32_t>(p >> 32) ^ ens ^ rk[1];  // round 0, word 2
  q.w0 = static_cast<uint32_t>(p);                                   // round 0, word 3
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(p) : "r"(z0), "r"(0xCD9E8D57u));
  const uint32_t x1 = static_cast<uint32_t>(p >> 32) ^ rk[2];        // round 1, word 0
  q.y1 = static_cast<uint32_t>(p);                                   // round 1, word 1
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(p) : "r"(x1), "r"(0xD2511F53u));
  q.h2 = static_cast<uint32_t>(p >> 32);                             // round 2, first product
  q.l2 = static_cast<uint32_t>(p);
  return q;
}
__device__ __forceinline__ uint4 philox10_pre(const PhiloxPre& q, uint32_t step,
                                              const uint32_t* rk) {
  uint64_t a, b;
  const uint32_t x0 = step ^ rk[0];  // round 0, word 0 (word 1 is 0)
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(a) : "r"(x0), "r"(0xD2511F53u));
  const uint32_t z1 = static_cast<uint32_t>(a >> 32) ^ q.w0 ^ rk[3];  // round 1, word 2
  const uint32_t w1 = static_cast<uint32_t>(a);                       // round 1, word 3
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(b) : "r"(z1), "r"(0xCD9E8D57u));
  uint4 c = make_uint4(static_cast<uint32_t>(b >> 32) ^ q.y1 ^ rk[4], static_cast<uint32_t>(b),
                       q.h2 ^ w1 ^ rk[5], q.l2);  // after round 2
#pragma unroll
  for (int r = 3; r < 10; ++r) {
    uint64_t p0, p1;
    asm("mul.wide.u32 %0, %1, %2;" : "=l"(p0) : "r"(c.x), "r"(0xD2511F53u));
    asm("mul.wide.u32 %0, %1, %2;" : "=l"(p1) : "r"(c.z), "r"(0xCD9E8D57u));
    const uint32_t lo0 = static_cast<uint32_t>(p0), hi0 = static_cast<uint32_t>(p0 >> 32);
    const uint32_t lo1 = static_cast<uint32_t>(p1), hi1 = static_cast<uint32_t>(p1 >> 32);
    c = make_uint4(hi1 ^ c.y ^ rk[2 * r], lo1, hi0 ^ c.w ^ rk[2 * r + 1], lo0);
  }
  return c;
}

// ---- compensated accumulators for the per-particle ledgers -----------------
// The FP32 path sums a launch's ledger increments in a float-float pair
// (Knuth TwoSum: the rounding error of every add is kept in `lo`), about
// 48 bits, and adds the pair to the FP64 ledger once per launch.  This keeps
// the slow FP64 pipe out of the per-step loop.  The FP64 path accumulates in
// double directly.
template <typename R>
struct Acc;
template <>
struct Acc<float> {
  float hi = 0.0f, lo = 0.0f;
  // _rn intrinsics: never contracted into an FMA with the product that
  // forms v, so TwoSum stays exact and the sum does not depend on how the
  // compiler schedules the surrounding kernel
  __device__ __forceinline__ void add(float v) {
    const float s = __fadd_rn(hi, v);
    const float bb = __fsub_rn(s, hi);
    lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(v, bb)));
    hi = s;
  }
  // FP64 value; a single add (one step per launch) leaves lo == 0 and costs
  // one conversion on the slow FP64 pipe instead of two plus an add
  __device__ __forceinline__ double value() const {
    double v = static_cast<double>(hi);
    if (lo != 0.0f) v += static_cast<double>(lo);
    return v;
  }
  __device__ __forceinline__ bool nonzero() const { return hi != 0.0f; }
  // after exactly one add, TwoSum leaves lo == 0: one conversion
  __device__ __forceinline__ double value_one() const { return static_cast<double>(hi); }
};
template <>
struct Acc<double> {
  double hi = 0.0;
  __device__ __forceinline__ void add(double v) { hi = __dadd_rn(hi, v); }
  __device__ __forceinline__ double value() const { return hi; }
  __device__ __forceinline__ double value_one() const { return hi; }
  __device__ __forceinline__ bool nonzero() const { return hi != 0.0; }
};

// ---- precision-generic helpers --------------------------------------------
// (w + 1/2) 2^-32: a Philox word as a uniform in (0, 1)
template <typename R>
__device__ __forceinline__ R unit_uniform(uint32_t w);
template <>
__device__ __forceinline__ float unit_uniform<float>(uint32_t w) {
  return fmaf(static_cast<float>(w), 0x1p-32f, 0x1p-33f);
}
template <>
__device__ __forceinline__ double unit_uniform<double>(uint32_t w) {
  return fma(static_cast<double>(w), 0x1p-32, 0x1p-33);
}
// psi = gamma theta of the emission's angular spread (Eqs. (5)-(6)) at x,
// from the table (prad_internal.h): the uniform u = (w0 + 1/2) 2^-32 of the
// one-sided CDF, the sign from bit 31 of w1.  v = sqrt(-ln(1 - u)) is taken
// as sqrt(-log1p(-u)) below u = 1/2 and from 1 - u = (~w0 + 1/2) 2^-32
// (exact) above it.  FP32 throughout (the table's accuracy, ~2e-4 in psi,
// is the limit).
template <typename R>
__device__ __forceinline__ R ang_psi(const float* __restrict__ tab, R x, uint32_t w0,
                                     uint32_t w1) {
  const float xf = static_cast<float>(x);
  const float lx = logf(xf);
  float fi = (lx - static_cast<float>(kAngLx0)) *
             static_cast<float>((kAngNL - 1) / (kAngLx1 - kAngLx0));
  fi = fminf(fmaxf(fi, 0.0f), static_cast<float>(kAngNL - 1));
  const int i = min(static_cast<int>(fi), kAngNL - 2);
  const float ti = fi - static_cast<float>(i);
  const float w = w0 < 0x80000000u
                      ? -log1pf(-fmaf(static_cast<float>(w0), 0x1p-32f, 0x1p-33f))
                      : -logf(fmaf(static_cast<float>(~w0), 0x1p-32f, 0x1p-33f));
  const float v = sqrtf(fmaxf(w, 0.0f));
  const float fj = fminf(v * static_cast<float>((kAngNV - 1) / kAngVmax),
                         static_cast<float>(kAngNV - 1));
  const int j = min(static_cast<int>(fj), kAngNV - 2);
  const float tj = fj - static_cast<float>(j);
  const float* r0 = tab + i * kAngNV + j;
  const float* r1 = r0 + kAngNV;
  const float y0 = fmaf(tj, __ldg(r0 + 1) - __ldg(r0), __ldg(r0));
  const float y1 = fmaf(tj, __ldg(r1 + 1) - __ldg(r1), __ldg(r1));
  const float y = fmaf(ti, y1 - y0, y0);
  // s(x) = (2/x)^(1/3) (1 + x)^(-1/6)
  const float sc = expf((0.693147181f - lx) * (1.0f / 3.0f) - log1pf(xf) * (1.0f / 6.0f));
  const float psi = y * v * sc;
  return static_cast<R>((w1 & 0x80000000u) ? -psi : psi);
}

__device__ __forceinline__ void sincos_r(float v, float* s, float* c) { sincosf(v, s, c); }
__device__ __forceinline__ void sincos_r(double v, double* s, double* c) { sincos(v, s, c); }

__device__ __forceinline__ float rsq(float v) { return rsqrtf(v); }
__device__ __forceinline__ double rsq(double v) { return rsqrt(v); }
__device__ __forceinline__ float rcp(float v) { return __fdividef(1.0f, v); }
__device__ __forceinline__ double rcp(double v) { return 1.0 / v; }
// v * rsqrt(v): one MUFU op instead of the IEEE square root (2 ulp), with
// sqr(0) = 0
__device__ __forceinline__ float sqr(float v) { return v > 0.0f ? v * rsqrtf(v) : 0.0f; }
__device__ __forceinline__ double sqr(double v) { return sqrt(v); }
// the same for an argument known to be >= 1 (1 + |u|^2): no zero guard (a
// non-finite argument belongs to a frozen particle, which is never stored)
__device__ __forceinline__ float sqr_pos(float v) { return v * rsqrtf(v); }
__device__ __forceinline__ double sqr_pos(double v) { return sqrt(v); }
__device__ __forceinline__ float flr(float v) { return floorf(v); }
__device__ __forceinline__ double flr(double v) { return floor(v); }
__device__ __forceinline__ float rnd_int(float v) { return rintf(v); }
__device__ __forceinline__ double rnd_int(double v) { return rint(v); }
// sin/cos of pi v for v in [-1, 1] (the caller reduces the phase exactly to
// half a cycle first): the MUFU sin/cos, absolute error ~2^-21.
__device__ __forceinline__ void sincos_pi(float v, float* s, float* c) {
  __sincosf(3.14159265358979323846f * v, s, c);
}
__device__ __forceinline__ void sincos_pi(double v, double* s, double* c) {
  sincospi(v, s, c);
}
// sin/cos of 2 pi v: the same values as sincos_pi(v + v) (2 v and the float
// 2 pi = 2 x the float pi are exact), one instruction fewer
__device__ __forceinline__ void sincos_2pi(float v, float* s, float* c) {
  __sincosf((2.0f * 3.14159265358979323846f) * v, s, c);
}
__device__ __forceinline__ void sincos_2pi(double v, double* s, double* c) {
  sincospi(v + v, s, c);
}

// ---------------------------------------------------------------------------
// Step 8 sampler.  From one Philox block: the proposal frequency
// x = P^-1(R') of Eqs. (11)-(12) and g = F(x) / S(x) from the table.
//   W = w1 2^32 + w0;  R' = (W + 1/2) 2^-64;  1 - R' = (~W + 1/2) 2^-64.
//   low branch  (W < thr, i.e. R' < a^(4/3)):  x = R'^(3/4),  t = R'^(1/4)
//   high branch:                               x = -ln((9/7)(1 - R'))
// The branch is an integer compare, identical in every precision.  Both
// branches share one log2, so the warp does not diverge.
// ---------------------------------------------------------------------------
// STAB: the table is read from a copy in shared memory (stab) instead of
// through L1 from global memory.
template <bool STAB = false>
__device__ __forceinline__ void sample_x_g(const StepParams<float>& P,
                                           uint32_t w0, uint32_t w1, float& x,
                                           float& g, const float4* stab = nullptr) {
  const uint64_t W = (static_cast<uint64_t>(w1) << 32) | w0;
  const bool low = W < kThr;
  const uint32_t h = low ? w1 : ~w1;
  const uint32_t l = low ? w0 : ~w0;
  // (h 2^32 + l + 1/2) 2^-64, never zero
  const float arg = fmaf(static_cast<float>(h), 0x1p-32f,
                         fmaf(static_cast<float>(l), 0x1p-64f, 0x1p-65f));
  // low branch: t = R'^(1/4) = rsqrt(rsqrt(R')) keeps the relative accuracy
  // of R' down to 2^-65 (a float log2 / exp2 route loses it for tiny R');
  // high branch: x = -ln(9/7) - ln(1 - R'), where a relative log2 error is
  // harmless because x >= a
  const float t = rsqrtf(rsqrtf(arg));
  const float x_lo = t * t * t;
  const float x_hi = fmaf(-__log2f(arg), 0.69314718055994531f, -0.25131442828090608f);
  x = low ? x_lo : x_hi;
  const float u = low ? t * static_cast<float>(kTScale)
                      : (x_hi - static_cast<float>(kA)) * static_cast<float>(kXScale);
  int i = static_cast<int>(fmaxf(u, 0.0f));
  const int nmax = low ? kN1 - 1 : kN2 - 1;
  i = min(i, nmax);
  const float s = u - static_cast<float>(i);
  const int ti = low ? i : kN1 + i;
  float4 c;
  if constexpr (STAB) c = stab[ti]; else c = __ldg(P.tab + ti);
  g = fmaf(s, fmaf(s, fmaf(s, c.w, c.z), c.y), c.x);
}

template <bool STAB = false>
__device__ __forceinline__ void sample_x_g(const StepParams<double>& P,
                                           uint32_t w0, uint32_t w1, double& x,
                                           double& g, const Coef4d* = nullptr) {
  static_assert(!STAB, "the FP64 table is read from global memory");
  const uint64_t W = (static_cast<uint64_t>(w1) << 32) | w0;
  const bool low = W < kThr;
  double u;
  if (low) {
    const double Rp = fma(static_cast<double>(W), 0x1p-64, 0x1p-65);
    const double L = log2(Rp);
    const double t = exp2(0.25 * L);
    x = exp2(0.75 * L);
    u = t * kTScale;
  } else {
    const double om = fma(static_cast<double>(~W), 0x1p-64, 0x1p-65);
    x = -(log(om) + 0.25131442828090608);
    u = (x - kA) * kXScale;
  }
  int i = static_cast<int>(fmax(u, 0.0));
  i = min(i, low ? kN1 - 1 : kN2 - 1);
  const double s = u - static_cast<double>(i);
  const Coef4d c = P.tab[low ? i : kN1 + i];
  g = fma(s, fma(s, fma(s, c.c3, c.c2), c.c1), c.c0);
}

// ---------------------------------------------------------------------------
// Step 1 field gather.
// ---------------------------------------------------------------------------
template <typename R>
struct EB {
  R Ex, Ey, Ez, Bx, By, Bz;
};

// Circularly polarised plane wave along dir * x (unit c):
//   E = E0 (0, cos phi, hand sin phi),  B = dir x_hat x E,
//   phi = omega t - dir k x + phase0.
// The time part of the phase is a 64-bit fixed-point fraction of a cycle
// (exact modular arithmetic), so only the x k term carries rounding.
template <typename R>
__device__ __forceinline__ void plane_wave_sc(const StepParams<R>& P, R x, uint64_t phase,
                                              R* s, R* c) {
  R psi_t;
  if constexpr (sizeof(R) == 4)
    psi_t = static_cast<float>(static_cast<uint32_t>(phase >> 32)) * 0x1p-32f;
  else
    psi_t = static_cast<double>(phase >> 11) * 0x1p-53;
  // k x / 2pi in float-float: exact product error (fma) plus the low part
  // of k/2pi; the whole cycles are removed from the high part exactly, so
  // the phase keeps ~1e-7-cycle accuracy at any |x|
  const R p_hi = P.kc * x;
  const R p_lo = fma(P.kc, x, -p_hi) + P.kc_lo * x;
  R psi = (psi_t - (p_hi - rnd_int(p_hi))) - p_lo;
  psi -= rnd_int(psi);
  sincos_2pi(psi, s, c);
}
template <typename R>
__device__ __forceinline__ EB<R> plane_wave(const StepParams<R>& P, R x,
                                            uint64_t phase) {
  R s, c;
  plane_wave_sc(P, x, phase, &s, &c);
  EB<R> f;
  f.Ex = R(0);
  f.Ey = P.E0 * c;
  f.Ez = P.pw_ez * s;  // hand E0 sin: the signs are exact factors
  f.Bx = R(0);
  f.By = P.pw_by * s;  // -dir E_z
  f.Bz = P.pw_bz * c;  // dir E_y
  return f;
}
// The sign variant of a plane wave (1..4): 1 + [hand > 0] + 2 [dir > 0].
template <typename R>
__host__ __device__ __forceinline__ int pw_signs(const StepParams<R>& p) {
  return 1 + (p.hand > R(0) ? 1 : 0) + (p.dir > R(0) ? 2 : 0);
}
// The same with the handedness and direction known at compile time
// (PWS = 1 + [hand > 0] + 2 [dir > 0]): E_z, B_y and B_z are sign changes of
// E0 sin and E_y, the same values from two products instead of four.
template <int PWS, typename R>
__device__ __forceinline__ EB<R> plane_wave_signed(const StepParams<R>& P, R x,
                                                   uint64_t phase) {
  constexpr bool hpos = ((PWS - 1) & 1) != 0, dpos = ((PWS - 1) & 2) != 0;
  R s, c;
  plane_wave_sc(P, x, phase, &s, &c);
  const R es = P.E0 * s;
  EB<R> f;
  f.Ex = R(0);
  f.Ey = P.E0 * c;
  f.Ez = hpos ? es : -es;
  f.Bx = R(0);
  f.By = dpos ? -f.Ez : f.Ez;
  f.Bz = dpos ? f.Ey : -f.Ey;
  return f;
}

// Cell coordinate of a position along one axis, split into the integer cell
// c in [0, n] and the offset f in [0, 1] within it.  (x - x0) / dx is formed
// in float-float (TwoSum of the difference, exact product error by fma, low
// part of 1/dx), so f keeps ~1e-7 cell accuracy even thousands of cells
// from the origin, where a plain FP32 product would be off by ~2e-4 cell.
// Periodic wrap; NaN and far-out values are clamped into the grid, so every
// stencil index derived from c stays in [-1, n + 1].
template <typename R>
struct Cell {
  int c;
  R f;
};

template <typename R>
__device__ __forceinline__ Cell<R> cell_of(R x, R x0, R inv, R inv_lo, int n) {
  const R d_hi = x - x0;
  const R bb = d_hi - x;
  const R d_lo = (x - (d_hi - bb)) - (x0 + bb);  // exact: x - x0 = d_hi + d_lo
  const R hi = d_hi * inv;
  const R lo = fma(d_hi, inv, -hi) + (d_hi * inv_lo + d_lo * inv);
  const R nr = static_cast<R>(n);
  R c = flr(hi);
  R f = (hi - c) + lo;             // hi - c is exact
  c -= nr * flr(c * (R(1) / nr));  // wrap the integer part
  const R fl = flr(f);             // f may leave [0,1) by the lo correction
  c += fl;
  f -= fl;
  c = c < R(0) ? c + nr : (c >= nr ? c - nr : c);
  Cell<R> r;
  const bool ok = c >= R(0) && c < nr && f >= R(0) && f <= R(1);
  r.c = ok ? static_cast<int>(c) : 0;
  r.f = ok ? f : R(0);
  return r;
}

// Quadratic-spline (second-order) weights about the nearest node for the
// offset t of a staggered component (t = f - shift, in [-1/2, 1]); returns
// the nearest node relative to the cell (0 or 1, or -... never below -1).
template <typename R>
__device__ __forceinline__ int qs_weights(R t, R w[3]) {
  const R nr = flr(t + R(0.5));
  const R d = t - nr;
  w[0] = R(0.5) * (R(0.5) - d) * (R(0.5) - d);
  w[1] = R(0.75) - d * d;
  w[2] = R(0.5) * (R(0.5) + d) * (R(0.5) + d);
  return static_cast<int>(nr);
}

// The quadratic-spline stencil of one axis for the two staggerings a
// component can have (node-centred and half-cell-shifted): weights and the
// three periodic node indices of each.
template <typename R>
struct AxisStencil {
  R w0[3], wh[3];
  int i0[3], ih[3];
};

template <typename R>
__device__ __forceinline__ AxisStencil<R> axis_stencil(const Cell<R>& c, int n) {
  AxisStencil<R> a;
  const int b0 = c.c + qs_weights(c.f, a.w0) - 1;
  const int bh = c.c + qs_weights(c.f - R(0.5), a.wh) - 1;
#pragma unroll
  for (int k = 0; k < 3; ++k) {  // periodic (b in [-1, n])
    int i = b0 + k, j = bh + k;
    i = i < 0 ? i + n : (i >= n ? i - n : i);
    j = j < 0 ? j + n : (j >= n ? j - n : j);
    a.i0[k] = i;
    a.ih[k] = j;
  }
  return a;
}

template <typename R>
__device__ __forceinline__ R yee_interp(const StepParams<R>& P, const float* __restrict__ F,
                                        const R wx[3], const int ii[3], const R wy[3],
                                        const int jj[3]) {
  R v = R(0);
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const float* row = F + static_cast<size_t>(jj[b]) * P.nx;
    R r = wx[0] * R(__ldg(row + ii[0])) + wx[1] * R(__ldg(row + ii[1])) +
          wx[2] * R(__ldg(row + ii[2]));
    v += wy[b] * r;
  }
  return v;
}

// 2D Yee grid: Ex (i+1/2, j), Ey (i, j+1/2), Ez (i, j), Bx (i, j+1/2),
// By (i+1/2, j), Bz (i+1/2, j+1/2).
template <typename R>
__device__ __forceinline__ EB<R> yee2d_cells(const StepParams<R>& P, const Cell<R>& cx,
                                             const Cell<R>& cy) {
  const AxisStencil<R> ax = axis_stencil(cx, P.nx);
  const AxisStencil<R> ay = axis_stencil(cy, P.ny);
  EB<R> f;
  f.Ex = yee_interp(P, P.yee[0], ax.wh, ax.ih, ay.w0, ay.i0);
  f.Ey = yee_interp(P, P.yee[1], ax.w0, ax.i0, ay.wh, ay.ih);
  f.Ez = yee_interp(P, P.yee[2], ax.w0, ax.i0, ay.w0, ay.i0);
  f.Bx = yee_interp(P, P.yee[3], ax.w0, ax.i0, ay.wh, ay.ih);
  f.By = yee_interp(P, P.yee[4], ax.wh, ax.ih, ay.w0, ay.i0);
  f.Bz = yee_interp(P, P.yee[5], ax.wh, ax.ih, ay.wh, ay.ih);
  return f;
}

template <typename R>
__device__ __forceinline__ EB<R> yee2d(const StepParams<R>& P, R x, R y) {
  const Cell<R> cx = cell_of(x, P.x0, P.inv_dx, P.inv_dx_lo, P.nx);
  const Cell<R> cy = cell_of(y, P.y0, P.inv_dy, P.inv_dy_lo, P.ny);
  return yee2d_cells(P, cx, cy);
}

template <typename R, int FIELD>
__device__ __forceinline__ EB<R> gather(const StepParams<R>& P, R x, R y,
                                        uint64_t phase) {
  if constexpr (FIELD == PRAD_FIELD_CONST) {
    EB<R> f;
    f.Ex = P.E[0]; f.Ey = P.E[1]; f.Ez = P.E[2];
    f.Bx = P.B[0]; f.By = P.B[1]; f.Bz = P.B[2];
    return f;
  } else if constexpr (FIELD == PRAD_FIELD_PLANE_WAVE) {
    return plane_wave(P, x, phase);
  } else {
    return yee2d(P, x, y);
  }
}

// ---------------------------------------------------------------------------
// Photon append, staged per warp in shared memory.  Emitting lanes write
// their record into the warp's staging buffer at positions given by a ballot
// prefix count; when the buffer would overflow (and at the end of the
// kernel) the warp reserves a contiguous run of slots with ONE atomicAdd and
// copies the buffer out with coalesced stores.  The atomic's round trip is
// paid once per ~kStage records instead of once per emitting warp-step.
// Slots at or beyond the capacity are not written (they count as dropped:
// dropped = cursor - capacity).
// ---------------------------------------------------------------------------
constexpr int kStage = 64;
constexpr int kMaxWarps = 8;  // 256 threads per block at most

// Two layouts of the staging buffer.  Fields (SoA): one 32-bit store per
// field and record; it keeps the fewest registers live, which the batched,
// tiled and control kernels need.  Records (AoS): record r in three 16-byte
// vectors, (x, y, z, u_x), (u_y, u_z, eps, weight), (pid, step, -, -) as
// bits, and the learned sampler's payload (r, gamma, eps_c, ledger index)
// in a fourth: three or four vector stores per record, which the plain
// step kernels use (the learned sampler's has 14 words per record); the 48-byte record
// stride keeps the 8 lanes of each quarter-warp on distinct banks.  u is the
// raw mean momentum, normalised at the flush.
struct PhotonStageSoA {
  float f[8][kStage];  // x y z u_x u_y u_z eps weight
  uint32_t pid[kStage];
  uint32_t step[kStage];
  float pend[4][kStage];  // learned sampler: r, gamma, eps_c, ledger index
};
struct PhotonStageAoS {
  float4 q[kStage][3];
  float4 pend[kStage];
};
// The record layout without the payload slot (table sampler), for a kernel
// whose shared memory also holds the sampling table.
struct PhotonStageRec {
  float4 q[kStage][3];
};
// The control kernels' layout with the emission's angular spread (CTRL = 2):
// the fields, plus per record the inputs of its turn, which the flush
// evaluates for up to 32 records at a time instead of in every warp-step
// where some lane emits: x, 1/gamma, |u_avg| times the orbit normal, and
// the two Philox words of psi.
struct PhotonStageSpread {
  float f[8][kStage];
  uint32_t pid[kStage];
  uint32_t step[kStage];
  float ex[7][kStage];  // x, 1/gamma, b_x, b_y, b_z, w0, w1 (words as bits)
};

template <class ST>
constexpr bool kRecordStage =
    std::is_same<ST, PhotonStageAoS>::value || std::is_same<ST, PhotonStageRec>::value;

template <bool PEND>
__device__ __forceinline__ void stage_put(PhotonStageSoA& st, int pos, const float rec[8],
                                          uint32_t pid, uint32_t step, const float* pend) {
#pragma unroll
  for (int k = 0; k < 8; ++k) st.f[k][pos] = rec[k];
  st.pid[pos] = pid;
  st.step[pos] = step;
  if constexpr (PEND) {
#pragma unroll
    for (int k = 0; k < 4; ++k) st.pend[k][pos] = pend[k];
  }
}
template <bool PEND>
__device__ __forceinline__ void stage_put(PhotonStageAoS& st, int pos, const float rec[8],
                                          uint32_t pid, uint32_t step, const float* pend) {
  st.q[pos][0] = make_float4(rec[0], rec[1], rec[2], rec[3]);
  st.q[pos][1] = make_float4(rec[4], rec[5], rec[6], rec[7]);
  st.q[pos][2] = make_float4(__uint_as_float(pid), __uint_as_float(step), 0.0f, 0.0f);
  if constexpr (PEND) st.pend[pos] = make_float4(pend[0], pend[1], pend[2], pend[3]);
}
template <bool PEND>
__device__ __forceinline__ void stage_put(PhotonStageRec& st, int pos, const float rec[8],
                                          uint32_t pid, uint32_t step, const float*) {
  static_assert(!PEND, "no payload slot");
  st.q[pos][0] = make_float4(rec[0], rec[1], rec[2], rec[3]);
  st.q[pos][1] = make_float4(rec[4], rec[5], rec[6], rec[7]);
  st.q[pos][2] = make_float4(__uint_as_float(pid), __uint_as_float(step), 0.0f, 0.0f);
}
template <bool PEND>
__device__ __forceinline__ void stage_put(PhotonStageSpread& st, int pos, const float rec[8],
                                          uint32_t pid, uint32_t step, const float* ex) {
  static_assert(!PEND, "no payload slot");
#pragma unroll
  for (int k = 0; k < 8; ++k) st.f[k][pos] = rec[k];
  st.pid[pos] = pid;
  st.step[pos] = step;
#pragma unroll
  for (int k = 0; k < 7; ++k) st.ex[k][pos] = ex[k];
}
__device__ __forceinline__ float4 stage_pend(const PhotonStageSoA& st, int r) {
  return make_float4(st.pend[0][r], st.pend[1][r], st.pend[2][r], st.pend[3][r]);
}
__device__ __forceinline__ float4 stage_pend(const PhotonStageAoS& st, int r) {
  return st.pend[r];
}
__device__ __forceinline__ float stage_weight(const PhotonStageSoA& st, int r) {
  return st.f[7][r];
}
__device__ __forceinline__ float stage_weight(const PhotonStageAoS& st, int r) {
  return st.q[r][1].w;
}

// The layout a kernel stages in: records or fields.
template <bool Aos>
using PhotonStageT = typename std::conditional<Aos, PhotonStageAoS, PhotonStageSoA>::type;

struct PhotonOut {
  float* f[8];
  uint32_t *pid, *step;
  int64_t cap;
  unsigned long long* cursor;
  // learned sampler: per-slot payload for the finishing kernel; a record
  // beyond the capacity takes its energy from the G^-1 table at once
  float4* pend;
  const float* ginv;
  double* led_base;
  unsigned long long* fallback;
  const float* ang;  // angular-spread table (CTRL = 2 kernels)
};

template <bool PEND = false, class ST>
__device__ __forceinline__ void flush_stage(ST& st, int fill, const PhotonOut& o) {
  const int lane = threadIdx.x & 31;
  unsigned long long base = 0ull;
  if (lane == 0) base = atomicAdd(o.cursor, static_cast<unsigned long long>(fill));
  base = __shfl_sync(0xffffffffu, base, 0);
  __syncwarp();
  for (int r = lane; r < fill; r += 32) {
    const unsigned long long slot = base + static_cast<unsigned>(r);
    if (slot < static_cast<unsigned long long>(o.cap)) {
      // the direction is staged as the raw mean momentum: normalise here,
      // once per record, instead of in every lane of every step
      if constexpr (std::is_same<ST, PhotonStageSpread>::value) {
        // angular spread: u_avg turned by theta = psi / gamma toward b
        float dx = st.f[3][r], dy = st.f[4][r], dz = st.f[5][r];
        const float bx = st.ex[2][r], by = st.ex[3][r], bz = st.ex[4][r];
        if (bx != 0.0f || by != 0.0f || bz != 0.0f) {
          const float th = ang_psi<float>(o.ang, st.ex[0][r], __float_as_uint(st.ex[5][r]),
                                          __float_as_uint(st.ex[6][r])) *
                           st.ex[1][r];
          float sn, cs;
          sincosf(th, &sn, &cs);
          dx = cs * dx + sn * bx;
          dy = cs * dy + sn * by;
          dz = cs * dz + sn * bz;
        }
        const float d2 = dx * dx + dy * dy + dz * dz;
        const float inv = d2 > 0.0f ? rsqrtf(d2) : 0.0f;
        o.f[0][slot] = st.f[0][r]; o.f[1][slot] = st.f[1][r]; o.f[2][slot] = st.f[2][r];
        o.f[3][slot] = dx * inv; o.f[4][slot] = dy * inv; o.f[5][slot] = dz * inv;
        o.f[6][slot] = st.f[6][r]; o.f[7][slot] = st.f[7][r];
        o.pid[slot] = st.pid[r];
        o.step[slot] = st.step[r];
      } else if constexpr (kRecordStage<ST>) {
        const float4 qa = st.q[r][0], qb = st.q[r][1], qc = st.q[r][2];
        const float d2 = qa.w * qa.w + qb.x * qb.x + qb.y * qb.y;
        const float inv = d2 > 0.0f ? rsqrtf(d2) : 0.0f;
        o.f[0][slot] = qa.x; o.f[1][slot] = qa.y; o.f[2][slot] = qa.z;
        o.f[3][slot] = qa.w * inv; o.f[4][slot] = qb.x * inv; o.f[5][slot] = qb.y * inv;
        o.f[6][slot] = qb.z; o.f[7][slot] = qb.w;
        o.pid[slot] = __float_as_uint(qc.x);
        o.step[slot] = __float_as_uint(qc.y);
      } else {
        const float dx = st.f[3][r], dy = st.f[4][r], dz = st.f[5][r];
        const float d2 = dx * dx + dy * dy + dz * dz;
        const float inv = d2 > 0.0f ? rsqrtf(d2) : 0.0f;
        o.f[0][slot] = st.f[0][r]; o.f[1][slot] = st.f[1][r]; o.f[2][slot] = st.f[2][r];
        o.f[3][slot] = dx * inv; o.f[4][slot] = dy * inv; o.f[5][slot] = dz * inv;
        o.f[6][slot] = st.f[6][r]; o.f[7][slot] = st.f[7][r];
        o.pid[slot] = st.pid[r];
        o.step[slot] = st.step[r];
      }
      if constexpr (PEND) o.pend[slot] = stage_pend(st, r);
    } else if constexpr (PEND) {
      // dropped record: its energy still enters the ledger
      const float4 pd = stage_pend(st, r);
      const float x = __expf(ginv_ln(o.ginv, pd.x));
      const int li = __float_as_int(pd.w);
      if (li >= 0)
        atomicAdd(o.led_base + li, f32_to_f64(stage_weight(st, r) * (x * pd.z)));
      atomicAdd(o.fallback, 1ull);
    }
  }
  __syncwarp();
}

// Warp-collective, with the warp's ballot of `want` already taken (mask != 0).
// rec = position, mean momentum (normalised at flush), energy, weight;
// pend (PEND) = the learned sampler's payload.
template <bool PEND = false, class ST>
__device__ __forceinline__ void stage_photon_mask(ST& st, int& fill,
                                                  const PhotonOut& o, bool want,
                                                  unsigned mask, const float rec[8],
                                                  uint32_t pid, uint32_t step,
                                                  const float* pend = nullptr) {
  const int cnt = __popc(mask);
  if (fill + cnt > kStage) {
    flush_stage<PEND>(st, fill, o);
    fill = 0;
  }
  if (want) {
    const int lane = threadIdx.x & 31;
    const int pos = fill + __popc(mask & ((1u << lane) - 1u));
    stage_put<PEND>(st, pos, rec, pid, step, pend);
  }
  fill += cnt;
}

// Warp-collective: every lane of the warp calls it with its own `want`.
template <class ST>
__device__ __forceinline__ void stage_photon(ST& st, int& fill,
                                             const PhotonOut& o, bool want,
                                             const float rec[8], uint32_t pid,
                                             uint32_t step) {
  const unsigned mask = __ballot_sync(0xffffffffu, want);
  if (mask == 0u) return;
  stage_photon_mask(st, fill, o, want, mask, rec, pid, step);
}

// ---------------------------------------------------------------------------
// Gathers for the shared-memory tile of the sorted Yee path.
// ---------------------------------------------------------------------------
template <typename R, int FIELD>
struct FieldGather {
  const StepParams<R>& P;
  __device__ __forceinline__ EB<R> operator()(R x, R y, uint64_t phase) const {
    return gather<R, FIELD>(P, x, y, phase);
  }
};

// Field values of one 32 x 32-cell tile plus a 6-cell halo, all six
// components, staged in shared memory ([component][row][column], 44 x 44).
// A particle within 2 cells of the staged edge (it drifted since the last
// sort) is gathered from global memory instead, so the result never depends
// on the tile assignment.
template <typename R>
struct TileGather {
  const StepParams<R>& P;
  const float* sm;
  int gx0, gy0;  // grid cell of staged value (0, 0)
  // Staged layout (tile coordinates, row-major kStageW x kStageW per plane):
  // (Ex, By) and (Ey, Bx) interleaved in pairs, since each pair shares its
  // staggering and so its stencil, then the Ez and Bz planes.
  static constexpr int kPlane = kStageW * kStageW;
  __host__ __device__ static constexpr int pos(int c, int r) {
    return c == 0 ? 2 * r
                  : c == 4 ? 2 * r + 1
                  : c == 1 ? 2 * kPlane + 2 * r
                  : c == 3 ? 2 * kPlane + 2 * r + 1
                  : c == 2 ? 4 * kPlane + r : 5 * kPlane + r;
  }
  // one plane (Ez: p = 4, Bz: p = 5), stencil origin (i0, j0)
  __device__ __forceinline__ R comp(int p, int i0, const R wx[3], int j0, const R wy[3]) const {
    const float* base = sm + p * kPlane + j0 * kStageW + i0;
    R v = R(0);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const float* row = base + b * kStageW;
      v += wy[b] * (wx[0] * R(row[0]) + wx[1] * R(row[1]) + wx[2] * R(row[2]));
    }
    return v;
  }
  // an interleaved pair (pair 0: Ex, By; pair 1: Ey, Bx)
  __device__ __forceinline__ void comp2(int pair, int i0, const R wx[3], int j0, const R wy[3],
                                        R& a, R& b) const {
    const float2* base =
        reinterpret_cast<const float2*>(sm) + pair * kPlane + j0 * kStageW + i0;
    a = R(0);
    b = R(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float2* row = base + k * kStageW;
      const float2 v0 = row[0], v1 = row[1], v2 = row[2];
      a += wy[k] * (wx[0] * R(v0.x) + wx[1] * R(v1.x) + wx[2] * R(v2.x));
      b += wy[k] * (wx[0] * R(v0.y) + wx[1] * R(v1.y) + wx[2] * R(v2.y));
    }
  }
  __device__ __forceinline__ EB<R> operator()(R x, R y, uint64_t) const {
    const Cell<R> cx = cell_of(x, P.x0, P.inv_dx, P.inv_dx_lo, P.nx);
    const Cell<R> cy = cell_of(y, P.y0, P.inv_dy, P.inv_dy_lo, P.ny);
    const int cl = cx.c - gx0, rl = cy.c - gy0;
    // staged stencil rows/columns cl-1 .. cl+2 must lie in [0, kStageW)
    if (!(cl >= 1 && cl <= kStageW - 3 && rl >= 1 && rl <= kStageW - 3))
      return yee2d_cells(P, cx, cy);
    // the two staggerings per axis share their weights across components
    R wx0[3], wxh[3], wy0[3], wyh[3];
    const int ix0 = cl + qs_weights(cx.f, wx0) - 1;
    const int ixh = cl + qs_weights(cx.f - R(0.5), wxh) - 1;
    const int iy0 = rl + qs_weights(cy.f, wy0) - 1;
    const int iyh = rl + qs_weights(cy.f - R(0.5), wyh) - 1;
    EB<R> f;
    comp2(0, ixh, wxh, iy0, wy0, f.Ex, f.By);
    comp2(1, ix0, wx0, iyh, wyh, f.Ey, f.Bx);
    f.Ez = comp(4, ix0, wx0, iy0, wy0);
    f.Bz = comp(5, ixh, wxh, iyh, wyh);
    return f;
  }
};

struct Counts {
  uint32_t dn1 = 0, clamp = 0, chi = 0, nan = 0, fallback = 0, wig = 0;
  bool bad_id = false;
};

// ---------------------------------------------------------------------------
// One particle, nsub steps (the whole per-step path).  Warp-collective: every
// lane of the warp calls it, inactive lanes with act = false.
// ---------------------------------------------------------------------------
// What a launch reads of one particle: its state, id and, for one-step
// launches, its LL ledger entry.  Loaded separately from the step so a thread
// can issue the loads of its next particle before computing the current one.
template <typename R>
struct PState {
  R x, y, z, ux, uy, uz, w;
  uint32_t pid;
  double ll_old, emit_old;  // ledger entries (LL = true)
  bool act;
};

// LL: 0 state and id only; 1 with the ledger entries (one-step launches);
// 2 the same for a dense launch (implicit ids pid0 + i, every particle inside
// the ledger, n >= 1; checked on the host): loads at a valid index for
// every lane, i or, for an inactive lane, 0 (its values are never stored),
// instead of zeroed registers and a branch, and ledger entry i directly.
template <typename R, int LL = 0>
__device__ __forceinline__ void load_state(const StepParams<R>& P, int64_t i, bool act,
                                           PState<R>& s) {
  s.act = act;
  if constexpr (LL == 2) {
    const int64_t k = act ? i : 0;
    s.x = P.x[k]; s.y = P.y[k];
    s.z = P.z ? P.z[k] : R(0);
    s.ux = P.ux[k]; s.uy = P.uy[k]; s.uz = P.uz[k];
    s.w = P.w[k];
    s.pid = P.pid0 + static_cast<uint32_t>(i);
    s.ll_old = P.rr_mode >= PRAD_RR_LEDGER ? P.led_ll[k] : 0.0;
    s.emit_old = P.led_emit[k];
    return;
  }
  s.x = s.y = s.z = s.ux = s.uy = s.uz = s.w = R(0);
  s.pid = 0;
  s.ll_old = s.emit_old = 0.0;
  if (act) {
    s.x = P.x[i]; s.y = P.y[i];
    if (P.z) s.z = P.z[i];
    s.ux = P.ux[i]; s.uy = P.uy[i]; s.uz = P.uz[i];
    s.w = P.w[i];
    s.pid = P.pid ? P.pid[i] : P.pid0 + static_cast<uint32_t>(i);
    if constexpr (LL) {
      const int64_t li = static_cast<int64_t>(s.pid - P.pid0);
      if (li < P.led_n) {
        if (P.rr_mode >= PRAD_RR_LEDGER) s.ll_old = P.led_ll[li];
        s.emit_old = P.led_emit[li];
      }
    }
  }
}

// One-step launches of the FP32 table sampler without control read the
// sampling table from a copy in shared memory (advance_particle's STAB):
// there the streamed state passes through L1 and would evict it.  (Fused
// launches keep it in L1: the copy's 20 KB would cost them a resident block
// per SM.)
template <typename R, int SAMP, int ONE, int CTRL>
constexpr bool kSharedTab =
    sizeof(R) == 4 && SAMP == PRAD_SAMPLER_TABLE && ONE != 0 && !CTRL;

// The new state is written back to global memory.  The launch's ledger increments reach the FP64 ledgers as one add
// per entry per launch, so the sums are sequenced by the launches and
// bit-reproducible.  Multi-step launches add them with fire-and-forget
// atomics performed in L2 (no load, no FP64 add and no wait on the SM).
// One-step launches (ONE) store st.ll_old + increment and st.emit_old +
// increment instead, both entries prefetched with the state: there an
// atomic per particle per launch would keep L2's atomic units busy, and the
// photon cursor's atomic waits behind them.
// ONE: the launch is known to advance exactly one step (P.nsub == 1); 2: a
// dense one (implicit ids, every particle inside the ledger: entry i).
// CTRL: super-photon control or diagnostics are enabled (the plain method
// compiles without their per-step work).
// rk: the Philox round keys, in the kernel's parameter space.
// STD: the standard configuration (LL kick applied, field form of H_eff,
// three dimensions, two for the Yee grid) fixed at compile time, so the step
// tests no mode.
template <typename R, int FIELD, int SAMP, int ONE = 0, int CTRL = 0,
          bool STD = false, bool STAB = false, int PWS = 0, class G, class ST>
__device__ __forceinline__ void advance_particle(const StepParams<R>& P, const uint32_t (&rk)[20],
                                                 const G& gat,
                                                 int64_t i, const PState<R>& st,
                                                 ST& stage, int& fill,
                                                 const PhotonOut& pout, Counts& cnt,
                                                 const typename TabOf<R>::T* stab = nullptr) {
  const bool act = st.act;
  R x = st.x, y = st.y, z = st.z, ux = st.ux, uy = st.uy, uz = st.uz;
  const R w = st.w;
  const uint32_t pid = st.pid;
  Acc<R> ll, le;
  const R chk = x + y + z + ux + uy + uz + w;
  const bool live = act && isfinite(chk);
  if (act && !live) ++cnt.nan;
  uint64_t phase = P.phase_t0;
  // absolute ledger entry of this particle (-1: outside the ledger)
  const int64_t li_rel = static_cast<int64_t>(pid - P.pid0);
  const int32_t li_abs = li_rel < P.led_n ? static_cast<int32_t>(P.led_off + li_rel) : -1;
  (void)li_abs;

  const int nsub = ONE ? 1 : P.nsub;
  // The learned sampler without control draws two uniforms per step (the
  // network's r and the emission decision's R), so one Philox block, counter
  // (pid, step / 2, tag 4, ensemble), serves an even step (words 0, 1) and
  // the odd step after it (words 2, 3); the table sampler and the control
  // variants draw one block per step, counter (pid, step, 0, ensemble).
  constexpr bool kPairDraws = SAMP != PRAD_SAMPLER_TABLE && !CTRL;
  uint4 pair_blk = make_uint4(0u, 0u, 0u, 0u);
  // the table sampler's per-particle Philox words (one-step launches and the
  // Yee grid; the fused analytic-field kernels, at 48 registers, are faster
  // recomputing them than keeping four more words live)
  constexpr bool kPre = SAMP == PRAD_SAMPLER_TABLE && (ONE != 0 || FIELD == PRAD_FIELD_YEE2D);
  PhiloxPre ppre{};
  if constexpr (kPre) ppre = philox_pre(pid, P.ensemble, rk);
  const int rr_mode = STD ? PRAD_RR_APPLY : P.rr_mode;
  const int heff_form = STD ? PRAD_HEFF_FIELD : P.heff_form;
  const int dims = STD ? (FIELD == PRAD_FIELD_YEE2D ? 2 : 3) : P.dims;
  for (int s = 0; s < nsub; ++s) {
    const uint32_t step = static_cast<uint32_t>(P.t0 + s);
    // 1. field at x^n, t^n
    EB<R> f;
    if constexpr (FIELD == PRAD_FIELD_PLANE_WAVE && PWS != 0)
      f = plane_wave_signed<PWS>(P, x, phase);
    else
      f = gat(x, y, phase);
    phase += P.phase_step;
    // 2. Boris: half E kick, rotation, half E kick
    const R hq = P.half_q_dtn;
    R nux, nuy, nuz;
    if constexpr (FIELD == PRAD_FIELD_PLANE_WAVE) {
      // the wave has E_x = B_x = 0: the same push with those terms dropped
      const R umx = ux, umy = uy + hq * f.Ey, umz = uz + hq * f.Ez;
      const R igm = rsq(R(1) + umx * umx + umy * umy + umz * umz);
      const R ty = hq * f.By * igm, tz = hq * f.Bz * igm;
      const R sf = R(2) * rcp(R(1) + ty * ty + tz * tz);
      const R sy = sf * ty, sz = sf * tz;
      const R vx = umx + (umy * tz - umz * ty);
      const R vy = umy - umx * tz;
      const R vz = umz + umx * ty;
      nux = umx + (vy * sz - vz * sy);
      nuy = umy - vx * sz + hq * f.Ey;
      nuz = umz + vx * sy + hq * f.Ez;
    } else {
      const R umx = ux + hq * f.Ex, umy = uy + hq * f.Ey, umz = uz + hq * f.Ez;
      const R igm = rsq(R(1) + umx * umx + umy * umy + umz * umz);
      const R tx = hq * f.Bx * igm, ty = hq * f.By * igm, tz = hq * f.Bz * igm;
      const R sf = R(2) * rcp(R(1) + tx * tx + ty * ty + tz * tz);
      const R sx = sf * tx, sy = sf * ty, sz = sf * tz;
      const R vx = umx + (umy * tz - umz * ty);
      const R vy = umy + (umz * tx - umx * tz);
      const R vz = umz + (umx * ty - umy * tx);
      nux = umx + (vy * sz - vz * sy) + hq * f.Ex;
      nuy = umy + (vz * sx - vx * sz) + hq * f.Ey;
      nuz = umz + (vx * sy - vy * sx) + hq * f.Ez;
    }
    // 3. mean momentum of the step
    const R ax = R(0.5) * (ux + nux), ay = R(0.5) * (uy + nuy), az = R(0.5) * (uz + nuz);
    const R ua2 = ax * ax + ay * ay + az * az;
    const R iga = rsq(R(1) + ua2);
    const R ga = (R(1) + ua2) * iga;
    // 4. effective field, limited by dp_perp/p <= 1 (Omega dt <= gamma)
    R Om;
    if (heff_form == PRAD_HEFF_FIELD) {
      const R bx = ax * iga, by = ay * iga, bz = az * iga;
      R fx, fy, fz, eb;
      if constexpr (FIELD == PRAD_FIELD_PLANE_WAVE) {
        fx = by * f.Bz - bz * f.By;
        fy = f.Ey - bx * f.Bz;
        fz = f.Ez + bx * f.By;
        eb = f.Ey * by + f.Ez * bz;
      } else {
        fx = f.Ex + (by * f.Bz - bz * f.By);
        fy = f.Ey + (bz * f.Bx - bx * f.Bz);
        fz = f.Ez + (bx * f.By - by * f.Bx);
        eb = f.Ex * bx + f.Ey * by + f.Ez * bz;
      }
      const R h2 = fx * fx + fy * fy + fz * fz - eb * eb;
      Om = (STD ? R(1) : P.abs_q) * sqr(h2 > R(0) ? h2 : R(0));
    } else {  // Eq. (9), gamma = mean of the end-point Lorentz factors
      const R dx_ = nux - ux, dy_ = nuy - uy, dz_ = nuz - uz;
      const R dp2 = dx_ * dx_ + dy_ * dy_ + dz_ * dz_;
      const R pdp = ax * dx_ + ay * dy_ + az * dz_;
      const R g0 = sqr_pos(R(1) + ux * ux + uy * uy + uz * uz);
      const R g1 = sqr_pos(R(1) + nux * nux + nuy * nuy + nuz * nuz);
      R c2 = ua2 * dp2 - pdp * pdp;
      c2 = c2 > R(0) ? c2 : R(0);
      Om = ua2 > R(0) ? R(0.5) * (g0 + g1) * sqr(c2) * rcp(ua2) * P.inv_dtn : R(0);
    }
    if constexpr (FIELD == PRAD_FIELD_PLANE_WAVE && CTRL) {
      if (P.diag & PRAD_DIAG_WIGGLER) {
        // synchrotron (wiggler) regime: Omega tau_EM > 1 with tau_EM the
        // field period the particle sees, 1 / (omega_L |1 - dir beta_x|)
        const R seen = P.wl * fabs(R(1) - P.dir * ax * iga);
        if (live && Om < seen) ++cnt.wig;
      }
    }
    if (Om * P.dtn > ga) {
      Om = ga * P.inv_dtn;
      if (live) ++cnt.clamp;
    }
    // 5. omega_c (Eq. (1)) as hbar omega_c / m c^2; chi = eps_r Omega gamma,
    //    tested as 1.5 chi > 1.5 on the product epsc is formed from
    const R e1 = P.eps_r15 * Om * ga;
    const R epsc = e1 * ga;
    if (live && e1 > R(1.5)) ++cnt.chi;
    // 6. Landau-Lifshitz loss (Eq. (4)): ledger and optional kick
    const R om2 = Om * Om;
    if (rr_mode >= PRAD_RR_LEDGER) ll.add(w * P.ll_coef * om2 * ua2);
    R n2 = nux * nux + nuy * nuy + nuz * nuz;
    if (rr_mode == PRAD_RR_APPLY) {
      const R gL = sqr_pos(R(1) + n2);
      const R fk = rcp(R(1) + P.ll_coef * om2 * gL);
      nux *= fk; nuy *= fk; nuz *= fk;
      n2 *= fk * fk;
    }
    // 7. position x^{n+1}
    const R ign = rsq(R(1) + n2);
    const R dtg = P.dtn * ign;
    R xn = x + dtg * nux, yn = y + dtg * nuy, zn = z;
    if (dims == 3) zn = z + dtg * nuz;
    if constexpr (FIELD == PRAD_FIELD_YEE2D) {
      xn -= P.Lx * flr((xn - P.x0) * (R(1) / P.Lx));
      yn -= P.Ly * flr((yn - P.y0) * (R(1) / P.Ly));
    }
    uint4 rnd;
    if constexpr (kPairDraws) {
      // (step & 1) is the same in every lane: no divergence
      if (s == 0 || (step & 1u) == 0u)
        pair_blk = philox10_rk(make_uint4(pid, step >> 1, 4u, P.ensemble), rk);
      // r in word 0 and R in word 2 of rnd, as in the one-block-per-step layout
      rnd = (step & 1u) ? make_uint4(pair_blk.z, 0u, pair_blk.w, 0u)
                        : make_uint4(pair_blk.x, 0u, pair_blk.y, 0u);
    } else {
      if constexpr (kPre)
        rnd = philox10_pre(ppre, step, rk);
      else
        rnd = philox10_rk<SAMP == PRAD_SAMPLER_TABLE>(make_uint4(pid, step, 0u, P.ensemble), rk);
    }
    const R Rr = unit_uniform<R>(rnd.z);
    if constexpr (SAMP == PRAD_SAMPLER_TABLE) {
      // 8. Monte Carlo emission: proposal x = P^-1(R'), dN of Eq. (13);
      //    one trial with the Philox words (w0, w1) and uniform Rd, dN
      //    scaled by dn_scale, record weights by wmul, for lanes with part
      auto trial = [&](uint32_t w0, uint32_t w1, R Rd, R dn_scale, R wmul, bool part,
                       uint32_t j) {
        R xs, g;
        sample_x_g<STAB>(P, w0, w1, xs, g, stab);
        const R dN = P.cn_dt * Om * g * rcp(xs) * dn_scale;
        const R fl = flr(dN);
        const R k = fl + ((Rd < dN - fl) ? R(1) : R(0));
        if (part && dN > R(1)) ++cnt.dn1;
        const bool want = part && k > R(0) && w > R(0);
        // 9. append + emitted-energy ledger; the record is built only when
        //    some lane of the warp emits
        const unsigned mask = __ballot_sync(0xffffffffu, want);
        if (mask) {
          const R eps = xs * epsc;
          const R kw = k * w * wmul;
          if (want) le.add(kw * eps);
          const float rec[8] = {static_cast<float>(xn), static_cast<float>(yn),
                                static_cast<float>(zn), static_cast<float>(ax),
                                static_cast<float>(ay), static_cast<float>(az),
                                static_cast<float>(eps), static_cast<float>(kw)};
          if constexpr (CTRL == 2) {
            // angular spread (Eqs. (5)-(6)): the record carries what its
            // turn needs (psi's Philox words, block (pid, step, 0x20000 +
            // trial, ensemble); x; 1/gamma; b = |u_avg| times the orbit
            // normal u^n x u^(n+1) / |u^n x u^(n+1)|, zero if there is none)
            // and the flush turns u_avg by theta = psi / gamma toward b
            const uint4 ra = philox10_rk(make_uint4(pid, step, 0x20000u + j, P.ensemble), rk);
            const R cx = uy * nuz - uz * nuy, cy = uz * nux - ux * nuz, cz = ux * nuy - uy * nux;
            const R c2 = cx * cx + cy * cy + cz * cz;
            const R fb = c2 > R(0) ? sqrt(ua2 / c2) : R(0);
            const float ex[7] = {static_cast<float>(xs), static_cast<float>(iga),
                                 static_cast<float>(fb * cx), static_cast<float>(fb * cy),
                                 static_cast<float>(fb * cz), __uint_as_float(ra.x),
                                 __uint_as_float(ra.y)};
            stage_photon_mask(stage, fill, pout, want, mask, rec, pid, step, ex);
          } else {
            stage_photon_mask(stage, fill, pout, want, mask, rec, pid, step);
          }
        }
      };
      if constexpr (!CTRL) {
        trial(rnd.x, rnd.y, Rr, R(1), R(1), live, 0u);
      } else {
        // super-photon control: a particle takes part with probability
        // sel_q (Philox word 3 of trial 0), with weight 1 / sel_q; ntry
        // trials of 1 / ntry of dN each, trial j >= 1 from its own block
        const bool part = live && unit_uniform<R>(rnd.w) < P.sel_q;
        trial(rnd.x, rnd.y, Rr, P.inv_ntry, P.inv_sel_q, part, 0u);
        for (int j = 1; j < P.ntry; ++j) {
          const uint4 cj = make_uint4(pid, step, 0x10000u + static_cast<uint32_t>(j), P.ensemble);
          const uint4 rb = philox10_rk(cj, rk);
          trial(rb.x, rb.y, unit_uniform<R>(rb.z), P.inv_ntry, P.inv_sel_q, part,
                static_cast<uint32_t>(j));
        }
      }
    } else {
      // 8'. direct scheme: photons of this step ~ mean (5 sqrt3/6) alpha
      //     Omega dt (the integral of Eq. (13)'s spectrum), multiplicity as in
      //     the table path; the frequency x = G^-1(r') from the MLP
      const R pm = P.cp_dt * Om;
      const R fl = flr(pm);
      const R k = fl + ((Rr < pm - fl) ? R(1) : R(0));
      if (live && pm > R(1)) ++cnt.dn1;
      // super-photon control: selection with probability sel_q
      bool part = live;
      if constexpr (CTRL) part = live && unit_uniform<R>(rnd.w) < P.sel_q;
      const bool want = part && k > R(0) && w > R(0);
      const unsigned wmask = __ballot_sync(0xffffffffu, want);
      if (wmask) {
        // the record and the network's inputs; the energy is filled in by
        // the finishing kernel (batched tensor-core evaluation)
        const float rec[8] = {static_cast<float>(xn), static_cast<float>(yn),
                              static_cast<float>(zn), static_cast<float>(ax),
                              static_cast<float>(ay), static_cast<float>(az),
                              0.0f, static_cast<float>(CTRL ? k * w * P.inv_sel_q : k * w)};
        const float pend[4] = {fmaf(static_cast<float>(rnd.x), 0x1p-32f, 0x1p-33f),
                               static_cast<float>(ga), static_cast<float>(epsc),
                               __int_as_float(li_abs)};
        stage_photon_mask<true>(stage, fill, pout, want, wmask, rec, pid, step, pend);
      }
    }
    // a particle that is not live (inactive lane or non-finite state) is
    // never stored, emits nothing and counts nothing, so its registers may
    // advance like the others' (no select per step)
    x = xn; y = yn; z = zn;
    ux = nux; uy = nuy; uz = nuz;
  }
  if (live) {
    P.x[i] = x; P.y[i] = y;
    if (P.z) P.z[i] = z;
    P.ux[i] = ux; P.uy[i] = uy; P.uz[i] = uz;
    if constexpr (ONE == 2) {
      if (rr_mode >= PRAD_RR_LEDGER) P.led_ll[i] = st.ll_old + ll.value_one();
      // (with control a step may add several trials: the full value)
      if (le.nonzero()) P.led_emit[i] = st.emit_old + (CTRL ? le.value() : le.value_one());
      return;
    }
    const int64_t li = static_cast<int64_t>(pid - P.pid0);
    if (li < P.led_n) {
      if (rr_mode >= PRAD_RR_LEDGER) {
        if constexpr (ONE)
          P.led_ll[li] = st.ll_old + ll.value_one();
        else
          atomicAdd(P.led_ll + li, ll.value());
      }
      if (le.nonzero()) {
        // (with control a step may add several trials: the full value)
        if constexpr (ONE)
          P.led_emit[li] = st.emit_old + (CTRL ? le.value() : le.value_one());
        else
          atomicAdd(P.led_emit + li, le.value());
      }
    } else {
      cnt.bad_id = true;
    }
  }
}

template <typename R>
__device__ __forceinline__ PhotonOut make_pout(const StepParams<R>& P) {
  PhotonOut o;
  o.f[0] = P.px; o.f[1] = P.py; o.f[2] = P.pz;
  o.f[3] = P.pnx; o.f[4] = P.pny; o.f[5] = P.pnz;
  o.f[6] = P.peps; o.f[7] = P.pw;
  o.pid = P.ppid; o.step = P.pstep;
  o.cap = P.cap; o.cursor = P.counters + kCursor;
  o.pend = P.ppend;
  o.ginv = P.ginv;
  o.led_base = P.led_base;
  o.fallback = P.counters + kMlpFallback;
  o.ang = P.ang;
  return o;
}

// Block reduction of the counters: one atomic per nonzero block total.
__device__ __forceinline__ void flush_counts(const Counts& c, unsigned long long* counters) {
  constexpr int kN = 7;
  __shared__ uint32_t red[kN][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t v[kN] = {__reduce_add_sync(0xffffffffu, c.dn1),
                          __reduce_add_sync(0xffffffffu, c.clamp),
                          __reduce_add_sync(0xffffffffu, c.chi),
                          __reduce_add_sync(0xffffffffu, c.nan),
                          __reduce_add_sync(0xffffffffu, c.fallback),
                          __reduce_add_sync(0xffffffffu, c.bad_id ? 1u : 0u),
                          __reduce_add_sync(0xffffffffu, c.wig)};
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < kN; ++k) red[k][warp] = v[k];
  }
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    // counter slot of each value (bad ids set status bit 1)
    constexpr int kSlot[kN] = {kDnGt1, kClamp, kChiGt1, kNan, kMlpFallback, kStatus, kWiggler};
#pragma unroll
    for (int k = 0; k < kN; ++k) {
      const uint32_t vv = lane < nw ? red[k][lane] : 0u;
      const uint32_t t = __reduce_add_sync(0xffffffffu, vv);
      if (lane == 0 && t) {
        if (kSlot[k] == kStatus)
          atomicOr(counters + kStatus, 2ull);  // status bit 1: id outside ledger
        else
          atomicAdd(counters + kSlot[k], static_cast<unsigned long long>(t));
      }
    }
  }
}

// ---------------------------------------------------------------------------
// The fused kernel: grid-stride over particles.
// ---------------------------------------------------------------------------
// Resident blocks per SM the FP32 kernels are compiled for (registers are
// capped at 65536 / (256 * MINB)); the FP64 kernels keep the default.
#ifndef PRAD_F32_MINB
#define PRAD_F32_MINB 5
#endif
// The Yee gather (54 loads in flight) needs more registers than the
// analytic-field paths.
template <typename R, int FIELD, int SAMP>
struct MinBlocks {
  static constexpr int value =
      sizeof(R) == 8 ? 1 : (FIELD == PRAD_FIELD_YEE2D ? 4 : PRAD_F32_MINB);
};

#ifndef __CUDACC_RTC__
// Resident blocks per SM of a kernel at this block size and dynamic shared
// memory (1 if the query fails).
template <typename K>
int occupancy_of(K kernel, int block, size_t dyn) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, block, dyn) != cudaSuccess)
    return 1;
  return nb > 0 ? nb : 1;
}
#endif  // __CUDACC_RTC__

#ifndef PRAD_PF_MINB
#define PRAD_PF_MINB 4
#endif

#ifdef PRAD_SPEC
// Run-time specialisation (a kernel compiled by NVRTC for one context): the
// per-run constants of the standard step -- the normalised time
// step and charge factors, the radiation coefficients of Eqs. (1), (4), (7)
// and (13), the wave's amplitude, wavenumber and phase increment, the ensemble and
// the Philox round keys, and on the Yee grid its geometry -- given as literals, so that they fold into the
// arithmetic instead of being read from the kernel's parameter space.  The
// values are those the host would pass, so the results are the same bits.
template <typename R>
__device__ __forceinline__ StepParams<R> spec_params(const StepParams<R>& in) {
  static_assert(sizeof(R) == 4, "run-time specialisation: FP32 kernels only");
  StepParams<R> p = in;
  p.half_q_dtn = PRAD_SPEC_HALF_Q_DTN;
  p.dtn = PRAD_SPEC_DTN;
  p.inv_dtn = PRAD_SPEC_INV_DTN;
  p.cn_dt = PRAD_SPEC_CN_DT;
  p.eps_r15 = PRAD_SPEC_EPS_R15;
  p.ll_coef = PRAD_SPEC_LL_COEF;
  p.E0 = PRAD_SPEC_E0;
  p.kc = PRAD_SPEC_KC;
  p.kc_lo = PRAD_SPEC_KC_LO;
  p.cp_dt = PRAD_SPEC_CP_DT;
  p.phase_step = PRAD_SPEC_PHASE_STEP;
  p.ensemble = PRAD_SPEC_ENSEMBLE;
  constexpr uint32_t rk[20] = PRAD_SPEC_RKEY;
#pragma unroll
  for (int k = 0; k < 20; ++k) p.rkey[k] = rk[k];
#ifdef PRAD_SPEC_YEE
  // the Yee grid's size, spacing (with the low parts of 1/dx, 1/dy), origin,
  // periods and tiles per row
  p.nx = PRAD_SPEC_NX;
  p.ny = PRAD_SPEC_NY;
  p.inv_dx = PRAD_SPEC_INV_DX;
  p.inv_dy = PRAD_SPEC_INV_DY;
  p.inv_dx_lo = PRAD_SPEC_INV_DX_LO;
  p.inv_dy_lo = PRAD_SPEC_INV_DY_LO;
  p.x0 = PRAD_SPEC_X0;
  p.y0 = PRAD_SPEC_Y0;
  p.Lx = PRAD_SPEC_LX;
  p.Ly = PRAD_SPEC_LY;
  p.ntx = PRAD_SPEC_NTX;
#endif
  return p;
}
#endif
// PF: 0 no prefetch (multi-step launches); 1 one step per launch, the next
// particle prefetched; 2 the same for a dense launch (see dense_launch).
// PWS: the plane wave's signs at compile time (0: from the parameters).
template <typename R, int FIELD, int SAMP, int PF, int CTRL, bool STD = false, int PWS = 0>
__global__ void __launch_bounds__(256, (PF ? PRAD_PF_MINB : MinBlocks<R, FIELD, SAMP>::value))
    k_push_emit(const StepParams<R> P_arg) {
#ifdef PRAD_SPEC
  const StepParams<R> P = spec_params(P_arg);
#else
  const StepParams<R>& P = P_arg;
#endif
  constexpr bool kSTab = kSharedTab<R, SAMP, PF, CTRL>;
  using Stage = typename std::conditional<
      CTRL == 2, PhotonStageSpread,
      typename std::conditional<kSTab, PhotonStageRec,
                                PhotonStageT<SAMP != PRAD_SAMPLER_TABLE || !CTRL>>::type>::type;
  __shared__ Stage stage_all[kMaxWarps];
  __shared__ typename TabOf<R>::T stab[kSTab ? kNTab : 1];
  if constexpr (kSTab) {
    for (int k = threadIdx.x; k < kNTab; k += blockDim.x) stab[k] = __ldg(P.tab + k);
    __syncthreads();
  }
  Stage& stage = stage_all[threadIdx.x >> 5];
  int fill = 0;  // warp-uniform
  const PhotonOut pout = make_pout(P);
  Counts cnt;
  const FieldGather<R, FIELD> gat{P};
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t first = static_cast<int64_t>(blockIdx.x) * blockDim.x;
  if constexpr (PF) {
    // one step per launch (the state streams through HBM): a software
    // pipeline issues the loads of the thread's next particle before the
    // current one is advanced, so DRAM latency overlaps compute
    PState<R> nxt;
    load_state<R, PF>(P, first + threadIdx.x, first + threadIdx.x < P.n, nxt);
    for (int64_t base = first; base < P.n; base += stride) {
      const int64_t i = base + threadIdx.x;
      const PState<R> cur = nxt;
      const int64_t j = i + stride;
      load_state<R, PF>(P, j, j < P.n, nxt);
      advance_particle<R, FIELD, SAMP, PF, CTRL, STD, kSTab, PWS>(
          P, P.rkey, gat, i, cur, stage, fill, pout, cnt, kSTab ? stab : nullptr);
    }
  } else {
    for (int64_t base = first; base < P.n; base += stride) {
      const int64_t i = base + threadIdx.x;
      PState<R> cur;
      load_state(P, i, i < P.n, cur);
      advance_particle<R, FIELD, SAMP, 0, CTRL, STD, kSTab, PWS>(
          P, P.rkey, gat, i, cur, stage, fill, pout, cnt, kSTab ? stab : nullptr);
    }
  }
  if (fill > 0) flush_stage<SAMP != PRAD_SAMPLER_TABLE>(stage, fill, pout);
  flush_counts(cnt, P.counters);
}

// ---------------------------------------------------------------------------
// Persistent batched kernel: the grid draws work items (a chunk of one
// ensemble's particles) from an atomic counter until none are left.  The
// item's ensemble parameters are copied to shared memory when the ensemble
// changes; the per-particle path is the same as in k_push_emit.
// ---------------------------------------------------------------------------
#ifndef PRAD_BATCH_MINB
#define PRAD_BATCH_MINB 3
#endif
template <int SAMP, bool CTRL, bool STD = false>
__global__ void __launch_bounds__(256, PRAD_BATCH_MINB)
    k_push_emit_batch(const BatchParams bp) {
  const long long t_begin = clock64();
  __shared__ PhotonStageSoA stage_all[kMaxWarps];
  __shared__ StepParams<float> Ps;
  __shared__ long long s_item;
  __shared__ int s_ens;
  PhotonStageSoA& stage = stage_all[threadIdx.x >> 5];
  int fill = 0;
  Counts cnt;
  int cur = -1;
  PhotonOut pout;
  for (;;) {
    if (threadIdx.x == 0) {
      const unsigned long long it = atomicAdd(bp.next_item, 1ull);
      s_item = static_cast<long long>(it);
      int e = -1;
      if (static_cast<int64_t>(it) < bp.total_items) {  // last e with off[e] <= it
        int lo = 0, hi = bp.n_ens;
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (bp.item_off[mid] <= static_cast<int64_t>(it)) lo = mid; else hi = mid;
        }
        e = lo;
      }
      s_ens = e;
    }
    __syncthreads();
    const long long item = s_item;
    const int e = s_ens;
    if (e < 0) break;
    if (e != cur) {
      // photons staged so far belong to the previous ensemble's buffer view;
      // all ensembles share the context's buffer, so no flush is needed
      constexpr int kWords = static_cast<int>(sizeof(StepParams<float>) / 4);
      const uint32_t* src = reinterpret_cast<const uint32_t*>(bp.ens + e);
      uint32_t* dst = reinterpret_cast<uint32_t*>(&Ps);
      __syncthreads();
      for (int w = threadIdx.x; w < kWords; w += blockDim.x) dst[w] = src[w];
      __syncthreads();
      if (threadIdx.x == 0) {
        Ps.t0 += bp.step_base;
        Ps.phase_t0 += static_cast<uint64_t>(bp.step_base) * Ps.phase_step;
        Ps.nsub = bp.nsub;
      }
      __syncthreads();
      cur = e;
      pout = make_pout(Ps);
    }
    const int64_t first = (item - bp.item_off[e]) * static_cast<int64_t>(bp.chunk);
    const int64_t last = first + bp.chunk < Ps.n ? first + bp.chunk : Ps.n;
    if (Ps.field_kind == PRAD_FIELD_CONST) {
      const FieldGather<float, PRAD_FIELD_CONST> gat{Ps};
      for (int64_t base = first; base < last; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        PState<float> st;
        load_state(Ps, i, i < last, st);
        advance_particle<float, PRAD_FIELD_CONST, SAMP, 0, CTRL, STD>(Ps, bp.rkey, gat, i, st,
                                                                          stage, fill, pout, cnt);
      }
    } else {
      const FieldGather<float, PRAD_FIELD_PLANE_WAVE> gat{Ps};
      // the standard variant takes the ensemble's wave signs at compile time,
      // as a single-ensemble launch does (the same code, the same results)
      auto items = [&](auto pws) {
        for (int64_t base = first; base < last; base += blockDim.x) {
          const int64_t i = base + threadIdx.x;
          PState<float> st;
          load_state(Ps, i, i < last, st);
          advance_particle<float, PRAD_FIELD_PLANE_WAVE, SAMP, 0, CTRL, STD, false,
                           decltype(pws)::value>(Ps, bp.rkey, gat, i, st, stage, fill, pout,
                                                 cnt);
        }
      };
      if constexpr (STD) {
        switch (pw_signs(Ps)) {
          case 1: items(std::integral_constant<int, 1>{}); break;
          case 2: items(std::integral_constant<int, 2>{}); break;
          case 3: items(std::integral_constant<int, 3>{}); break;
          default: items(std::integral_constant<int, 4>{}); break;
        }
      } else {
        items(std::integral_constant<int, 0>{});
      }
    }
    __syncthreads();
  }
  if (cur >= 0 && fill > 0) flush_stage<SAMP != PRAD_SAMPLER_TABLE>(stage, fill, pout);
  // counters: any ensemble's pointer to the shared counter array will do
  flush_counts(cnt, bp.ens[0].counters);
  if (threadIdx.x == 0 && bp.busy)  // after the block's last barrier: its busy time
    atomicAdd(bp.busy + blockIdx.x, static_cast<unsigned long long>(clock64() - t_begin));
}

#ifndef __CUDACC_RTC__
// std_cfg: every ensemble runs the standard configuration (STD variant, the
// same per-step code as the standard k_push_emit variants)
template <int SAMP>
cudaError_t launch_batch_samp(const BatchParams& bp, bool ctrl, bool std_cfg, int grid,
                              int block, cudaStream_t s) {
  if (ctrl)
    k_push_emit_batch<SAMP, true><<<grid, block, 0, s>>>(bp);
  else if (std_cfg)
    k_push_emit_batch<SAMP, false, true><<<grid, block, 0, s>>>(bp);
  else
    k_push_emit_batch<SAMP, false><<<grid, block, 0, s>>>(bp);
  return cudaGetLastError();
}

cudaError_t launch_push_emit_batch(const BatchParams& bp, int sampler, bool ctrl, bool std_cfg,
                                   int grid, int block, cudaStream_t s) {
  switch (sampler) {
    case PRAD_SAMPLER_TABLE:
      return launch_batch_samp<PRAD_SAMPLER_TABLE>(bp, ctrl, std_cfg, grid, block, s);
    case PRAD_SAMPLER_MLP:
      return launch_batch_samp<PRAD_SAMPLER_MLP>(bp, ctrl, std_cfg, grid, block, s);
    case PRAD_SAMPLER_MLP_FALLBACK:
      return launch_batch_samp<PRAD_SAMPLER_MLP_FALLBACK>(bp, ctrl, std_cfg, grid, block, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int SAMP>
int batch_occupancy_samp(int block, bool ctrl, bool std_cfg) {
  if (ctrl) return occupancy_of(k_push_emit_batch<SAMP, true>, block, 0);
  if (std_cfg) return occupancy_of(k_push_emit_batch<SAMP, false, true>, block, 0);
  return occupancy_of(k_push_emit_batch<SAMP, false>, block, 0);
}

int batch_max_blocks_per_sm(int block, int sampler, bool ctrl, bool std_cfg) {
  switch (sampler) {
    case PRAD_SAMPLER_MLP: return batch_occupancy_samp<PRAD_SAMPLER_MLP>(block, ctrl, std_cfg);
    case PRAD_SAMPLER_MLP_FALLBACK:
      return batch_occupancy_samp<PRAD_SAMPLER_MLP_FALLBACK>(block, ctrl, std_cfg);
    default: return batch_occupancy_samp<PRAD_SAMPLER_TABLE>(block, ctrl, std_cfg);
  }
}

#endif  // __CUDACC_RTC__
// ---------------------------------------------------------------------------
// Tile-sorted Yee kernel: one block per work item (a chunk of <= kChunk
// particles of one tile).  The block stages the tile's six field components
// (+ halo, periodic) in shared memory with coalesced row loads, then runs the
// same per-particle path with the shared-memory gather.
// ---------------------------------------------------------------------------
template <typename R, int CTRL, bool STD = false>
__global__ void __launch_bounds__(256, 3) k_push_emit_tiled(const StepParams<R> P_arg) {
#ifdef PRAD_SPEC
  const StepParams<R> P = spec_params(P_arg);
#else
  const StepParams<R>& P = P_arg;
#endif
  if (blockIdx.x >= *P.work_count) return;
  extern __shared__ __align__(16) float tile_sm[];
  using Stage = typename std::conditional<CTRL == 2, PhotonStageSpread, PhotonStageSoA>::type;
  __shared__ Stage stage_all[kMaxWarps];
  const int4 wk = P.work[blockIdx.x];
  const int tx = wk.x % P.ntx, ty = wk.x / P.ntx;
  const int gx0 = tx * kTile - kHalo, gy0 = ty * kTile - kHalo;
  constexpr int kPlane = kStageW * kStageW;
  // periodic indices: gx0 + lx lies in [-kHalo, nx + kTile + kHalo), one
  // wrap suffices when the grid is at least as wide as the staged region;
  // smaller grids take a full modulo
  const bool wide = P.nx >= kStageW && P.ny >= kStageW;
  for (int e = threadIdx.x; e < 6 * kPlane; e += blockDim.x) {
    const int c = e / kPlane;
    const int r = e - c * kPlane;
    const int ly = r / kStageW;
    const int lx = r - ly * kStageW;
    int gx = gx0 + lx, gy = gy0 + ly;
    if (wide) {
      gx += gx < 0 ? P.nx : (gx >= P.nx ? -P.nx : 0);
      gy += gy < 0 ? P.ny : (gy >= P.ny ? -P.ny : 0);
    } else {
      gx %= P.nx;
      gy %= P.ny;
      gx += gx < 0 ? P.nx : 0;
      gy += gy < 0 ? P.ny : 0;
    }
    // (the plane pointer indexed by a run-time c from the kernel's parameter
    // space: a specialised kernel's copy of the parameters stays in registers)
    tile_sm[TileGather<R>::pos(c, r)] =
        __ldg(P_arg.yee[c] + static_cast<size_t>(gy) * P.nx + gx);
  }
  __syncthreads();
  Stage& stage = stage_all[threadIdx.x >> 5];
  int fill = 0;
  const PhotonOut pout = make_pout(P);
  Counts cnt;
  const TileGather<R> gat{P, tile_sm, gx0, gy0};
  for (int64_t base = wk.y; base < wk.z; base += blockDim.x) {
    const int64_t i = base + threadIdx.x;
    PState<R> st;
    load_state(P, i, i < wk.z, st);
    advance_particle<R, PRAD_FIELD_YEE2D, PRAD_SAMPLER_TABLE, 0, CTRL, STD>(
        P, P.rkey, gat, i, st, stage, fill, pout, cnt);
  }
  if (fill > 0) flush_stage(stage, fill, pout);
  flush_counts(cnt, P.counters);
}

#ifndef __CUDACC_RTC__
// The standard-configuration variant (STD) exists for FP32 without control
// or diagnostics.
template <typename R, int FIELD, int CTRL>
constexpr bool kHasStd = sizeof(R) == 4 && !CTRL;

// LL kick applied, field-form H_eff, the field's usual dimensions and unit
// charge (electrons, positrons)
template <typename R>
bool std_config(const StepParams<R>& p, int dims) {
  return p.rr_mode == PRAD_RR_APPLY && p.heff_form == PRAD_HEFF_FIELD && p.dims == dims &&
         p.abs_q == R(1);
}

template <typename R, int CTRL, bool STD>
cudaError_t launch_tiled_v(const StepParams<R>& p, int max_work, int block, cudaStream_t s) {
  // dynamic tile (46.5 KB) + static photon staging exceed the 48 KB default
  cudaError_t e = cudaFuncSetAttribute(k_push_emit_tiled<R, CTRL, STD>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kTileSmemBytes);
  if (e != cudaSuccess) return e;
  k_push_emit_tiled<R, CTRL, STD><<<max_work, block, kTileSmemBytes, s>>>(p);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_push_emit_tiled(const StepParams<R>& p, int max_work, int block,
                                   cudaStream_t s) {
  if (p.ang != nullptr) return launch_tiled_v<R, 2, false>(p, max_work, block, s);
  const bool ctrl = p.ntry > 1 || p.sel_q < R(1) || p.diag != 0;
  if (ctrl) return launch_tiled_v<R, 1, false>(p, max_work, block, s);
  if constexpr (kHasStd<R, PRAD_FIELD_YEE2D, 0>)
    if (std_config(p, 2)) return launch_tiled_v<R, 0, true>(p, max_work, block, s);
  return launch_tiled_v<R, 0, false>(p, max_work, block, s);
}


template <typename R, int FIELD, int SAMP, int PF, int CTRL>
void launch_k(const StepParams<R>& p, int grid, int block, cudaStream_t s) {
  if constexpr (kHasStd<R, FIELD, CTRL>) {
    if (std_config(p, FIELD == PRAD_FIELD_YEE2D ? 2 : 3)) {
      if constexpr (FIELD == PRAD_FIELD_PLANE_WAVE) {
        switch (pw_signs(p)) {
          case 1: k_push_emit<R, FIELD, SAMP, PF, CTRL, true, 1><<<grid, block, 0, s>>>(p); return;
          case 2: k_push_emit<R, FIELD, SAMP, PF, CTRL, true, 2><<<grid, block, 0, s>>>(p); return;
          case 3: k_push_emit<R, FIELD, SAMP, PF, CTRL, true, 3><<<grid, block, 0, s>>>(p); return;
          default: k_push_emit<R, FIELD, SAMP, PF, CTRL, true, 4><<<grid, block, 0, s>>>(p); return;
        }
      } else {
        k_push_emit<R, FIELD, SAMP, PF, CTRL, true><<<grid, block, 0, s>>>(p);
        return;
      }
    }
  }
  k_push_emit<R, FIELD, SAMP, PF, CTRL, false><<<grid, block, 0, s>>>(p);
}

template <typename R, int FIELD, int SAMP, int PF, int CTRL>
int occupancy_k(int block, bool std_cfg, int pws) {
  if constexpr (kHasStd<R, FIELD, CTRL>) {
    if (std_cfg) {
      if constexpr (FIELD == PRAD_FIELD_PLANE_WAVE) {
        switch (pws) {
          case 1: return occupancy_of(k_push_emit<R, FIELD, SAMP, PF, CTRL, true, 1>, block, 0);
          case 2: return occupancy_of(k_push_emit<R, FIELD, SAMP, PF, CTRL, true, 2>, block, 0);
          case 3: return occupancy_of(k_push_emit<R, FIELD, SAMP, PF, CTRL, true, 3>, block, 0);
          default: return occupancy_of(k_push_emit<R, FIELD, SAMP, PF, CTRL, true, 4>, block, 0);
        }
      } else {
        return occupancy_of(k_push_emit<R, FIELD, SAMP, PF, CTRL, true>, block, 0);
      }
    }
  }
  return occupancy_of(k_push_emit<R, FIELD, SAMP, PF, CTRL, false>, block, 0);
}

// A one-step launch is dense when ids are implicit (pid0 + i) and every
// particle has a ledger entry: its kernel indexes the ledgers by i and loads
// without per-particle range checks.
template <typename R>
bool dense_launch(const StepParams<R>& p) {
  return p.pid == nullptr && p.n >= 1 && p.led_n >= p.n && p.led_emit != nullptr &&
         (p.rr_mode < PRAD_RR_LEDGER || p.led_ll != nullptr);
}

template <typename R, int FIELD, int CTRL>
cudaError_t launch_field_c(const StepParams<R>& p, int sampler, int grid, int block,
                           cudaStream_t s) {
  if constexpr (CTRL == 2) {  // angular spread: table sampler, no prefetch variant
    if (sampler != PRAD_SAMPLER_TABLE) return cudaErrorInvalidValue;
    launch_k<R, FIELD, PRAD_SAMPLER_TABLE, 0, 2>(p, grid, block, s);
    return cudaGetLastError();
  } else {
    if (sampler == PRAD_SAMPLER_TABLE) {
      // prefetching pays when the state streams through HBM (one step per
      // launch); for long fused launches it only costs registers
      bool pf = false;
      if constexpr (sizeof(R) == 4) pf = p.nsub == 1;
      if constexpr (sizeof(R) == 4) {
        if (pf) {
          if (dense_launch(p))
            launch_k<R, FIELD, PRAD_SAMPLER_TABLE, 2, CTRL>(p, grid, block, s);
          else
            launch_k<R, FIELD, PRAD_SAMPLER_TABLE, 1, CTRL>(p, grid, block, s);
        }
      }
      if (!pf) launch_k<R, FIELD, PRAD_SAMPLER_TABLE, 0, CTRL>(p, grid, block, s);
      return cudaGetLastError();
    }
    if constexpr (sizeof(R) == 4) {
      if (sampler == PRAD_SAMPLER_MLP)
        launch_k<R, FIELD, PRAD_SAMPLER_MLP, 0, CTRL>(p, grid, block, s);
      else
        launch_k<R, FIELD, PRAD_SAMPLER_MLP_FALLBACK, 0, CTRL>(p, grid, block, s);
      return cudaGetLastError();
    }
    return cudaErrorInvalidValue;
  }
}

template <typename R, int FIELD>
cudaError_t launch_field(const StepParams<R>& p, int sampler, int grid, int block,
                         cudaStream_t s) {
  if (p.ang != nullptr) return launch_field_c<R, FIELD, 2>(p, sampler, grid, block, s);
  const bool ctrl = p.ntry > 1 || p.sel_q < R(1) || p.diag != 0;
  return ctrl ? launch_field_c<R, FIELD, 1>(p, sampler, grid, block, s)
              : launch_field_c<R, FIELD, 0>(p, sampler, grid, block, s);
}

template <typename R, int FIELD, int CTRL>
int field_occupancy_c(int sampler, int pf, int block, bool std_cfg, int pws) {
  if constexpr (CTRL == 2) {
    return occupancy_k<R, FIELD, PRAD_SAMPLER_TABLE, 0, 2>(block, false, 0);
  } else {
    if (sampler == PRAD_SAMPLER_TABLE) {
      if constexpr (sizeof(R) == 4) {
        if (pf == 2) return occupancy_k<R, FIELD, PRAD_SAMPLER_TABLE, 2, CTRL>(block, std_cfg, pws);
        if (pf == 1) return occupancy_k<R, FIELD, PRAD_SAMPLER_TABLE, 1, CTRL>(block, std_cfg, pws);
      }
      return occupancy_k<R, FIELD, PRAD_SAMPLER_TABLE, 0, CTRL>(block, std_cfg, pws);
    }
    if constexpr (sizeof(R) == 4) {
      if (sampler == PRAD_SAMPLER_MLP)
        return occupancy_k<R, FIELD, PRAD_SAMPLER_MLP, 0, CTRL>(block, std_cfg, pws);
      return occupancy_k<R, FIELD, PRAD_SAMPLER_MLP_FALLBACK, 0, CTRL>(block, std_cfg, pws);
    }
    return 1;
  }
}

template <typename R, int FIELD>
int field_occupancy(int sampler, int pf, int block, int ctrl, bool std_cfg, int pws) {
  if (ctrl == 2) return field_occupancy_c<R, FIELD, 2>(sampler, pf, block, std_cfg, pws);
  return ctrl ? field_occupancy_c<R, FIELD, 1>(sampler, pf, block, std_cfg, pws)
              : field_occupancy_c<R, FIELD, 0>(sampler, pf, block, std_cfg, pws);
}

// Resident blocks per SM of the kernel variant a launch would use.
template <typename R>
int push_emit_occupancy(const StepParams<R>& p, int field_kind, int sampler, int nsub, int block,
                        bool ctrl) {
  const int pf = nsub == 1 ? (dense_launch(p) ? 2 : 1) : 0;
  const bool sc = std_config(p, field_kind == PRAD_FIELD_YEE2D ? 2 : 3);
  // the control variant, or its angular-spread form
  const int cv = ctrl ? (p.ang != nullptr ? 2 : 1) : 0;
  switch (field_kind) {
    case PRAD_FIELD_CONST:
      return field_occupancy<R, PRAD_FIELD_CONST>(sampler, pf, block, cv, sc, pw_signs(p));
    case PRAD_FIELD_PLANE_WAVE:
      return field_occupancy<R, PRAD_FIELD_PLANE_WAVE>(sampler, pf, block, cv, sc, pw_signs(p));
    default: return field_occupancy<R, PRAD_FIELD_YEE2D>(sampler, pf, block, cv, sc, pw_signs(p));
  }
}
template int push_emit_occupancy<float>(const StepParams<float>&, int, int, int, int, bool);

bool push_emit_spec_variant(const StepParams<float>& p, int field_kind, int sampler, bool tiled,
                            SpecVariant* v) {
  const bool ctrl = p.ntry > 1 || p.sel_q < 1.0f || p.diag != 0;
  if (ctrl) return false;
  v->field = field_kind;
  v->samp = sampler;
  v->tiled = tiled ? 1 : 0;
  v->pf = 0;
  v->pws = 0;
  if (tiled) return field_kind == PRAD_FIELD_YEE2D && sampler == PRAD_SAMPLER_TABLE &&
                    std_config(p, 2);
  if (field_kind == PRAD_FIELD_PLANE_WAVE) {
    if (!std_config(p, 3)) return false;
    v->pws = pw_signs(p);
  } else if (field_kind == PRAD_FIELD_YEE2D) {
    if (!std_config(p, 2)) return false;
  } else {
    return false;
  }
  // (the learned samplers have no prefetching variant)
  v->pf = sampler != PRAD_SAMPLER_TABLE ? 0 : p.nsub == 1 ? (dense_launch(p) ? 2 : 1) : 0;
  return true;
}
template int push_emit_occupancy<double>(const StepParams<double>&, int, int, int, int, bool);

template <typename R>
cudaError_t launch_push_emit(const StepParams<R>& p, int field_kind, int sampler, int grid,
                             int block, cudaStream_t s) {
  switch (field_kind) {
    case PRAD_FIELD_CONST:
      return launch_field<R, PRAD_FIELD_CONST>(p, sampler, grid, block, s);
    case PRAD_FIELD_PLANE_WAVE:
      return launch_field<R, PRAD_FIELD_PLANE_WAVE>(p, sampler, grid, block, s);
    case PRAD_FIELD_YEE2D:
      return launch_field<R, PRAD_FIELD_YEE2D>(p, sampler, grid, block, s);
    default:
      return cudaErrorInvalidValue;
  }
}

// ---- diagnostics kernels ---------------------------------------------------
template <typename R>
__global__ void k_eval_sampler(const StepParams<R> P, const uint32_t* words,
                               R* x_out, R* g_out, int64_t n) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    R x, g;
    sample_x_g(P, words[4 * i], words[4 * i + 1], x, g);
    x_out[i] = x;
    g_out[i] = g;
  }
}

__global__ void k_philox(const uint32_t* ctr, uint32_t k0, uint32_t k1,
                         uint32_t* out, int64_t n) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
    const uint4 r = philox10(c, k0, k1);
    out[4 * i] = r.x; out[4 * i + 1] = r.y; out[4 * i + 2] = r.z; out[4 * i + 3] = r.w;
  }
}

template <typename R>
cudaError_t launch_eval_sampler(const StepParams<R>& p, const uint32_t* words,
                                R* x_out, R* g_out, int64_t n, cudaStream_t s) {
  const int block = 256;
  const int64_t want = (n + block - 1) / block;
  const int grid = static_cast<int>(want < 4096 ? (want > 0 ? want : 1) : 4096);
  k_eval_sampler<R><<<grid, block, 0, s>>>(p, words, x_out, g_out, n);
  return cudaGetLastError();
}

__global__ void k_angle_eval(const float* __restrict__ tab, const float* __restrict__ x,
                             const uint32_t* __restrict__ words, float* __restrict__ psi,
                             int64_t n) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    psi[i] = ang_psi<float>(tab, x[i], words[2 * i], words[2 * i + 1]);
}

cudaError_t launch_angle_eval(const float* tab, const float* x, const uint32_t* words,
                              float* psi, int64_t n, cudaStream_t s) {
  const int block = 256;
  const int64_t want = (n + block - 1) / block;
  const int grid = static_cast<int>(want < 4096 ? (want > 0 ? want : 1) : 4096);
  k_angle_eval<<<grid, block, 0, s>>>(tab, x, words, psi, n);
  return cudaGetLastError();
}

cudaError_t launch_philox(const uint32_t* ctr, uint32_t k0, uint32_t k1,
                          uint32_t* out, int64_t n, cudaStream_t s) {
  const int block = 256;
  const int64_t want = (n + block - 1) / block;
  const int grid = static_cast<int>(want < 4096 ? (want > 0 ? want : 1) : 4096);
  k_philox<<<grid, block, 0, s>>>(ctr, k0, k1, out, n);
  return cudaGetLastError();
}

template cudaError_t launch_push_emit<float>(const StepParams<float>&, int, int, int, int,
                                            cudaStream_t);
template cudaError_t launch_push_emit<double>(const StepParams<double>&, int, int, int, int,
                                             cudaStream_t);
template cudaError_t launch_push_emit_tiled<float>(const StepParams<float>&, int, int, cudaStream_t);
template cudaError_t launch_push_emit_tiled<double>(const StepParams<double>&, int, int, cudaStream_t);
template cudaError_t launch_eval_sampler<float>(const StepParams<float>&, const uint32_t*, float*, float*, int64_t, cudaStream_t);
template cudaError_t launch_eval_sampler<double>(const StepParams<double>&, const uint32_t*, double*, double*, int64_t, cudaStream_t);

#endif  // __CUDACC_RTC__
}  // namespace prad
