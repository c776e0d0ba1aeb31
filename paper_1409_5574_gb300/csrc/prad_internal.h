// Internal declarations shared by the host ABI (prad_api.cu) and the kernel
// translation units.  Nothing here is part of the public C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/prad.h"

namespace prad {

// ---- sampling table geometry --------------------------------------------
// g(x) = F(x) / S(x) is tabulated as per-interval cubics (Horner form in the
// local coordinate s in [0,1)) on two branches of the proposal of Eq. (11):
//   low branch  (x < a):  variable t = x^(1/3) = R'^(1/4) in [0, a^(1/3)],
//   high branch (x >= a): variable x in [a, kXmax].
constexpr int kN1 = 256;
constexpr int kN2 = 1024;
constexpr int kNTab = kN1 + kN2;
constexpr double kXmax = 45.0;

// Counter slots of the per-context device counter array.
enum Counter {
  kCursor = 0,   // photon append cursor (counts attempts, may exceed cap)
  kDnGt1 = 1,
  kClamp = 2,
  kChiGt1 = 3,
  kNan = 4,
  kMlpFallback = 5,
  kStatus = 6,
  kNumCounters = 8
};

struct alignas(32) Coef4d {
  double c0, c1, c2, c3;
};

template <typename R>
struct TabOf;
template <>
struct TabOf<float> {
  using T = float4;
};
template <>
struct TabOf<double> {
  using T = Coef4d;
};

template <typename R>
struct StepParams {
  // particle state (SoA, in place)
  R *x, *y, *z, *ux, *uy, *uz;
  const R* w;
  double *led_emit, *led_ll;  // already offset to particle 0
  int64_t n;
  int64_t t0;                 // global step of the first substep
  uint32_t pid0, ensemble, key0, key1;
  int32_t nsub;               // substeps in this launch
  int32_t rr_mode, heff_form, dims;
  // normalised constants
  R half_q_dtn, dtn, inv_dtn, abs_q;
  R cn_dt;      // (sqrt3 / 2pi) alpha dtn
  R eps_r;      // hbar omega_ref / (m c^2)
  R eps_r15;    // 1.5 eps_r
  R ll_coef;    // (2/3) alpha eps_r dtn
  // field
  R E[3], B[3];
  R E0, kc, hand, dir;         // plane wave
  uint64_t phase_t0, phase_step;  // fixed-point phase (cycles * 2^64)
  const float* yee[6];
  int32_t nx, ny;
  R inv_dx, inv_dy, x0, y0, Lx, Ly;
  // sampling table
  const typename TabOf<R>::T* tab;
  R t_scale, x_scale, a;
  uint64_t thr;
  // photons
  float *px, *py, *pz, *pnx, *pny, *pnz, *peps, *pw;
  uint32_t *ppid, *pstep;
  int64_t cap;
  unsigned long long* counters;
};

// Launchers (defined in the kernel translation units).
template <typename R>
cudaError_t launch_push_emit(const StepParams<R>& p, int field_kind, int grid,
                             int block, cudaStream_t s);
template <typename R>
cudaError_t launch_eval_sampler(const StepParams<R>& p, const uint32_t* words,
                                R* x_out, R* g_out, int64_t n, cudaStream_t s);
cudaError_t launch_philox(const uint32_t* ctr, uint32_t k0, uint32_t k1,
                          uint32_t* out, int64_t n, cudaStream_t s);
cudaError_t launch_ledger_reduce(const double* a, const double* b, int64_t n,
                                 double* partials, int nblocks, double* out,
                                 cudaStream_t s);

}  // namespace prad
