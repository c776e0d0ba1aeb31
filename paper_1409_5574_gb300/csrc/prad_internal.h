// Internal declarations shared by the host ABI (prad_api.cu) and the kernel
// translation units.  Nothing here is part of the public C ABI.
#pragma once

#ifdef __CUDACC_RTC__
#include "rtc_prelude.h"
#else
#include <cuda_runtime.h>
#include <stdint.h>
#endif

#include "prad.h"  // include/ is on the include path
#include "mlp_device.cuh"

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
// Proposal constant of Eq. (11): root of a^(4/3) + (7/9) e^(-a) = 1, and its
// cube root (the low branch's end, t = a^(1/3); correctly rounded).
constexpr double kA = 0.69020670216845766;
constexpr double kCbrtA = 0x1.c47a11f9c597ep-1;
// round(a^(4/3) 2^64): 64-bit words W below it take the x < a branch.
constexpr uint64_t kThr = 0x9C26B9CE251FFCB8ull;
// Table coordinates: u = t kTScale on the low branch, (x - a) kXScale on the
// high one.  The step kernels take these (and kA, kThr) as compile-time
// constants: immediate operands instead of parameter loads in every step.
constexpr double kTScale = kN1 / kCbrtA;
constexpr double kXScale = kN2 / (kXmax - kA);

// ---- angular spread of the emission (Eqs. (5)-(6), PRAD_DIAG_ANGLE_SPREAD)
// psi = gamma theta, theta the angle out of the plane of the orbit, is drawn
// from Eq. (5)'s density at the photon's x = omega / omega_c.  The table
// holds y = psi / (v s(x)) on kAngNL rows uniform in ln x over
// [kAngLx0, kAngLx1] and kAngNV columns uniform in v = sqrt(-ln(1 - u))
// over [0, kAngVmax] (u the uniform, one-sided CDF), with
// s(x) = (2/x)^(1/3) (1 + x)^(-1/6), psi's scale for small and large x;
// bilinear interpolation, x clamped into the rows' range.
constexpr int kAngNL = 225;
constexpr int kAngNV = 257;
constexpr double kAngLx0 = -18.420680743952367;  // ln 1e-8
constexpr double kAngLx1 = 3.6888794541139363;   // ln 40
constexpr double kAngVmax = 4.8;                 // u <= 1 - 2^-33: v <= 4.79

// float -> double by the IEEE-754 formats (normal numbers: the exponent
// rebiased by 1023 - 127 = 896, the 23 fraction bits moved to the top of
// the 52), with integer instructions; zeros, subnormals, infinities and NaNs
// take the conversion instruction.  Exact, like the conversion; it keeps the
// learned sampler's per-record ledger increments off the FP64 pipe, which
// runs at a small fraction of the FP32 rate on GB300 (in the step kernels,
// which are bound by instruction issue, the conversion instruction is
// cheaper: one-step launches lost 3% with this form).
__device__ __forceinline__ double f32_to_f64(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t e = (b >> 23) & 0xffu;
  if (e == 0u || e == 0xffu) return static_cast<double>(f);
  const uint32_t hi = (b & 0x80000000u) | (((b & 0x7fffffffu) >> 3) + (896u << 20));
  return __hiloint2double(static_cast<int>(hi), static_cast<int>(b << 29));
}

// Counter slots of the per-context device counter array.
enum Counter {
  kCursor = 0,   // photon append cursor (counts attempts, may exceed cap)
  kDnGt1 = 1,
  kClamp = 2,
  kChiGt1 = 3,
  kNan = 4,
  kMlpFallback = 5,
  kStatus = 6,
  kMlpDone = 7,    // learned sampler: records [0, kMlpDone) have their energy
  kMlpBlocks = 8,  // learned sampler: blocks of the finishing kernel done
  kWiggler = 9,    // PRAD_DIAG_WIGGLER: steps outside the synchrotron regime
  kNumCounters = 16
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
  const uint32_t* pid;        // optional explicit ids (NULL: pid0 + i)
  double *led_emit, *led_ll;  // already offset to the entry of id pid0
  int64_t led_n;              // ledger entries available from that offset
  int64_t n;
  int64_t t0;                 // global step of the first substep
  uint32_t pid0, ensemble, key0, key1;
  int32_t nsub;               // substeps in this launch
  int32_t rr_mode, heff_form, dims;
  int32_t field_kind;         // batch kernel: per-ensemble field model
  int32_t pad_fk;
  // normalised constants
  R half_q_dtn, dtn, inv_dtn, abs_q;
  R cn_dt;      // (sqrt3 / 2pi) alpha dtn
  R eps_r;      // hbar omega_ref / (m c^2)
  R eps_r15;    // 1.5 eps_r
  R ll_coef;    // (2/3) alpha eps_r dtn
  // field
  R E[3], B[3];
  R E0, kc, kc_lo, hand, dir;  // plane wave (kc + kc_lo: k/2pi to ~2^-48)
  R pw_ez, pw_by, pw_bz;       // plane wave: hand E0, -dir hand E0, dir E0 (exact)
  uint64_t phase_t0, phase_step;  // fixed-point phase (cycles * 2^64)
  const float* yee[6];
  int32_t nx, ny;
  R inv_dx, inv_dy, x0, y0, Lx, Ly;
  R inv_dx_lo, inv_dy_lo;      // low parts of 1/dx, 1/dy (float-float)
  // sampling table
  const typename TabOf<R>::T* tab;
  R t_scale, x_scale, a;
  uint64_t thr;
  // photons
  float *px, *py, *pz, *pnx, *pny, *pnz, *peps, *pw;
  uint32_t *ppid, *pstep;
  float4* ppend;              // learned sampler: (r, gamma, eps_c, ledger index) per slot
  int64_t cap;
  unsigned long long* counters;
  int64_t led_off;            // ledger entry of id pid0 in the context's ledger
  double* led_base;           // the context's emitted-energy ledger (entry 0)
  // super-photon control: trials per step, selection probability
  int32_t ntry;               // >= 1
  int32_t diag;               // PRAD_DIAG_* mask
  R inv_ntry, sel_q, inv_sel_q;
  R wl;                       // plane wave: omega_L / omega_ref
  // learned sampler (direct scheme): expected photons per step = cp_dt Omega
  R cp_dt;                    // (5 sqrt3 / 6) alpha dtn
  MlpDev mlp;
  const float* ginv;          // G^-1 table (ln x on a logit(r) grid)
  const float* ang;           // angular-spread table (PRAD_DIAG_ANGLE_SPREAD), else null
  // tile-sorted Yee gather (k_push_emit_tiled)
  const int4* work;           // (tile, first, end, 0) per work item
  const unsigned int* work_count;
  int32_t ntx;                // tiles along x
  // Philox4x32-10 round keys of (key0, key1) (philox_round_keys), read
  // from the kernel's parameter space by the kernels that take StepParams
  // by value
  uint32_t rkey[20];
};

// Tile geometry of the sorted Yee gather: 32 x 32-cell tiles, staged with a
// 6-cell halo (44 x 44 values per field component) in shared memory.
constexpr int kTile = 32;
constexpr int kHalo = 6;
constexpr int kStageW = kTile + 2 * kHalo;
constexpr int kTileSmemBytes = 6 * kStageW * kStageW * 4;
constexpr int kChunk = 4096;  // particles per work item of the tiled kernel

struct SortBuffers {
  void* tmp[7];               // scratch copies of x y z ux uy uz w
  uint32_t* tmp_pid;
  unsigned int* counts;       // per tile
  unsigned int* starts;       // per tile + 1 (exclusive scan)
  unsigned int* cursor;       // per tile scatter cursors
  int4* work;                 // work items of the tiled kernel
  unsigned int* work_count;
  int64_t capacity;           // particles
  int32_t ntiles, max_work;
};

// Batched ensembles (k_push_emit_batch): per-ensemble step parameters in a
// device array, the prefix sum of work items per ensemble, and the atomic
// work counter the persistent grid draws from.
struct BatchParams {
  const StepParams<float>* ens;
  const int64_t* item_off;     // n_ens + 1 entries
  unsigned long long* next_item;
  int64_t total_items;
  int64_t step_base;           // steps of this call done by earlier launches
  int32_t n_ens;
  int32_t chunk;               // particles per work item
  int32_t nsub;                // steps of this launch
  int32_t pad;
  uint32_t rkey[20];           // Philox round keys of the context's seed
  // per-CTA busy SM clocks, accumulated over a call's launches (load
  // balance); may be null
  unsigned long long* busy;
};

// Philox4x32-10 round keys of a 64-bit seed: (key0 + r 0x9E3779B9,
// key1 + r 0xBB67AE85) at rk[2r], rk[2r + 1], r = 0..9.
inline void philox_round_keys(uint64_t seed, uint32_t* rk) {
  const uint32_t k0 = static_cast<uint32_t>(seed & 0xffffffffull);
  const uint32_t k1 = static_cast<uint32_t>(seed >> 32);
  for (uint32_t r = 0; r < 10; ++r) {
    rk[2 * r] = k0 + r * 0x9E3779B9u;
    rk[2 * r + 1] = k1 + r * 0xBB67AE85u;
  }
}

#ifndef __CUDACC_RTC__
// Launchers (defined in the kernel translation units).
// std_cfg: the standard configuration (LL kick applied, field form of H_eff)
// in every ensemble, which selects the variant with those modes fixed at
// compile time (as for k_push_emit)
cudaError_t launch_push_emit_batch(const BatchParams& bp, int sampler, bool ctrl, bool std_cfg,
                                   int grid, int block, cudaStream_t s);
template <typename R>
int push_emit_occupancy(const StepParams<R>& p, int field_kind, int sampler, int nsub, int block,
                        bool ctrl);
int batch_max_blocks_per_sm(int block, int sampler, bool ctrl, bool std_cfg);
template <typename R>
cudaError_t launch_push_emit(const StepParams<R>& p, int field_kind, int sampler, int grid,
                             int block, cudaStream_t s);
template <typename R>
cudaError_t launch_eval_sampler(const StepParams<R>& p, const uint32_t* words,
                                R* x_out, R* g_out, int64_t n, cudaStream_t s);
cudaError_t launch_philox(const uint32_t* ctr, uint32_t k0, uint32_t k1,
                          uint32_t* out, int64_t n, cudaStream_t s);
template <typename R>
cudaError_t launch_push_emit_tiled(const StepParams<R>& p, int max_work, int block,
                                   cudaStream_t s);
template <typename R>
cudaError_t launch_tile_sort(R* arr[7], uint32_t* pid, int64_t n, const SortBuffers& b,
                             int nx, int ny, double x0, double y0, double inv_dx,
                             double inv_dy, cudaStream_t s);
size_t mlp_train_smem_bytes();
cudaError_t launch_mlp_train_block(const MlpDev& dev, uint32_t key0, uint32_t key1,
                                   uint64_t first, int64_t n_valid, int64_t n_total,
                                   const float4* explicit_samples, const float* ginv,
                                   float lng_lo, float lng_span, float lnh_lo,
                                   float lnh_span, float wdt_per_H_g2, float* partial,
                                   float* loss_part, int nblocks, unsigned long long* status,
                                   cudaStream_t s);
cudaError_t launch_mlp_reduce_adam(const float* partial, int nblocks, const float* loss_part,
                                   float* grad, float* params, float* m, float* v,
                                   __nv_bfloat16* w2, float lr, float b1t, float b2t,
                                   int apply, float* loss_out, float loss_scale,
                                   cudaStream_t s);
// withhold != 0: the self-test of the bounded tensor-core waits (no MMA
// completion is signalled; every wait runs out and status bit 2 is set)
cudaError_t launch_mlp_eval(const MlpDev& dev, const float* in, float* out, int64_t n,
                            unsigned long long* status, int withhold, cudaStream_t s);
// Energies of the learned sampler's records appended since the last call:
// records [counters[kMlpDone], min(cursor, cap)) get x from the network (table
// fallback), eps = x eps_c, and their emitted-energy ledger entries.
struct MlpFinishArgs {
  MlpDev mlp;
  const float* ginv;
  float* eps;                 // record energies (written)
  const float* weight;        // record weights
  const float4* pend;         // (r, gamma, eps_c, ledger index or -1)
  unsigned long long* counters;
  double* led_emit;           // the context's ledger, entry 0
  int64_t cap;
  float wdt_per_eps;          // omega_c dt / eps_c = dt / eps_r (normalised)
  int32_t check_output;       // MLP_FALLBACK: invalid network output -> table
};
cudaError_t launch_mlp_finish(const MlpFinishArgs& a, int grid, cudaStream_t s);
// Angular histogram of the held photon records (diagnostics.cu).
constexpr int kMaxAngularBins = 8192;  // 64 KB of FP64 bins in shared memory
struct AngularArgs {
  const float *nx, *ny, *nz, *eps, *weight;
  const unsigned long long* cursor;
  int64_t cap;
  double axis[3], e1[3], e2[3];  // orthonormal frame: polar axis, phi = 0, phi = pi/2
  double theta_max;
  int32_t ntheta, nphi;
  double* out;                   // device, ntheta x nphi
};
cudaError_t launch_angular_hist(const AngularArgs& a, int grid, cudaStream_t s);
int mlp_finish_blocks_per_sm();
cudaError_t launch_ginv_eval(const float* tab, const float* r, float* out, int64_t n,
                             cudaStream_t s);
// psi of the angular spread for x[i] and the Philox words words[2i],
// words[2i + 1] (the table lookup of the step kernels; push_emit.cu)
cudaError_t launch_angle_eval(const float* tab, const float* x, const uint32_t* words,
                              float* psi, int64_t n, cudaStream_t s);
cudaError_t launch_ledger_reduce(const double* a, const double* b, int64_t n,
                                 double* partials, int nblocks, double* out,
                                 cudaStream_t s);

// Run-time specialised kernels (spec.cu): the standard FP32 plane-wave and
// Yee-grid step kernels compiled by NVRTC with the context's constants as
// literals.  A variant names the kernel (k_push_emit, or k_push_emit_tiled
// when tiled), field model, sampler, prefetch mode and plane-wave signs.
// spec_get returns its kernel for these parameters' constants, compiling it
// on first use (an error, with a message in msg, when NVRTC or the driver
// cannot provide it).
struct SpecVariant {
  int32_t tiled, field, samp, pf, pws;
};
struct SpecFn;
struct SpecCache;
SpecCache* spec_create();
void spec_destroy(SpecCache* c);
cudaError_t spec_get(SpecCache* c, int device, const StepParams<float>& p, const SpecVariant& v,
                     const SpecFn** out, char* msg, size_t msg_len);
int spec_occupancy(const SpecFn* f, int block);
// grid blocks of block threads; the tiled kernel gets its tile's dynamic
// shared memory
cudaError_t spec_launch(const SpecFn* f, const StepParams<float>& p, int grid, int block,
                        cudaStream_t s);
// Whether a launch with these parameters runs a specialisable variant (FP32
// standard configuration of the plane wave or the Yee grid, no control or
// diagnostics; the tiled kernel with the table sampler), and which.
bool push_emit_spec_variant(const StepParams<float>& p, int field_kind, int sampler, bool tiled,
                            SpecVariant* v);
#endif  // __CUDACC_RTC__

}  // namespace prad
