// Learned inverse-CDF sampler: a 3 -> 64 -> 64 -> 1 MLP with SiLU hidden
// activations, BF16 weights and FP32 accumulation.
//
// It replaces the tabulated inversion of the synchrotron spectrum (Eqs. (7),
// (8)): for a uniform r it returns x = omega / omega_c with G(x) = r, where G
// is the photon-number CDF int_0^x F(t)/t dt / (5 pi/3).  Inputs are
// (r, gamma, omega_c dt); in the classical model G does not depend on gamma
// or omega_c dt, and the network is trained to ignore them.
//
// Numerics (shared by training and evaluation):
//   features f = (logit(r)/8, clamp((ln gamma - c1)/s1), clamp((ln w - c2)/s2))
//   z1 = W1 f + b1 (BF16 weights, FP32 accumulate);  h1 = f16(silu(z1))
//   z2 = W2 h1 + b2 (tensor-core MMA, FP32 accumulate);  h2 = f16(silu(z2))
//   o = W3 h2 + b3 (FP32 accumulate);  ln x = prior(r) + kOutScale * o
// with the fixed prior(r) = ln(-ln(1 - r)) + 2 (1 - r) ln r, which carries
// both asymptotes of ln G^-1 (3 ln r at r -> 0, ln(-ln(1 - r)) at r -> 1),
// so the network only learns a bounded, smooth residual (in [-1.5, -0.2]).
// The weights are stored in BF16; a BF16 value is exact in f16 (11 > 8
// significant bits) down to 2^-17 in magnitude, so the f16 x f16 products of
// layers 2 and 3 multiply exactly the BF16 weights.  SiLU runs in packed f16
// arithmetic (tanh.approx.f16x2), within ~1 f16 ulp of f16(silu(z)).
#pragma once

#ifdef __CUDACC_RTC__
#include "rtc_prelude.h"
#endif
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#ifndef __CUDACC_RTC__
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstddef>
#endif

namespace prad {

constexpr int kHid = 64;
// parameter vector (FP32 master copy and the layout of get/set weights):
//   W1 [64][3], b1 [64], W2 [64][64] (row j = output unit), b2 [64],
//   W3 [64], b3
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kHid * 3;
constexpr int kOffW2 = kOffB1 + kHid;
constexpr int kOffB2 = kOffW2 + kHid * kHid;
constexpr int kOffW3 = kOffB2 + kHid;
constexpr int kOffB3 = kOffW3 + kHid;
constexpr int kNumParams = kOffB3 + 1;  // 4481

// feature normalisation (fixed; part of the model definition)
constexpr float kLogitScale = 0.125f;
constexpr float kLnGamC = 5.7565f;   // ln sqrt(10 * 1e4)
constexpr float kLnGamS = 3.4539f;   // ln sqrt(1e4 / 10)
constexpr float kLnWC = 8.2f;        // centre of ln(omega_c dt) over training
constexpr float kLnWS = 11.6f;
constexpr float kOutScale = 1.0f;
// uniforms the network was trained on; outside, the G^-1 table is used
constexpr float kRMin = 1.0e-7f;
constexpr float kRMax = 1.0f - 1.0e-7f;

// Device copy of the network: FP32 master parameters and the BF16 W2.
struct MlpDev {
  const float* params;                 // kNumParams FP32
  const __nv_bfloat16* w2;             // [64][64] BF16 (row j)
};

__device__ __forceinline__ float bf16_round(float v) {
  return __bfloat162float(__float2bfloat16(v));
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// SiLU from half arguments: h = hz + hz tanh(hz) with hz = z / 2 given
// (hz0, hz1); returns (silu(z0), silu(z1)) as f16x2 (z0 in the low half).
// f16(z / 2) = f16(z) / 2, so this equals silu_f16x2(z0, z1) bit for bit.
// (The packed tanh issues two MUFU operations, like two tanh.approx.f32; the
// FP32 form rounded to f16 measured 1.6% slower in the finishing kernel.)
__device__ __forceinline__ uint32_t silu_half_f16x2(float hz0, float hz1) {
  uint32_t hz, th, h;
  asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(hz) : "f"(hz1), "f"(hz0));
  asm("tanh.approx.f16x2 %0, %1;" : "=r"(th) : "r"(hz));
  asm("fma.rn.f16x2 %0, %1, %2, %3;" : "=r"(h) : "r"(hz), "r"(th), "r"(hz));
  return h;
}

// SiLU of two FP32 values in packed f16 arithmetic, h = hz + hz tanh(hz) with
// hz = z / 2; returns (silu(z0), silu(z1)) as f16x2 (z0 in the low half).
__device__ __forceinline__ uint32_t silu_f16x2(float z0, float z1) {
  uint32_t zz, hz, th, h;
  asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(zz) : "f"(z1), "f"(z0));
  asm("mul.rn.f16x2 %0, %1, %2;" : "=r"(hz) : "r"(zz), "r"(0x38003800u));
  asm("tanh.approx.f16x2 %0, %1;" : "=r"(th) : "r"(hz));
  asm("fma.rn.f16x2 %0, %1, %2, %3;" : "=r"(h) : "r"(hz), "r"(th), "r"(hz));
  return h;
}

__device__ __forceinline__ float silu(float z) {
  // z * sigmoid(z) = 0.5 z (1 + tanh(z / 2))
  float t;
  asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(0.5f * z));
  return 0.5f * z * (1.0f + t);
}

__device__ __forceinline__ float silu_grad(float z) {
  // d/dz [z sigmoid(z)] = s + z s (1 - s),  s = sigmoid(z)
  float t;
  asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(0.5f * z));
  const float s = 0.5f * (1.0f + t);
  return s + z * s * (1.0f - s);
}

// -ln(1 - r) for r in (0, 1): below r = 1/64 the series r (1 + r/2 + r^2/3 +
// r^3/4) (truncation < r^4 / 5 relative, < 2e-8); above it the MUFU
// logarithm of 1 - r (exact for r >= 1/2, relatively within 2^-24 below;
// the logarithm's absolute error ~2^-22 is < 1e-5 of |ln(1 - r)| >= 1/64).
__device__ __forceinline__ float neg_log1m(float r) {
  const float s = r * fmaf(r, fmaf(r, fmaf(r, 0.25f, 1.0f / 3.0f), 0.5f), 1.0f);
  const float l = -__logf(1.0f - r);
  return r < 0.015625f ? s : l;
}

__device__ __forceinline__ float mlp_prior(float r) {
  return __logf(neg_log1m(r)) + 2.0f * (1.0f - r) * __logf(r);
}

__device__ __forceinline__ float3 mlp_features(float r, float gamma, float wdt) {
  const float lg = (__logf(r) - __logf(1.0f - r)) * kLogitScale;
  float f1 = (__logf(gamma) - kLnGamC) * (1.0f / kLnGamS);
  float f2 = (__logf(wdt) - kLnWC) * (1.0f / kLnWS);
  f1 = fminf(fmaxf(f1, -1.0f), 1.0f);
  f2 = fminf(fmaxf(f2, -1.0f), 1.0f);
  return make_float3(lg, f1, f2);
}

// G^-1 table: ln x at nodes uniform in logit(r) on [-kGiL, kGiL], linear
// interpolation (training targets, fallback, device-side spectral check).
constexpr int kGiN = 8192;
constexpr float kGiL = 24.0f;

__device__ __forceinline__ float ginv_ln(const float* tab, float r) {
  const float lg = __logf(r) - __logf(1.0f - r);
  const float u = (fminf(fmaxf(lg, -kGiL), kGiL) + kGiL) * ((kGiN - 1) / (2.0f * kGiL));
  int i = static_cast<int>(u);
  i = min(max(i, 0), kGiN - 2);
  const float s = u - static_cast<float>(i);
  return fmaf(s, tab[i + 1] - tab[i], tab[i]);
}

}  // namespace prad
