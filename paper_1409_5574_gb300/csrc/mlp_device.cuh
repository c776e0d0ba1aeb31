// Learned inverse-CDF sampler: a 3 -> 64 -> 64 -> 1 MLP with SiLU hidden
// activations, BF16 weights and FP32 accumulation, evaluated on tiles of 16
// samples per warp with the m16n8k16 BF16 tensor-core MMA.
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
// The weights are stored in BF16; a BF16 value is exact in f16 (11 > 8
// significant bits) down to 2^-17 in magnitude, so the f16 x f16 MMAs of
// layers 2 and 3 multiply exactly the BF16 weights.  SiLU runs in packed f16
// arithmetic (tanh.approx.f16x2), within ~1 f16 ulp of f16(silu(z)).  The
// tile evaluator forms z1 on the tensor cores as well: each feature and
// each bias enters as the sum of two BF16 numbers (high part + rounded
// remainder, 2^-17 relative), so z1 agrees with the FP32 form to ~1e-6.
// with the fixed prior(r) = ln(-ln(1 - r)) + 2 (1 - r) ln r, which carries
// both asymptotes of ln G^-1 (3 ln r at r -> 0, ln(-ln(1 - r)) at r -> 1),
// so the network only learns a bounded, smooth residual (in [-1.5, -0.2]).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstddef>

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

// Shared-memory image of the network used by the tile evaluator.
constexpr int kW2Ld = kHid + 8;  // padded row (bank-conflict free B loads)
struct MlpSmem {
  float4 w1b1[kHid];                       // (W1 row j, b1 j)
  float b2[kHid];
  float w3[kHid];
  float b3;
  float pad[3];
  __nv_bfloat16 w2[kHid * kW2Ld];          // W2 row-major [j][i], padded
  // layer 1 as the B operand of m16n8k16 MMAs (K = 16 x N = 64 units):
  // rows k = 0..2 W1[j][k], k = 3..5 W1[j][k-3] (they multiply the
  // features' low parts), k = 6, 7 the high and low BF16 parts of b1[j],
  // k >= 8 zero.  w1f[lane][nt] holds the lane's b0 register of n-tile nt.
  uint32_t w1f[32][8];
  // the tile evaluator's layer 2 in f16, halved (exact): W2 / 2 and b2 / 2
  __half w2h[kHid * kW2Ld];
  float b2h[kHid];
  // layer 3 as the B operand (K = 64 x N = 8, W3 in column 0, zero
  // elsewhere): w3f[lane][2q + u] = the lane's b_u register of k-step q
  uint32_t w3f[32][8];
};

static_assert(sizeof(MlpSmem) % 16 == 0 && offsetof(MlpSmem, w2) % 16 == 0 &&
                  offsetof(MlpSmem, w1f) % 16 == 0 && offsetof(MlpSmem, w2h) % 16 == 0 &&
                  offsetof(MlpSmem, w3f) % 16 == 0 && offsetof(MlpSmem, b2h) % 8 == 0,
              "16-byte alignment of the network image (uint4 and ldmatrix reads)");

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

// Weights enter as BF16 (rounded from the FP32 master), biases as FP32.
__device__ __forceinline__ void mlp_load_smem(MlpSmem& s, const MlpDev& d) {
  for (int j = threadIdx.x; j < kHid; j += blockDim.x) {
    s.w1b1[j] = make_float4(bf16_round(d.params[kOffW1 + 3 * j]),
                            bf16_round(d.params[kOffW1 + 3 * j + 1]),
                            bf16_round(d.params[kOffW1 + 3 * j + 2]), d.params[kOffB1 + j]);
    s.b2[j] = d.params[kOffB2 + j];
    s.w3[j] = bf16_round(d.params[kOffW3 + j]);
  }
  if (threadIdx.x == 0) s.b3 = d.params[kOffB3];
  for (int e = threadIdx.x; e < kHid * kHid; e += blockDim.x) {
    const int j = e / kHid, i = e - j * kHid;
    s.w2[j * kW2Ld + i] = d.w2[e];
  }
  for (int e = threadIdx.x; e < 32 * 8; e += blockDim.x) {
    const int lane = e >> 3, nt = e & 7;
    const int j = 8 * nt + (lane >> 2), t = lane & 3;
    float v[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int k = 2 * t + u;
      const float b1 = d.params[kOffB1 + j];
      const float b1h = bf16_round(b1);
      v[u] = k < 3 ? bf16_round(d.params[kOffW1 + 3 * j + k])
                   : (k < 6 ? bf16_round(d.params[kOffW1 + 3 * j + k - 3])
                            : (k == 6 ? b1h : bf16_round(b1 - b1h)));
    }
    // halved (exact): the layer-1 accumulators hold z1 / 2
    s.w1f[lane][nt] = pack_bf16x2(0.5f * v[0], 0.5f * v[1]);
  }
  // halved (exact): the layer-2 accumulators hold z2 / 2
  for (int e = threadIdx.x; e < kHid * kHid; e += blockDim.x) {
    const int j = e / kHid, i = e - j * kHid;
    s.w2h[j * kW2Ld + i] = __float2half_rn(0.5f * __bfloat162float(d.w2[e]));
  }
  for (int j = threadIdx.x; j < kHid; j += blockDim.x) s.b2h[j] = 0.5f * d.params[kOffB2 + j];
  for (int e = threadIdx.x; e < 32 * 8; e += blockDim.x) {
    const int lane = e >> 3, q = (e & 7) >> 1, u = e & 1;
    const int g = lane >> 2, t = lane & 3;
    const int i0 = 16 * q + 8 * u + 2 * t;
    uint32_t v = 0u;
    if (g == 0) {
      const __half2 h = __halves2half2(__float2half_rn(bf16_round(d.params[kOffW3 + i0])),
                                       __float2half_rn(bf16_round(d.params[kOffW3 + i0 + 1])));
      v = *reinterpret_cast<const uint32_t*>(&h);
    }
    s.w3f[lane][e & 7] = v;
  }
}

// SiLU from half arguments: h = hz + hz tanh(hz) with hz = z / 2 given
// (hz0, hz1); returns (silu(z0), silu(z1)) as f16x2 (z0 in the low half).
// f16(z / 2) = f16(z) / 2, so this equals silu_f16x2(z0, z1) bit for bit.
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

// D = A(16x16, row) * B(16x8, col) + C, BF16 inputs, FP32 accumulate.
// Fragment ownership (g = lane / 4, t = lane % 4):
//   a0: A[g][2t..2t+1]   a1: A[g+8][2t..]   a2: A[g][2t+8..]   a3: A[g+8][2t+8..]
//   b0: B[2t..2t+1][g]   b1: B[2t+8..2t+9][g]
//   c0,c1: C[g][2t..2t+1]   c2,c3: C[g+8][2t..2t+1]
__device__ __forceinline__ void mma_bf16_16816(float c[4], uint32_t a0, uint32_t a1,
                                               uint32_t a2, uint32_t a3, uint32_t b0,
                                               uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// D = A(16x16, row) * B(16x8, col) + C, f16 inputs, FP32 accumulate (the
// fragment layout of mma_bf16_16816).
__device__ __forceinline__ void mma_f16_16816(float c[4], uint32_t a0, uint32_t a1,
                                              uint32_t a2, uint32_t a3, uint32_t b0,
                                              uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float mlp_prior(float r) {
  return __logf(-log1pf(-r)) + 2.0f * (1.0f - r) * __logf(r);
}

__device__ __forceinline__ float3 mlp_features(float r, float gamma, float wdt) {
  const float lg = (__logf(r) - __logf(1.0f - r)) * kLogitScale;
  float f1 = (__logf(gamma) - kLnGamC) * (1.0f / kLnGamS);
  float f2 = (__logf(wdt) - kLnWC) * (1.0f / kLnWS);
  f1 = fminf(fmaxf(f1, -1.0f), 1.0f);
  f2 = fminf(fmaxf(f2, -1.0f), 1.0f);
  return make_float3(lg, f1, f2);
}

// Four 8x8 BF16 matrices from shared memory in the MMA fragment layout
// (lane l supplies the address of row l % 8 of matrix l / 8).
__device__ __forceinline__ void ldmatrix_x4(uint32_t d[4], const void* row_addr) {
  const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(row_addr));
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3])
               : "r"(a));
}

// Columns 2t, 2t+1 of a layer-1 A row [f0h f1h f2h f0l f1l f2l 1 1 0 ...]
// (h: BF16 high part, l: the remainder, rounded to BF16 when packed).
__device__ __forceinline__ uint32_t mlp_feature_pair(float3 f, int t) {
  const float h0 = bf16_round(f.x), h1 = bf16_round(f.y), h2 = bf16_round(f.z);
  const float a = t == 0 ? h0 : (t == 1 ? h2 : (t == 2 ? f.y - h1 : 1.0f));
  const float b = t == 0 ? h1 : (t == 1 ? f.x - h0 : (t == 2 ? f.z - h2 : 1.0f));
  return pack_bf16x2(a, b);
}

// Warp-collective: the 16 rows of a tile are the features of lanes' rows
// g and g+8 (f_lo, f_hi); returns kOutScale * o (ln x minus the prior) of rows
// g (out_lo) and g+8 (out_hi), valid in lane 4g.  Every layer runs on the
// tensor cores; an accumulator fragment of one layer, after SiLU, is the A
// fragment of the next (n-tiles 2q, 2q+1 -> k-step q).
__device__ __forceinline__ void mlp_tile16(const MlpSmem& S, float3 f_lo, float3 f_hi,
                                           float& out_lo, float& out_hi) {
  const int lane = threadIdx.x & 31;
  const int t = lane & 3;
  // layer 1 (BF16, split features and bias)
  const uint32_t fa0 = mlp_feature_pair(f_lo, t), fa1 = mlp_feature_pair(f_hi, t);
  const uint4 wlo = *reinterpret_cast<const uint4*>(&S.w1f[lane][0]);
  const uint4 whi = *reinterpret_cast<const uint4*>(&S.w1f[lane][4]);
  const uint32_t wb[8] = {wlo.x, wlo.y, wlo.z, wlo.w, whi.x, whi.y, whi.z, whi.w};
  uint32_t a[4][4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float c0[4] = {0.0f, 0.0f, 0.0f, 0.0f}, c1[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    mma_bf16_16816(c0, fa0, fa1, 0u, 0u, wb[2 * q], 0u);
    mma_bf16_16816(c1, fa0, fa1, 0u, 0u, wb[2 * q + 1], 0u);
    a[q][0] = silu_half_f16x2(c0[0], c0[1]);
    a[q][1] = silu_half_f16x2(c0[2], c0[3]);
    a[q][2] = silu_half_f16x2(c1[0], c1[1]);
    a[q][3] = silu_half_f16x2(c1[2], c1[3]);
  }
  // layers 2 and 3 (f16): the accumulators start from b2 / 2; the SiLU of
  // each pair of n-tiles is one k-step of layer 3
  const uint4 vlo = *reinterpret_cast<const uint4*>(&S.w3f[lane][0]);
  const uint4 vhi = *reinterpret_cast<const uint4*>(&S.w3f[lane][4]);
  const uint32_t w3b[8] = {vlo.x, vlo.y, vlo.z, vlo.w, vhi.x, vhi.y, vhi.z, vhi.w};
  const int m = lane >> 3, r = lane & 7;
  float o[4] = {S.b3, 0.0f, S.b3, 0.0f};
#pragma unroll
  for (int q3 = 0; q3 < 4; ++q3) {
    // n-tiles 2 q3 (c0) and 2 q3 + 1 (c1): two independent MMA chains
    const float2 b0 = *reinterpret_cast<const float2*>(&S.b2h[16 * q3 + 2 * t]);
    const float2 b1 = *reinterpret_cast<const float2*>(&S.b2h[16 * q3 + 8 + 2 * t]);
    float c0[4] = {b0.x, b0.y, b0.x, b0.y}, c1[4] = {b1.x, b1.y, b1.x, b1.y};
#pragma unroll
    for (int qq = 0; qq < 4; qq += 2) {
      uint32_t w0[4], w1[4];
      const int col = 16 * (qq + (m >> 1)) + 8 * (m & 1);
      ldmatrix_x4(w0, S.w2h + (16 * q3 + r) * kW2Ld + col);
      ldmatrix_x4(w1, S.w2h + (16 * q3 + 8 + r) * kW2Ld + col);
      mma_f16_16816(c0, a[qq][0], a[qq][1], a[qq][2], a[qq][3], w0[0], w0[1]);
      mma_f16_16816(c1, a[qq][0], a[qq][1], a[qq][2], a[qq][3], w1[0], w1[1]);
      mma_f16_16816(c0, a[qq + 1][0], a[qq + 1][1], a[qq + 1][2], a[qq + 1][3], w0[2], w0[3]);
      mma_f16_16816(c1, a[qq + 1][0], a[qq + 1][1], a[qq + 1][2], a[qq + 1][3], w1[2], w1[3]);
    }
    uint32_t h[4];
    h[0] = silu_half_f16x2(c0[0], c0[1]);  // row g, n-tile 2 q3
    h[1] = silu_half_f16x2(c0[2], c0[3]);  // row g + 8
    h[2] = silu_half_f16x2(c1[0], c1[1]);  // row g, n-tile 2 q3 + 1
    h[3] = silu_half_f16x2(c1[2], c1[3]);
    // k-step q3 of layer 3: a0 = (g, n-tile 2q3), a1 = (g+8, 2q3),
    // a2 = (g, 2q3+1), a3 = (g+8, 2q3+1)
    mma_f16_16816(o, h[0], h[1], h[2], h[3], w3b[2 * q3], w3b[2 * q3 + 1]);
  }
  // column 0 of the output tile: rows g (o[0]) and g + 8 (o[2]) in lane 4g
  out_lo = kOutScale * o[0];
  out_hi = kOutScale * o[2];
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
