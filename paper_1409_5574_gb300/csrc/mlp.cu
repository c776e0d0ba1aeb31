// Training and evaluation kernels of the learned inverse-CDF sampler
// (mlp_device.cuh): sample generation with the device G^-1 table, a fused
// forward + backward pass per block of 128 samples on the tcgen05 tensor
// cores (f16 forward, BF16 gradient products, accumulators in TMEM),
// per-block partial gradients, and a deterministic reduction + Adam update;
// the evaluators (the learned sampler's finishing kernel and prad_mlp_eval)
// run the network on the tcgen05 tensor cores too (mlp_tc.cuh).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "mlp_device.cuh"
#include "mlp_tc.cuh"
#include "prad_internal.h"

namespace prad {

__device__ __forceinline__ uint4 philox10_mlp(uint4 c, uint32_t k0, uint32_t k1) {
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

namespace {

constexpr int kTB = 128;  // samples per block (one tile: one sample per thread)
constexpr int kTZ = kHid + 1;  // padded FP32 rows: column sums without bank conflicts

// Canonical K-major strides (bytes per 8-row group) of the training tiles:
// K = 64 (delta2 [s][j], W2^T [i][j]) and K = 128 (delta2^T [j][s], h1^T [i][s]).
constexpr uint32_t kTrSbo64 = (kHid / 8) * 128;
constexpr uint32_t kTrSbo128 = (kTB / 8) * 128;

// Shared memory of the training kernel (~104 KB: two CTAs per SM).  The
// operand tiles are in the canonical K-major layout of the tensor cores (no
// swizzle, mlp_tc.cuh).  The forward operands are dead once the forward MMA
// has completed, and the backward operands take their place.  The dW2 product
// reads its A operand as 128 rows from d2t: rows 64..127 are h1t's bytes
// (d2t is followed by h1t), and give TMEM lanes 64..127 that are never read.
struct alignas(128) TrainTcSmem {
  union {
    struct {
      uint16_t a2[kTB * kTcK2];    // [h1 f16 | 1 1 0..] (forward layer 2, A)
      uint16_t b2[kHid * kTcK2];   // halved W2 | split b2, f16 (forward layer 2, B)
    } fwd;
    struct {
      uint16_t d2[kTB * kHid];     // bf16 delta2 [s][j] (delta1, A)
      uint16_t w2t[kHid * kHid];   // BF16 W2^T [i][j] (delta1, B)
    } bwd;
  } u;
  uint16_t d2t[kHid * kTB];        // bf16 delta2^T [j][s] (dW2, A rows 0..63)
  uint16_t h1t[kHid * kTB];        // bf16(silu(z1))^T [i][s] (dW2, B)
  float z1[kTB][kTZ];              // z1, then delta1
  float wsum[kTB / 32][2 * kHid];  // per-warp sums of dL/dW3 and dL/db2
  float4 w1b1[kHid];               // (BF16 W1 row j, b1 j)
  float w3[kHid];
  float x[kTB][4];                 // features; x[s][3] = 0 valid, -1 padding
  float tgt[kTB];
  float wgt[kTB];
  float loss[kTB];
  float dout[kTB];
  float b3;
  uint32_t tmem;
  uint64_t bar;
};
static_assert(offsetof(TrainTcSmem, u.fwd.b2) % 128 == 0 &&
                  offsetof(TrainTcSmem, u.bwd.w2t) % 128 == 0 &&
                  offsetof(TrainTcSmem, d2t) % 128 == 0 &&
                  offsetof(TrainTcSmem, h1t) == offsetof(TrainTcSmem, d2t) + kHid * kTB * 2 &&
                  offsetof(TrainTcSmem, bar) % 8 == 0,
              "operand and mbarrier alignment; h1t directly after d2t");
static_assert(tc_off(kTB - 1, kTB - 1, kTrSbo128) < 2 * kHid * kTB &&
                  tc_off(kHid - 1, kTB - 1, kTrSbo128) < kHid * kTB &&
                  tc_off(kTB - 1, kHid - 1, kTrSbo64) < kTB * kHid &&
                  tc_off(kHid - 1, kHid - 1, kTrSbo64) < kHid * kHid,
              "training tiles stay inside their arrays (dW2's A: d2t and h1t)");

// Warp sums of 64 per-lane values v[0..63] (recursive halving: each round a
// lane keeps one half of its range and adds its partner's copy of it); lane l
// ends with the sums of entries 2l and 2l + 1 in v[0] and v[1].
__device__ __forceinline__ void warp_sum64(float (&v)[kHid], int lane) {
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    const int half = 32 >> r;           // entries kept after this round
    const int bit = 16 >> r;            // partner lane distance
    const bool upper = (lane & bit) != 0;
#pragma unroll
    for (int k = 0; k < half; ++k) {
      const float keep = upper ? v[k + half] : v[k];
      const float send = upper ? v[k] : v[k + half];
      v[k] = keep + __shfl_xor_sync(0xffffffffu, send, bit);
    }
  }
}

// Training samples: r from a Philox uniform (tag 3), gamma log-uniform in
// [g_lo, g_hi], H log-uniform in [h_lo, h_hi] T, omega_c dt = 1.5 e H / m
// gamma^2 dt; target ln G^-1(r) from the device table.
struct SampleSpec {
  uint32_t key0, key1;
  uint64_t first;           // global index of the block's first sample
  float lng_lo, lng_span, lnh_lo, lnh_span;
  float wdt_per_H_g2;       // 1.5 (e/m) dt  [1 / (T)]
  const float* ginv;        // G^-1 table
  const float4* explicit_samples;  // (r, gamma, wdt, ln x target) or null
  int64_t n_total;          // samples in the whole batch (loss mean)
  int64_t n_valid;          // samples available from `first`
};

__device__ void make_sample(const SampleSpec& sp, int64_t idx, float* f, float* tgt,
                            float* wgt) {
  float r, gam, wdt, lnx;
  if (sp.explicit_samples) {
    const float4 v = sp.explicit_samples[idx];
    r = v.x; gam = v.y; wdt = v.z; lnx = v.w;
  } else {
    const uint64_t s = sp.first + static_cast<uint64_t>(idx);
    const uint4 w = philox10_mlp(make_uint4(static_cast<uint32_t>(s),
                                            static_cast<uint32_t>(s >> 32), 3u, 0u),
                                 sp.key0, sp.key1);
    // r uniform in [kRMin, kRMax], the trained range
    const float u = fmaf(static_cast<float>(w.x), 0x1p-32f, 0x1p-33f);
    r = fminf(fmaxf(u, kRMin), kRMax);
    const float ug = fmaf(static_cast<float>(w.y), 0x1p-32f, 0x1p-33f);
    const float uh = fmaf(static_cast<float>(w.z), 0x1p-32f, 0x1p-33f);
    gam = __expf(sp.lng_lo + sp.lng_span * ug);
    const float H = __expf(sp.lnh_lo + sp.lnh_span * uh);
    wdt = sp.wdt_per_H_g2 * H * gam * gam;
    lnx = ginv_ln(sp.ginv, r);
  }
  const float3 ff = mlp_features(r, gam, wdt);
  f[0] = ff.x; f[1] = ff.y; f[2] = ff.z; f[3] = 0.0f;
  *tgt = (lnx - mlp_prior(r)) * (1.0f / kOutScale);
  // energy weighting: (1 + x) / 1.308 (mean 1 over r uniform), so the
  // high-x part of the spectrum, which carries the emitted energy, is fitted
  // as tightly as the photon number
  *wgt = (1.0f + __expf(lnx)) * (1.0f / 1.308f);
}

// Block-wide wait for the MMA group committed to the block's mbarrier: warp
// 0 polls (bounded), the block agrees at a barrier; true if it ran out.
__device__ __forceinline__ bool train_wait(TrainTcSmem& S, uint32_t parity) {
  bool ok = true;
  if (threadIdx.x < 32) ok = tc_mbar_wait(&S.bar, parity, kTcWaitCycles);
  const bool bad = __syncthreads_or(!ok) != 0;
  tc_fence_after_sync();
  return bad;
}

// One block: 128 samples (one per thread), forward and backward on the
// tcgen05 tensor cores; writes the block's partial gradient (kNumParams
// floats) and partial loss sum.  The three products:
//   forward  z2 / 2 = [h1 | 1 1] [W2 / 2 | b2]^T   M 128, N 64, K 80 (f16)
//   dW2      = delta2^T h1                          M 128 (64 used), N 64, K 128 (BF16)
//   dh1      = delta2 W2                            M 128, N 64, K 64 (BF16)
// with accumulators in TMEM (128 columns: the forward result, then dW2 in
// columns 0..63 and dh1 in 64..127).  Numerics: h1 = f16(silu(z1)) in
// packed f16 arithmetic forward (as in the evaluator), BF16 copies of
// delta2, bf16(silu(z1)) and W2 in the gradient products, FP32 elsewhere.
// A tensor-core wait that runs out zeroes the block's partials and sets
// status bit 2.
__global__ void __launch_bounds__(kTB, 2)
    k_mlp_train_tc(MlpDev dev, SampleSpec sp, float* __restrict__ partial,
                   float* __restrict__ loss_part, unsigned long long* status) {
  extern __shared__ unsigned char raw[];
  TrainTcSmem& S = *reinterpret_cast<TrainTcSmem*>(
      (reinterpret_cast<uintptr_t>(raw) + 127) & ~static_cast<uintptr_t>(127));
  const int s = threadIdx.x, lane = s & 31, warp = s >> 5;
  // ---- set-up: the forward weight image, constant columns, mbarrier, TMEM
  for (int e = s; e < kHid * kTcK2; e += kTB) {  // forward B (unit n, k)
    const int n = e / kTcK2, k = e - n * kTcK2;
    float v = 0.0f;
    if (k < kHid) {
      v = 0.5f * __bfloat162float(dev.w2[n * kHid + k]);
    } else if (k < kHid + 2) {
      const float hb = 0.5f * dev.params[kOffB2 + n];
      const float hi = __half2float(__float2half_rn(hb));
      v = k == kHid ? hi : hb - hi;
    }
    S.u.fwd.b2[tc_off(n, k, kTcSbo2)] = tc_f16_bits(v);
  }
  for (int e = s; e < kTB * 16; e += kTB) {  // forward A columns 64..79: 1 1 0..
    const int m = e >> 4, k = kHid + (e & 15);
    S.u.fwd.a2[tc_off(m, k, kTcSbo2)] = k < kHid + 2 ? static_cast<uint16_t>(0x3C00u) : 0;
  }
  if (s < kHid) {
    S.w1b1[s] = make_float4(bf16_round(dev.params[kOffW1 + 3 * s]),
                            bf16_round(dev.params[kOffW1 + 3 * s + 1]),
                            bf16_round(dev.params[kOffW1 + 3 * s + 2]), dev.params[kOffB1 + s]);
    S.w3[s] = bf16_round(dev.params[kOffW3 + s]);
  }
  if (s == 0) {
    S.b3 = dev.params[kOffB3];
    tc_mbar_init(&S.bar);
  }
  __syncwarp();
  if (s < 32) tc_tmem_alloc(&S.tmem, 128);
  // ---- the block's samples and layer 1 (FP32, BF16 weights)
  const int64_t idx = static_cast<int64_t>(blockIdx.x) * kTB + s;
  if (idx < sp.n_valid) {
    make_sample(sp, idx, S.x[s], &S.tgt[s], &S.wgt[s]);
  } else {  // padding rows contribute nothing
    S.x[s][0] = S.x[s][1] = S.x[s][2] = 0.0f;
    S.x[s][3] = -1.0f;
    S.tgt[s] = 0.0f;
    S.wgt[s] = 0.0f;
  }
  __syncthreads();
  {
    const float f0 = S.x[s][0], f1 = S.x[s][1], f2 = S.x[s][2];
#pragma unroll 4
    for (int c = 0; c < kHid / 8; ++c) {
      float z[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int j = 8 * c + q;
        const float4 w = S.w1b1[j];
        z[q] = fmaf(w.x, f0, fmaf(w.y, f1, fmaf(w.z, f2, w.w)));
        S.z1[s][j] = z[q];
        S.h1t[tc_off(j, s, kTrSbo128)] = tc_bf16_bits(silu(z[q]));
      }
      uint4 q4;
      q4.x = silu_f16x2(z[0], z[1]);
      q4.y = silu_f16x2(z[2], z[3]);
      q4.z = silu_f16x2(z[4], z[5]);
      q4.w = silu_f16x2(z[6], z[7]);
      *reinterpret_cast<uint4*>(&S.u.fwd.a2[tc_off(s, 8 * c, kTcSbo2)]) = q4;
    }
  }
  tc_fence_proxy_async();
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  const uint32_t tmem = S.tmem;
  const uint32_t lanes = tmem + (static_cast<uint32_t>(s & ~31) << 16);
  // ---- forward layer 2 on the tensor cores
  if (s == 0) {
    const uint64_t ad = tc_desc(S.u.fwd.a2, kTcLbo, kTcSbo2);
    const uint64_t bd = tc_desc(S.u.fwd.b2, kTcLbo, kTcSbo2);
#pragma unroll
    for (int k = 0; k < kTcK2 / 16; ++k)
      tc_mma_f16(tmem, ad + k * (kTcKStep >> 4), bd + k * (kTcKStep >> 4),
                 tc_idesc(false, kTB, kHid), k > 0 ? 1u : 0u);
    tc_commit(&S.bar);
  }
  uint32_t pend_par = 0u;  // parity of the MMA group last committed
  bool bad = train_wait(S, 0u);
  if (!bad) {
    // the forward operands are dead: W2^T for the delta1 product takes
    // their place
    for (int e = s; e < kHid * kHid; e += kTB) {  // W2^T [i][j] = W2[j][i]
      const int j = e / kHid, i = e - j * kHid;
      S.u.bwd.w2t[tc_off(i, j, kTrSbo64)] = *reinterpret_cast<const uint16_t*>(dev.w2 + e);
    }
    // z2 = 2 c; output o = W3 h2 + b3 with h2 = f16(silu(z2)); loss, dL/do,
    // delta2 = dL/do W3 silu'(z2)
    float c2[kHid];
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      uint32_t v[32];
      tmem_ld_wait_32x32b_x32(lanes + 32 * half, v);
#pragma unroll
      for (int q = 0; q < 32; ++q) c2[32 * half + q] = __uint_as_float(v[q]);
    }
    float o = S.b3;
#pragma unroll
    for (int j = 0; j < kHid; j += 2) {
      const uint32_t hh = silu_half_f16x2(c2[j], c2[j + 1]);
      const float2 h2 = __half22float2(*reinterpret_cast<const __half2*>(&hh));
      o = fmaf(S.w3[j], h2.x, o);
      o = fmaf(S.w3[j + 1], h2.y, o);
    }
    const bool valid = S.x[s][3] == 0.0f;
    const float diff = o - S.tgt[s];
    const float wg = S.wgt[s];
    S.loss[s] = valid ? wg * diff * diff : 0.0f;
    const float dout = valid ? 2.0f * wg * diff / static_cast<float>(sp.n_total) : 0.0f;
    S.dout[s] = dout;
    // dL/dW3_j = sum_s dout silu(z2), dL/db2_j = sum_s dout W3_j silu'(z2):
    // per-warp sums in FP32, then over the warps
    {
      float v[kHid];
#pragma unroll
      for (int j = 0; j < kHid; ++j) v[j] = dout * silu(2.0f * c2[j]);
      warp_sum64(v, lane);
      S.wsum[warp][2 * lane] = v[0];
      S.wsum[warp][2 * lane + 1] = v[1];
#pragma unroll
      for (int j = 0; j < kHid; ++j) v[j] = dout * S.w3[j] * silu_grad(2.0f * c2[j]);
      warp_sum64(v, lane);
      S.wsum[warp][kHid + 2 * lane] = v[0];
      S.wsum[warp][kHid + 2 * lane + 1] = v[1];
    }
#pragma unroll
    for (int c = 0; c < kHid / 8; ++c) {
      uint32_t pk[4];
#pragma unroll
      for (int q = 0; q < 8; q += 2) {
        const int j = 8 * c + q;
        const float da = dout * S.w3[j] * silu_grad(2.0f * c2[j]);
        const float db = dout * S.w3[j + 1] * silu_grad(2.0f * c2[j + 1]);
        pk[q / 2] = pack_bf16x2(da, db);
        S.d2t[tc_off(j, s, kTrSbo128)] = static_cast<uint16_t>(pk[q / 2] & 0xffffu);
        S.d2t[tc_off(j + 1, s, kTrSbo128)] = static_cast<uint16_t>(pk[q / 2] >> 16);
      }
      *reinterpret_cast<uint4*>(&S.u.bwd.d2[tc_off(s, 8 * c, kTrSbo64)]) =
          make_uint4(pk[0], pk[1], pk[2], pk[3]);
    }
  }
  // ---- backward products on the tensor cores
  tc_fence_proxy_async();
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  if (!bad && s == 0) {
    const uint64_t ad = tc_desc(S.d2t, kTcLbo, kTrSbo128), bd = tc_desc(S.h1t, kTcLbo, kTrSbo128);
#pragma unroll
    for (int k = 0; k < kTB / 16; ++k)
      tc_mma_f16(tmem, ad + k * (kTcKStep >> 4), bd + k * (kTcKStep >> 4),
                 tc_idesc(true, kTB, kHid), k > 0 ? 1u : 0u);
    const uint64_t ad3 = tc_desc(S.u.bwd.d2, kTcLbo, kTrSbo64);
    const uint64_t bd3 = tc_desc(S.u.bwd.w2t, kTcLbo, kTrSbo64);
#pragma unroll
    for (int k = 0; k < kHid / 16; ++k)
      tc_mma_f16(tmem + kHid, ad3 + k * (kTcKStep >> 4), bd3 + k * (kTcKStep >> 4),
                 tc_idesc(true, kTB, kHid), k > 0 ? 1u : 0u);
    tc_commit(&S.bar);
  }
  if (!bad) {
    pend_par = 1u;
    bad = train_wait(S, 1u);
  }
  float* gp = partial + static_cast<size_t>(blockIdx.x) * kNumParams;
  if (!bad) {
    // dW2 row j = s (TMEM lanes 0..63: warps 0 and 1)
    if (s < kHid) {
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        uint32_t v[32];
        tmem_ld_wait_32x32b_x32(lanes + 32 * half, v);
        // (scalar stores: a block's partials start at a multiple of
        // kNumParams = 4481 floats, only 4-byte aligned)
#pragma unroll
        for (int q = 0; q < 32; ++q) gp[kOffW2 + s * kHid + 32 * half + q] = __uint_as_float(v[q]);
      }
    }
    // delta1 = dh1 silu'(z1), in place of z1
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      uint32_t v[32];
      tmem_ld_wait_32x32b_x32(lanes + kHid + 32 * half, v);
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const int i = 32 * half + q;
        S.z1[s][i] = __uint_as_float(v[q]) * silu_grad(S.z1[s][i]);
      }
    }
  }
  tc_fence_before_sync();
  __syncthreads();
  if (bad) {
    // tensor-core wait ran out: this block contributes nothing
    for (int p = s; p < kNumParams; p += kTB) gp[p] = 0.0f;
    if (s == 0) {
      loss_part[blockIdx.x] = 0.0f;
      atomicOr(status, 4ull);
    }
  } else {
    // per-unit sums over the block's samples (FP32)
    if (s < kHid) {
      const int j = s;
      float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, b1 = 0.0f;
      for (int r = 0; r < kTB; ++r) {
        const float d = S.z1[r][j];
        a0 = fmaf(d, S.x[r][0], a0);
        a1 = fmaf(d, S.x[r][1], a1);
        a2 = fmaf(d, S.x[r][2], a2);
        b1 += d;
      }
      gp[kOffW1 + 3 * j] = a0;
      gp[kOffW1 + 3 * j + 1] = a1;
      gp[kOffW1 + 3 * j + 2] = a2;
      gp[kOffB1 + j] = b1;
      float dw3 = 0.0f, db2 = 0.0f;
#pragma unroll
      for (int w = 0; w < kTB / 32; ++w) {
        dw3 += S.wsum[w][j];
        db2 += S.wsum[w][kHid + j];
      }
      gp[kOffW3 + j] = dw3;
      gp[kOffB2 + j] = db2;
    }
    if (s == kHid) {
      float db3 = 0.0f, ls = 0.0f;
      for (int r = 0; r < kTB; ++r) {
        db3 += S.dout[r];
        ls += S.loss[r];
      }
      gp[kOffB3] = db3;
      loss_part[blockIdx.x] = ls;
    }
  }
  // tear-down: after a timeout, wait (bounded) for the MMAs in flight
  if (bad && threadIdx.x < 32) tc_mbar_wait(&S.bar, pend_par, kTcWaitCycles);
  __syncthreads();
  tc_fence_after_sync();
  if (s < 32) tc_tmem_dealloc(tmem, 128);
}

// Sum the block partials in a fixed order; optionally Adam-update the FP32
// master parameters and refresh the BF16 copy of W2.
__global__ void k_mlp_reduce_adam(const float* __restrict__ partial, int nblocks,
                                  const float* __restrict__ loss_part, float* __restrict__ grad,
                                  float* __restrict__ params, float* __restrict__ m,
                                  float* __restrict__ v, __nv_bfloat16* __restrict__ w2,
                                  float lr, float b1t, float b2t, int apply,
                                  float* __restrict__ loss_out, float loss_scale) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p == kNumParams) {
    float ls = 0.0f;
    for (int b = 0; b < nblocks; ++b) ls += loss_part[b];
    *loss_out = ls * loss_scale;
  }
  if (p >= kNumParams) return;
  float gsum = 0.0f;
  for (int b = 0; b < nblocks; ++b) gsum += partial[static_cast<size_t>(b) * kNumParams + p];
  grad[p] = gsum;
  if (!apply) return;
  const float beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f;
  const float mm = beta1 * m[p] + (1.0f - beta1) * gsum;
  const float vv = beta2 * v[p] + (1.0f - beta2) * gsum * gsum;
  m[p] = mm;
  v[p] = vv;
  const float mh = mm / (1.0f - b1t), vh = vv / (1.0f - b2t);
  const float np = params[p] - lr * mh / (sqrtf(vh) + eps);
  params[p] = np;
  if (p >= kOffW2 && p < kOffB2) w2[p - kOffW2] = __float2bfloat16(np);
}

// The finishing kernel on the tcgen05 tensor cores (mlp_tc.cuh): tiles of
// 128 consecutive records, one per thread of a warpgroup, each warpgroup on
// its own tiles (tile (blockIdx.x * kTcGroups + g) + k * gridDim.x *
// kTcGroups).  A tile's payload (r, gamma, eps_c, ledger index) and weights
// are loaded one tile ahead.  A tensor-core wait that runs out stops the
// warpgroup and sets status bit 2.
struct FinishSrc {
  const MlpFinishArgs& a;
  unsigned long long first, stride, end;
  float4 pd, nx;  // payload of the current tile and of the next
  float w, nw;
  uint32_t fb = 0;

  __device__ FinishSrc(const MlpFinishArgs& args, unsigned long long beg)
      : a(args) {
    const unsigned long long cur = a.counters[kCursor];
    const unsigned long long cap = static_cast<unsigned long long>(a.cap);
    end = cur < cap ? cur : cap;
    const unsigned long long tile =
        static_cast<unsigned long long>(blockIdx.x) * kTcGroups + tc_group();
    first = beg + tile * kTcRows + tc_row();
    stride = static_cast<unsigned long long>(gridDim.x) * kTcGroups * kTcRows;
    load(first, nx, nw);
  }
  __device__ void load(unsigned long long row, float4& p, float& wt) const {
    // past the end: a harmless payload that books nothing (ledger index -1)
    p = row < end ? a.pend[row] : make_float4(0.5f, 1.0f, 0.0f, __int_as_float(-1));
    wt = row < end ? a.weight[row] : 0.0f;
  }
  __device__ bool has(long long k) const { return first - tc_row() + k * stride < end; }
  __device__ float3 features(long long k) {
    pd = nx;
    w = nw;
    load(first + (k + 1) * stride, nx, nw);
    return mlp_features(pd.x, pd.y, pd.z * a.wdt_per_eps);
  }
  __device__ void finish(long long k, float o) {
    const unsigned long long row = first + k * stride;
    if (row >= end) return;
    float x = __expf(o + mlp_prior(pd.x));
    // uniforms outside the trained range always take the G^-1 table
    const bool tail = pd.x < kRMin || pd.x > kRMax;
    const bool ok = x > 0.0f && x < 80.0f;  // also false for NaN
    if (tail || (a.check_output && !ok)) {
      x = __expf(ginv_ln(a.ginv, pd.x));
      ++fb;
    } else if (!ok) {
      x = 0.0f;  // no fallback requested: an invalid draw carries no energy
    }
    const float eps = x * pd.z;
    a.eps[row] = eps;
    const int li = __float_as_int(pd.w);
    // the increment rounded to float as in the table sampler's ledger sums,
    // converted without the FP64 pipe
    if (li >= 0) atomicAdd(a.led_emit + li, f32_to_f64(w * eps));
  }
};

// Resident CTAs per SM the finishing kernel is compiled for: shared memory
// holds four CTAs of two warpgroups (54 KB each), or six of one (34 KB).
#ifndef PRAD_TC_MINB
#define PRAD_TC_MINB (kTcGroups == 2 ? 4 : 6)
#endif
__global__ void __launch_bounds__(kTcThreads, PRAD_TC_MINB) k_mlp_finish_tc(const MlpFinishArgs a) {
  extern __shared__ unsigned char tc_raw[];
  TcSmem& S = tc_smem(tc_raw);
  tc_setup(S, a.mlp);
  FinishSrc src(a, a.counters[kMlpDone]);
  const bool failed = tc_run(S, src);
  const uint32_t fb = __reduce_add_sync(0xffffffffu, src.fb);
  if ((threadIdx.x & 31) == 0 && fb)
    atomicAdd(a.counters + kMlpFallback, static_cast<unsigned long long>(fb));
  __syncthreads();
  if (threadIdx.x == 0) {
    if (failed) atomicOr(a.counters + kStatus, 4ull);  // status bit 2: tensor-core wait
    __threadfence();
    const unsigned long long t = atomicAdd(a.counters + kMlpBlocks, 1ull);
    if (t == gridDim.x - 1ull) {
      a.counters[kMlpDone] = src.end;
      a.counters[kMlpBlocks] = 0ull;
    }
  }
}

// ln x for n (r, gamma, omega_c dt) triples with the finishing kernel's
// network.  A tensor-core wait that runs out sets status bit 2.
struct EvalSrc {
  const float* in;
  float* out;
  int64_t n, first, stride;
  float3 v, nx;

  __device__ EvalSrc(const float* i, float* o, int64_t count) : in(i), out(o), n(count) {
    const int64_t tile = static_cast<int64_t>(blockIdx.x) * kTcGroups + tc_group();
    first = tile * kTcRows + tc_row();
    stride = static_cast<int64_t>(gridDim.x) * kTcGroups * kTcRows;
    nx = load(first);
  }
  __device__ float3 load(int64_t i) const {
    return i < n ? make_float3(in[3 * i], in[3 * i + 1], in[3 * i + 2])
                 : make_float3(0.5f, 1.0f, 1.0f);
  }
  __device__ bool has(long long k) const { return first - tc_row() + k * stride < n; }
  __device__ float3 features(long long k) {
    v = nx;
    nx = load(first + (k + 1) * stride);
    return mlp_features(v.x, v.y, v.z);
  }
  __device__ void finish(long long k, float o) {
    const int64_t i = first + k * stride;
    if (i < n) out[i] = o + mlp_prior(v.x);
  }
};

__global__ void __launch_bounds__(kTcThreads) k_mlp_eval_tc(MlpDev dev,
                                                            const float* __restrict__ in,
                                                            float* __restrict__ out, int64_t n,
                                                            unsigned long long* status,
                                                            int withhold) {
  extern __shared__ unsigned char tc_raw[];
  TcSmem& S = tc_smem(tc_raw);
  tc_setup(S, dev, withhold != 0);
  EvalSrc src(in, out, n);
  if (tc_run(S, src) && threadIdx.x == 0) atomicOr(status, 4ull);
}

__global__ void k_ginv_eval(const float* __restrict__ tab, const float* __restrict__ r,
                            float* __restrict__ out, int64_t n) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    out[i] = ginv_ln(tab, r[i]);
}

}  // namespace

size_t mlp_train_smem_bytes() { return sizeof(TrainTcSmem) + 128; }

cudaError_t launch_mlp_train_block(const MlpDev& dev, uint32_t key0, uint32_t key1,
                                   uint64_t first, int64_t n_valid, int64_t n_total,
                                   const float4* explicit_samples, const float* ginv,
                                   float lng_lo, float lng_span, float lnh_lo,
                                   float lnh_span, float wdt_per_H_g2, float* partial,
                                   float* loss_part, int nblocks, unsigned long long* status,
                                   cudaStream_t s) {
  SampleSpec sp;
  sp.key0 = key0; sp.key1 = key1; sp.first = first;
  sp.lng_lo = lng_lo; sp.lng_span = lng_span; sp.lnh_lo = lnh_lo; sp.lnh_span = lnh_span;
  sp.wdt_per_H_g2 = wdt_per_H_g2; sp.ginv = ginv; sp.explicit_samples = explicit_samples;
  sp.n_total = n_total; sp.n_valid = n_valid;
  const int bytes = static_cast<int>(mlp_train_smem_bytes());
  cudaError_t e = cudaFuncSetAttribute(k_mlp_train_tc,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  k_mlp_train_tc<<<nblocks, kTB, bytes, s>>>(dev, sp, partial, loss_part, status);
  return cudaGetLastError();
}

cudaError_t launch_mlp_reduce_adam(const float* partial, int nblocks, const float* loss_part,
                                   float* grad, float* params, float* m, float* v,
                                   __nv_bfloat16* w2, float lr, float b1t, float b2t,
                                   int apply, float* loss_out, float loss_scale,
                                   cudaStream_t s) {
  const int threads = 256;
  const int blocks = (kNumParams + 1 + threads - 1) / threads;
  k_mlp_reduce_adam<<<blocks, threads, 0, s>>>(partial, nblocks, loss_part, grad, params, m,
                                                v, w2, lr, b1t, b2t, apply, loss_out,
                                                loss_scale);
  return cudaGetLastError();
}

// The tcgen05 kernels take more than 48 KB of dynamic shared memory: the
// attribute is set before every launch (cheap; independent of the device).
cudaError_t tc_allow_smem(const void* fn) {
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(kTcSmemBytes));
}

cudaError_t launch_mlp_eval(const MlpDev& dev, const float* in, float* out, int64_t n,
                            unsigned long long* status, int withhold, cudaStream_t s) {
  cudaError_t e = tc_allow_smem(reinterpret_cast<const void*>(k_mlp_eval_tc));
  if (e != cudaSuccess) return e;
  const int64_t tiles = (n + kTcRows - 1) / kTcRows;
  const int64_t want = (tiles + kTcGroups - 1) / kTcGroups;
  const int grid = static_cast<int>(want < 1024 ? (want > 0 ? want : 1) : 1024);
  k_mlp_eval_tc<<<grid, kTcThreads, kTcSmemBytes, s>>>(dev, in, out, n, status, withhold);
  return cudaGetLastError();
}

cudaError_t launch_mlp_finish(const MlpFinishArgs& a, int grid, cudaStream_t s) {
  cudaError_t e = tc_allow_smem(reinterpret_cast<const void*>(k_mlp_finish_tc));
  if (e != cudaSuccess) return e;
  k_mlp_finish_tc<<<grid, kTcThreads, kTcSmemBytes, s>>>(a);
  return cudaGetLastError();
}

// Resident CTAs per SM, from the kernel's registers and shared memory and
// the SM's limits (4 on GB300 with two warpgroups per CTA: shared memory);
// every resident CTA holds kTcCols of the SM's 512 TMEM columns, so the
// allocations never wait on one another.
int mlp_finish_blocks_per_sm() {
  int dev = 0, smem_sm = 0, smem_rsv = 0, regs_sm = 0, thr_sm = 0;
  cudaFuncAttributes fa;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaFuncGetAttributes(&fa, k_mlp_finish_tc) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) !=
          cudaSuccess ||
      cudaDeviceGetAttribute(&smem_rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev) !=
          cudaSuccess ||
      cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) !=
          cudaSuccess ||
      cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess)
    return 1;
  const int per_cta_smem = static_cast<int>(kTcSmemBytes + fa.sharedSizeBytes) + smem_rsv;
  int nb = smem_sm / per_cta_smem;
  // registers are allocated per warp in units of 256
  const int regs_warp = ((fa.numRegs > 0 ? fa.numRegs : 1) * 32 + 255) / 256 * 256;
  nb = min(nb, regs_sm / (regs_warp * (kTcThreads / 32)));
  nb = min(nb, thr_sm / kTcThreads);
  nb = min(nb, 512 / static_cast<int>(kTcCols));
  return nb > 0 ? nb : 1;
}

cudaError_t launch_ginv_eval(const float* tab, const float* r, float* out, int64_t n,
                             cudaStream_t s) {
  const int64_t want = (n + 255) / 256;
  const int grid = static_cast<int>(want < 4096 ? (want > 0 ? want : 1) : 4096);
  k_ginv_eval<<<grid, 256, 0, s>>>(tab, r, out, n);
  return cudaGetLastError();
}

}  // namespace prad
