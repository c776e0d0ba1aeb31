// Training and evaluation kernels of the learned inverse-CDF sampler
// (mlp_device.cuh): sample generation with the device G^-1 table, a fused
// forward + backward pass per block of 128 samples (m16n8k16 MMAs for the
// 64 x 64 layer: f16 forward, BF16 gradient products), per-block partial
// gradients, and a deterministic reduction + Adam update; the evaluators
// (the learned sampler's finishing kernel and prad_mlp_eval) run the
// network on the tcgen05 tensor cores (mlp_tc.cuh).
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

constexpr int kTB = 128;  // samples per block
constexpr int kTThreads = 256;
constexpr int kLdT = kTB + 8;  // transposed [unit][sample] rows, bf16

struct TrainSmem {
  MlpSmem net;
  __nv_bfloat16 w2t[kHid * kW2Ld];    // W2 transposed [i][j]
  float x[kTB][4];                    // features
  float tgt[kTB];                     // target (ln x - prior) / kOutScale
  float wgt[kTB];                     // loss weight
  float dout[kTB];                    // dL/do per sample
  float loss[kTB];
  float z1[kTB][kHid];
  float z2[kTB][kHid];                // later: delta1
  __nv_bfloat16 h1t[kHid * kLdT];     // h1 transposed [i][s]
  __nv_bfloat16 d2[kTB * kW2Ld];      // delta2 [s][j]
  __nv_bfloat16 d2t[kHid * kLdT];     // delta2 transposed [j][s]
};

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

// One block: 128 samples, forward + backward; writes the block's partial
// gradient (kNumParams floats) and partial loss sum.
__global__ void __launch_bounds__(kTThreads)
    k_mlp_train_block(MlpDev dev, SampleSpec sp, float* __restrict__ partial,
                      float* __restrict__ loss_part) {
  extern __shared__ __align__(16) unsigned char raw[];
  TrainSmem& S = *reinterpret_cast<TrainSmem*>(raw);
  mlp_load_smem(S.net, dev);
  for (int e = threadIdx.x; e < kHid * kHid; e += blockDim.x) {
    const int j = e / kHid, i = e - j * kHid;
    S.w2t[i * kW2Ld + j] = dev.w2[e];
  }
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kTB;
  if (threadIdx.x < kTB) {
    const int64_t idx = base + threadIdx.x;
    if (idx < sp.n_valid) {
      make_sample(sp, idx, S.x[threadIdx.x], &S.tgt[threadIdx.x], &S.wgt[threadIdx.x]);
    } else {  // padding rows contribute nothing
      S.x[threadIdx.x][0] = S.x[threadIdx.x][1] = S.x[threadIdx.x][2] = 0.0f;
      S.x[threadIdx.x][3] = -1.0f;  // marker
      S.tgt[threadIdx.x] = 0.0f;
      S.wgt[threadIdx.x] = 0.0f;
    }
  }
  __syncthreads();
  // layer 1 (FP32, BF16 weights): z1 and bf16(silu(z1)) transposed
  for (int e = threadIdx.x; e < kTB * kHid; e += blockDim.x) {
    const int s = e / kHid, j = e - s * kHid;
    const float4 w = S.net.w1b1[j];
    const float z = fmaf(w.x, S.x[s][0], fmaf(w.y, S.x[s][1], fmaf(w.z, S.x[s][2], w.w)));
    S.z1[s][j] = z;
    S.h1t[j * kLdT + s] = __float2bfloat16(silu(z));
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  // layer 2 forward, warp w: samples 16w .. 16w + 15
  {
    const int s0 = 16 * warp;
    // h1 = f16(silu(z1)) in packed f16 arithmetic, as in the evaluator
    uint32_t a[4][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = 16 * q + 2 * t;
      a[q][0] = silu_f16x2(S.z1[s0 + g][j], S.z1[s0 + g][j + 1]);
      a[q][1] = silu_f16x2(S.z1[s0 + g + 8][j], S.z1[s0 + g + 8][j + 1]);
      a[q][2] = silu_f16x2(S.z1[s0 + g][j + 8], S.z1[s0 + g][j + 9]);
      a[q][3] = silu_f16x2(S.z1[s0 + g + 8][j + 8], S.z1[s0 + g + 8][j + 9]);
    }
    // the network image holds W2 / 2 and b2 / 2 (exact): z2 = 2 c
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const int j0 = 8 * nt + 2 * t;
      float c[4] = {S.net.b2h[j0], S.net.b2h[j0 + 1], S.net.b2h[j0], S.net.b2h[j0 + 1]};
      const __half* wrow = S.net.w2h + (8 * nt + g) * kW2Ld + 2 * t;
#pragma unroll
      for (int q = 0; q < 4; ++q)
        mma_f16_16816(c, a[q][0], a[q][1], a[q][2], a[q][3],
                      *reinterpret_cast<const uint32_t*>(wrow + 16 * q),
                      *reinterpret_cast<const uint32_t*>(wrow + 16 * q + 8));
      S.z2[s0 + g][j0] = 2.0f * c[0];
      S.z2[s0 + g][j0 + 1] = 2.0f * c[1];
      S.z2[s0 + g + 8][j0] = 2.0f * c[2];
      S.z2[s0 + g + 8][j0 + 1] = 2.0f * c[3];
    }
  }
  __syncthreads();
  // output (h2 = f16(silu(z2)) as in the evaluator), loss and dL/do per sample
  if (threadIdx.x < kTB) {
    const int s = threadIdx.x;
    float o = S.net.b3;
    for (int j = 0; j < kHid; j += 2) {
      const uint32_t hh = silu_f16x2(S.z2[s][j], S.z2[s][j + 1]);
      const float2 h2 = __half22float2(*reinterpret_cast<const __half2*>(&hh));
      o = fmaf(S.net.w3[j], h2.x, o);
      o = fmaf(S.net.w3[j + 1], h2.y, o);
    }
    const bool valid = S.x[s][3] == 0.0f;
    const float diff = o - S.tgt[s];
    const float wgt = S.wgt[s];
    S.loss[s] = valid ? wgt * diff * diff : 0.0f;
    S.dout[s] = valid ? 2.0f * wgt * diff / static_cast<float>(sp.n_total) : 0.0f;
  }
  __syncthreads();
  // delta2 = dout W3 silu'(z2): BF16 copies for the two tensor-core products
  for (int e = threadIdx.x; e < kTB * kHid; e += blockDim.x) {
    const int s = e / kHid, j = e - s * kHid;
    const __nv_bfloat16 d =
        __float2bfloat16(S.dout[s] * S.net.w3[j] * silu_grad(S.z2[s][j]));
    S.d2[s * kW2Ld + j] = d;
    S.d2t[j * kLdT + s] = d;
  }
  __syncthreads();
  float* gp = partial + static_cast<size_t>(blockIdx.x) * kNumParams;
  // per-unit sums: dW3, db2 (FP32 from z2), loss
  if (threadIdx.x < kHid) {
    const int j = threadIdx.x;
    float dw3 = 0.0f, db2 = 0.0f;
    for (int s = 0; s < kTB; ++s) {
      dw3 = fmaf(S.dout[s], silu(S.z2[s][j]), dw3);
      db2 = fmaf(S.dout[s] * S.net.w3[j], silu_grad(S.z2[s][j]), db2);
    }
    gp[kOffW3 + j] = dw3;
    gp[kOffB2 + j] = db2;
  }
  if (threadIdx.x == kHid) {
    float db3 = 0.0f, ls = 0.0f;
    for (int s = 0; s < kTB; ++s) {
      db3 += S.dout[s];
      ls += S.loss[s];
    }
    gp[kOffB3] = db3;
    loss_part[blockIdx.x] = ls;
  }
  __syncthreads();  // z2 is overwritten by delta1 below
  // delta1 = (delta2 W2) * silu'(z1), warp w: samples 16w .. 16w + 15
  {
    const int s0 = 16 * warp;
    uint32_t a[4][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const __nv_bfloat16* r0 = S.d2 + (s0 + g) * kW2Ld + 16 * q + 2 * t;
      const __nv_bfloat16* r1 = S.d2 + (s0 + g + 8) * kW2Ld + 16 * q + 2 * t;
      a[q][0] = *reinterpret_cast<const uint32_t*>(r0);
      a[q][1] = *reinterpret_cast<const uint32_t*>(r1);
      a[q][2] = *reinterpret_cast<const uint32_t*>(r0 + 8);
      a[q][3] = *reinterpret_cast<const uint32_t*>(r1 + 8);
    }
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      const __nv_bfloat16* brow = S.w2t + (8 * nt + g) * kW2Ld + 2 * t;
#pragma unroll
      for (int q = 0; q < 4; ++q)
        mma_bf16_16816(c, a[q][0], a[q][1], a[q][2], a[q][3],
                       *reinterpret_cast<const uint32_t*>(brow + 16 * q),
                       *reinterpret_cast<const uint32_t*>(brow + 16 * q + 8));
      const int i0 = 8 * nt + 2 * t;
      S.z2[s0 + g][i0] = c[0] * silu_grad(S.z1[s0 + g][i0]);
      S.z2[s0 + g][i0 + 1] = c[1] * silu_grad(S.z1[s0 + g][i0 + 1]);
      S.z2[s0 + g + 8][i0] = c[2] * silu_grad(S.z1[s0 + g + 8][i0]);
      S.z2[s0 + g + 8][i0 + 1] = c[3] * silu_grad(S.z1[s0 + g + 8][i0 + 1]);
    }
  }
  // dW2 = delta2^T h1 over the block's 128 samples: output [j][i];
  // warp w: rows j in 16 (w % 4) .., columns i in 32 (w / 4) .. (4 tiles)
  {
    const int mt = warp & 3, nb = (warp >> 2) * 4;
    float c[4][4] = {};
#pragma unroll
    for (int kt = 0; kt < kTB / 16; ++kt) {
      const __nv_bfloat16* ar0 = S.d2t + (16 * mt + g) * kLdT + 16 * kt + 2 * t;
      const __nv_bfloat16* ar1 = S.d2t + (16 * mt + g + 8) * kLdT + 16 * kt + 2 * t;
      const uint32_t a0 = *reinterpret_cast<const uint32_t*>(ar0);
      const uint32_t a1 = *reinterpret_cast<const uint32_t*>(ar1);
      const uint32_t a2 = *reinterpret_cast<const uint32_t*>(ar0 + 8);
      const uint32_t a3 = *reinterpret_cast<const uint32_t*>(ar1 + 8);
#pragma unroll
      for (int n = 0; n < 4; ++n) {
        const __nv_bfloat16* br = S.h1t + (8 * (nb + n) + g) * kLdT + 16 * kt + 2 * t;
        mma_bf16_16816(c[n], a0, a1, a2, a3, *reinterpret_cast<const uint32_t*>(br),
                       *reinterpret_cast<const uint32_t*>(br + 8));
      }
    }
#pragma unroll
    for (int n = 0; n < 4; ++n) {
      const int j = 16 * mt + g, i = 8 * (nb + n) + 2 * t;
      gp[kOffW2 + j * kHid + i] = c[n][0];
      gp[kOffW2 + j * kHid + i + 1] = c[n][1];
      gp[kOffW2 + (j + 8) * kHid + i] = c[n][2];
      gp[kOffW2 + (j + 8) * kHid + i + 1] = c[n][3];
    }
  }
  __syncthreads();
  // dW1, db1 from delta1 (held in z2)
  if (threadIdx.x < kHid) {
    const int j = threadIdx.x;
    float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, b = 0.0f;
    for (int s = 0; s < kTB; ++s) {
      const float d = S.z2[s][j];
      a0 = fmaf(d, S.x[s][0], a0);
      a1 = fmaf(d, S.x[s][1], a1);
      a2 = fmaf(d, S.x[s][2], a2);
      b += d;
    }
    gp[kOffW1 + 3 * j] = a0;
    gp[kOffW1 + 3 * j + 1] = a1;
    gp[kOffW1 + 3 * j + 2] = a2;
    gp[kOffB1 + j] = b;
  }
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

size_t mlp_train_smem_bytes() { return sizeof(TrainSmem); }

cudaError_t launch_mlp_train_block(const MlpDev& dev, uint32_t key0, uint32_t key1,
                                   uint64_t first, int64_t n_valid, int64_t n_total,
                                   const float4* explicit_samples, const float* ginv,
                                   float lng_lo, float lng_span, float lnh_lo,
                                   float lnh_span, float wdt_per_H_g2, float* partial,
                                   float* loss_part, int nblocks, cudaStream_t s) {
  SampleSpec sp;
  sp.key0 = key0; sp.key1 = key1; sp.first = first;
  sp.lng_lo = lng_lo; sp.lng_span = lng_span; sp.lnh_lo = lnh_lo; sp.lnh_span = lnh_span;
  sp.wdt_per_H_g2 = wdt_per_H_g2; sp.ginv = ginv; sp.explicit_samples = explicit_samples;
  sp.n_total = n_total; sp.n_valid = n_valid;
  const int bytes = static_cast<int>(sizeof(TrainSmem));
  cudaError_t e = cudaFuncSetAttribute(k_mlp_train_block,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  k_mlp_train_block<<<nblocks, kTThreads, bytes, s>>>(dev, sp, partial, loss_part);
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
