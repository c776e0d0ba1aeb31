// Learned-sampler network on the 5th-generation tensor cores (tcgen05):
// 128-row tiles, one row per thread of a 128-thread CTA.  Operands are
// staged in shared memory in the canonical K-major layout without swizzle
// (core matrices of 8 rows x 16 bytes; LBO = 128 B between core matrices
// along K, SBO between 8-row groups), accumulators live in tensor memory
// (TMEM lane = row, one 32-bit column per output unit), one thread issues
// the MMAs and an mbarrier signals their completion.  Per tile:
//   layer 1: A1 = [f0h f1h f2h f0l f1l f2l 1 1 0..] (128 x 16, BF16)
//            B1 = halved W1 | split b1 (64 x 16, BF16)      -> D = z1 / 2
//   layer 2: A2 = [h1 | 1 1 0..] (128 x 80, f16)
//            B2 = halved W2 | split b2 (64 x 80, f16)       -> D = z2 / 2
//   layer 3: A3 = h2 (A2's first 64 columns, K = 64, f16)
//            B3 = W3 in row 0 (16 x 64, f16)                -> D[:, 0] = o - b3
// with h = f16(SiLU) in packed f16 arithmetic between the layers (the
// halved images make the accumulators hold z / 2, the argument of SiLU's
// tanh form; halving is exact), the numerics of mlp_device.cuh; features
// and biases enter as sums of two parts (BF16 or f16 high part + rounded
// remainder), so z agrees with the FP32 form to ~1e-6, and the BF16 weights
// are exact in f16.  A CTA runs kTcGroups warpgroups, each on its own tiles;
// a tile's three accumulators share the group's 64 TMEM columns, each read
// out before the group's next MMA is issued.
//
// Every wait on the tensor cores is bounded.  A wait that runs out marks
// the thread bad; the block agrees on it at its next barrier and stops.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstddef>

#include "mlp_device.cuh"

namespace prad {

// ---- PTX wrappers --------------------------------------------------------
__device__ __forceinline__ uint32_t tc_smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void tc_mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem_addr(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Tests the phase of the given parity; a thread whose phase is not yet
// complete sleeps until it completes or about 0.1 ms have passed.
__device__ __forceinline__ bool tc_mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(tc_smem_addr(bar)), "r"(parity), "r"(100000u)
      : "memory");
  return done != 0;
}

// Waits until the mbarrier phase of the given parity has completed, for at
// most max_cycles SM clocks; false if it has not.
__device__ __forceinline__ bool tc_mbar_wait(uint64_t* bar, uint32_t parity,
                                             long long max_cycles) {
  if (tc_mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!tc_mbar_try_wait(bar, parity))
    if (clock64() - t0 > max_cycles) return false;
  return true;
}

// Warp-collective TMEM allocation of ncols columns (a power of two >= 32);
// the base address is written to *slot.
__device__ __forceinline__ void tc_tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   tc_smem_addr(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tc_tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

// D[tmem] = A[smem] * B[smem]^T (+ D if accumulate), A and B K-major.
__device__ __forceinline__ void tc_mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                           uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// One arrival on the mbarrier once every MMA this thread has issued is
// complete.
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          tc_smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// generic-proxy shared-memory writes -> later reads by the tensor cores
__device__ __forceinline__ void tc_fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// tcgen05.ld wrappers (generated: long operand lists).  Load and wait in one
// statement: the outputs are complete when it returns, so no separate wait
// has to carry them as operands.
__device__ __forceinline__ void tmem_ld_wait_32x32b_x32(uint32_t taddr, uint32_t* v) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n\t"
               "tcgen05.wait::ld.sync.aligned;"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
               : "r"(taddr)
               : "memory");
}

__device__ __forceinline__ void tmem_ld_wait_32x32b_x1(uint32_t taddr, uint32_t* v) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];\n\t"
               "tcgen05.wait::ld.sync.aligned;"
               : "=r"(v[0])
               : "r"(taddr)
               : "memory");
}

// Shared-memory matrix descriptor: canonical K-major layout, no swizzle,
// byte strides lbo (along K) and sbo (between 8-row groups).
__device__ __forceinline__ uint64_t tc_desc(const void* base, uint32_t lbo, uint32_t sbo) {
  uint64_t d = static_cast<uint64_t>((tc_smem_addr(base) & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16;
  d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32;
  d |= static_cast<uint64_t>(1) << 46;  // descriptor version of the tcgen05 MMAs
  return d;                             // base offset 0, relative LBO, no swizzle
}

// Instruction descriptor of kind::f16: FP32 accumulator, A and B K-major,
// both BF16 or both f16.
__host__ __device__ constexpr uint32_t tc_idesc(bool bf16, int m, int n) {
  return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) |
         (static_cast<uint32_t>(n >> 3) << 17) | (static_cast<uint32_t>(m >> 4) << 24);
}

// ---- 128-row tiles, one warpgroup per tile ----------------------------------
constexpr int kTcRows = 128;          // rows per tile = threads per warpgroup
// Warpgroups per CTA.  Each runs its own sequence of tiles (its A tile, its
// mbarrier, its 64 TMEM columns) and the weight images are shared by the
// CTA, so two warpgroups take 54 KB of shared memory where two one-warpgroup
// CTAs take 68 KB: eight tiles in flight per SM instead of six.  (A tile's
// three MMA rounds, each waited for, set the pace: with the arithmetic taken
// out the kernel still needs 72% of its time.)
#ifndef PRAD_TC_GROUPS
#define PRAD_TC_GROUPS 2
#endif
constexpr int kTcGroups = PRAD_TC_GROUPS;
static_assert(kTcGroups == 1 || kTcGroups == 2, "one or two warpgroups");
constexpr int kTcThreads = kTcRows * kTcGroups;  // threads per CTA
constexpr int kTcK2 = 80;             // layer-2 K: 64 units, 2 bias columns, zeros
constexpr uint32_t kTcCols = 64 * kTcGroups;     // TMEM columns per CTA: 64 per warpgroup
constexpr uint32_t kTcLbo = 128;      // core matrix: 8 rows x 16 B
constexpr uint32_t kTcSbo1 = 2 * 128;            // K = 16
constexpr uint32_t kTcSbo2 = (kTcK2 / 8) * 128;  // K = 80
constexpr uint32_t kTcSbo3 = (kHid / 8) * 128;   // K = 64
constexpr uint32_t kTcKStep = 2 * 128;           // bytes per K = 16 step
constexpr long long kTcWaitCycles = 1ll << 31;   // ~1 s at the SM clock

// A warpgroup's A1 tile lives in the first 16 columns of its A2 tile (same
// canonical layout, SBO of K = 80): layer 1 has read it before the
// activations overwrite those columns, and layer 3 has read h2 before the
// next tile's features are written there.
struct alignas(128) TcSmem {
  uint16_t a2[kTcGroups][kTcRows * kTcK2];
  uint16_t b1[kHid * 16];
  uint16_t b2[kHid * kTcK2];
  uint16_t b3[16 * kHid];
  uint64_t bar[kTcGroups];
  uint32_t tmem;
  float b3s;
  uint32_t withhold;  // self-test: commit no MMA group (every wait runs out)
};
static_assert(offsetof(TcSmem, a2) % 128 == 0 &&
                  (kTcRows * kTcK2 * 2) % 128 == 0 && offsetof(TcSmem, b1) % 128 == 0 &&
                  offsetof(TcSmem, b2) % 128 == 0 && offsetof(TcSmem, b3) % 128 == 0 &&
                  offsetof(TcSmem, bar) % 8 == 0,
              "operand and mbarrier alignment");
constexpr size_t kTcSmemBytes = sizeof(TcSmem) + 128;  // + alignment slack

// element offset of (row, k) in a canonical K-major tile with sbo bytes per
// 8-row group (16-bit elements)
__host__ __device__ constexpr int tc_off(int row, int k, uint32_t sbo) {
  return (row >> 3) * static_cast<int>(sbo / 2) + (k >> 3) * 64 + (row & 7) * 8 + (k & 7);
}
static_assert(tc_off(kHid - 1, 15, kTcSbo1) < kHid * 16 &&
                  tc_off(kTcRows - 1, kTcK2 - 1, kTcSbo2) < kTcRows * kTcK2 &&
                  tc_off(kHid - 1, kTcK2 - 1, kTcSbo2) < kHid * kTcK2 &&
                  tc_off(15, kHid - 1, kTcSbo3) < 16 * kHid,
              "canonical layouts stay inside their arrays");

__device__ __forceinline__ uint16_t tc_bf16_bits(float v) {
  const __nv_bfloat16 b = __float2bfloat16(v);
  return *reinterpret_cast<const uint16_t*>(&b);
}
__device__ __forceinline__ uint16_t tc_f16_bits(float v) {
  const __half h = __float2half_rn(v);
  return *reinterpret_cast<const uint16_t*>(&h);
}

// The CTA's TcSmem inside its dynamic shared memory (aligned to 128 B).
__device__ __forceinline__ TcSmem& tc_smem(unsigned char* raw) {
  const uintptr_t p = (reinterpret_cast<uintptr_t>(raw) + 127) & ~static_cast<uintptr_t>(127);
  return *reinterpret_cast<TcSmem*>(p);
}

// The thread's warpgroup and its row in the group's tiles.
__device__ __forceinline__ int tc_group() { return static_cast<int>(threadIdx.x) / kTcRows; }
__device__ __forceinline__ int tc_row() { return static_cast<int>(threadIdx.x) % kTcRows; }

// Barrier of warpgroup g alone (named barrier 1 + g, its 128 threads); true
// if any of them passes bad.
__device__ __forceinline__ bool tc_group_sync_or(int g, bool bad) {
  uint32_t any;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.or.pred q, %2, %3, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(any)
      : "r"(bad ? 1u : 0u), "r"(1 + g), "r"(kTcRows)
      : "memory");
  return any != 0;
}

// Block-collective set-up: the weight images, the constant columns of the
// A tiles, the mbarriers and the TMEM allocation (warp 0).  withhold: the
// self-test of the bounded waits, in which no MMA completion is signalled.
__device__ __forceinline__ void tc_setup(TcSmem& S, const MlpDev& d, bool withhold = false) {
  const int nt = blockDim.x;
  for (int e = threadIdx.x; e < kHid * 16; e += nt) {  // B1 (unit n, k)
    const int n = e >> 4, k = e & 15;
    const float b1 = d.params[kOffB1 + n];
    const float b1h = bf16_round(b1);
    float v = 0.0f;
    if (k < 3) v = bf16_round(d.params[kOffW1 + 3 * n + k]);
    else if (k < 6) v = bf16_round(d.params[kOffW1 + 3 * n + k - 3]);
    else if (k == 6) v = b1h;
    else if (k == 7) v = bf16_round(b1 - b1h);
    S.b1[tc_off(n, k, kTcSbo1)] = tc_bf16_bits(0.5f * v);  // halved: exact
  }
  for (int e = threadIdx.x; e < kHid * kTcK2; e += nt) {  // B2 (unit n, k)
    const int n = e / kTcK2, k = e - n * kTcK2;
    float v = 0.0f;
    if (k < kHid) {
      v = 0.5f * __bfloat162float(d.w2[n * kHid + k]);
    } else if (k < kHid + 2) {
      const float hb = 0.5f * d.params[kOffB2 + n];
      const float hi = __half2float(__float2half_rn(hb));
      v = k == kHid ? hi : hb - hi;
    }
    S.b2[tc_off(n, k, kTcSbo2)] = tc_f16_bits(v);
  }
  for (int e = threadIdx.x; e < 16 * kHid; e += nt) {  // B3: W3 in row 0
    const int n = e / kHid, k = e - n * kHid;
    S.b3[tc_off(n, k, kTcSbo3)] = tc_f16_bits(n == 0 ? bf16_round(d.params[kOffW3 + k]) : 0.0f);
  }
  for (int e = threadIdx.x; e < kTcGroups * kTcRows * 16; e += nt) {  // A2 cols 64..79: 1 1 0..
    const int g = e / (kTcRows * 16), r = e - g * kTcRows * 16;
    const int m = r >> 4, k = kHid + (r & 15);
    S.a2[g][tc_off(m, k, kTcSbo2)] = k < kHid + 2 ? static_cast<uint16_t>(0x3C00u) : 0;
  }
  if (threadIdx.x == 0) {
    S.b3s = d.params[kOffB3];
    S.withhold = withhold ? 1u : 0u;
    for (int g = 0; g < kTcGroups; ++g) tc_mbar_init(&S.bar[g]);
  }
  __syncwarp();
  if (threadIdx.x < 32) tc_tmem_alloc(&S.tmem, kTcCols);
  tc_fence_proxy_async();
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
}

// Warpgroup barrier that orders this thread's shared-memory writes and TMEM
// reads before the tensor-core work the next MMA issues; true if any thread
// of the group is bad.
__device__ __forceinline__ bool tc_sync_bad(int g, bool bad) {
  tc_fence_proxy_async();
  tc_fence_before_sync();
  const bool any = tc_group_sync_or(g, bad);
  tc_fence_after_sync();
  return any;
}

// Writes this thread's A1 row [f0h f1h f2h f0l f1l f2l 1 1 0 0 0 0 0 0 0 0]
// into columns 0..15 of its group's A2 tile.
__device__ __forceinline__ void tc_put_a1(uint16_t* a2, int row, float3 f) {
  const float h0 = bf16_round(f.x), h1 = bf16_round(f.y), h2 = bf16_round(f.z);
  uint4 q;
  q.x = pack_bf16x2(h0, h1);
  q.y = pack_bf16x2(h2, f.x - h0);
  q.z = pack_bf16x2(f.y - h1, f.z - h2);
  q.w = pack_bf16x2(1.0f, 1.0f);
  *reinterpret_cast<uint4*>(&a2[tc_off(row, 0, kTcSbo2)]) = q;
  *reinterpret_cast<uint4*>(&a2[tc_off(row, 8, kTcSbo2)]) = make_uint4(0u, 0u, 0u, 0u);
}

// Reads this thread's 64 accumulator columns z (= z_true / 2) and writes
// f16(SiLU(2 z)) into A2 columns 0..63.
// (two halves of 32 columns: 32 accumulator registers live at a time)
__device__ __forceinline__ void tc_silu_to_a2(uint16_t* a2, int row, uint32_t taddr) {
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    uint32_t z[32];
    tmem_ld_wait_32x32b_x32(taddr + 32 * half, z);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      uint4 q;
      q.x = silu_half_f16x2(__uint_as_float(z[8 * c + 0]), __uint_as_float(z[8 * c + 1]));
      q.y = silu_half_f16x2(__uint_as_float(z[8 * c + 2]), __uint_as_float(z[8 * c + 3]));
      q.z = silu_half_f16x2(__uint_as_float(z[8 * c + 4]), __uint_as_float(z[8 * c + 5]));
      q.w = silu_half_f16x2(__uint_as_float(z[8 * c + 6]), __uint_as_float(z[8 * c + 7]));
      *reinterpret_cast<uint4*>(&a2[tc_off(row, 32 * half + 8 * c, kTcSbo2)]) = q;
    }
  }
}

// MMA groups of one layer for warpgroup g (one thread), committed to the
// group's mbarrier.  Layer 1: D = A1 B1^T (BF16, K = 16, A1 = A2[:, 0..15]);
// layer 2: D = A2 B2^T (f16, K = 80); layer 3: D[:, 0..15] = A2[:, 0..63]
// B3^T (f16, K = 64).  D: the group's 64 TMEM columns.
__device__ __forceinline__ void tc_issue(TcSmem& S, int g, int layer) {
  const uint32_t d = S.tmem + static_cast<uint32_t>(g) * kHid;
  if (layer == 1) {
    tc_mma_f16(d, tc_desc(S.a2[g], kTcLbo, kTcSbo2), tc_desc(S.b1, kTcLbo, kTcSbo1),
               tc_idesc(true, kTcRows, kHid), 0u);
  } else if (layer == 2) {
    const uint64_t ad = tc_desc(S.a2[g], kTcLbo, kTcSbo2), bd = tc_desc(S.b2, kTcLbo, kTcSbo2);
#pragma unroll
    for (int k = 0; k < kTcK2 / 16; ++k)
      tc_mma_f16(d, ad + k * (kTcKStep >> 4), bd + k * (kTcKStep >> 4),
                 tc_idesc(false, kTcRows, kHid), k > 0 ? 1u : 0u);
  } else {
    const uint64_t ad = tc_desc(S.a2[g], kTcLbo, kTcSbo2), bd = tc_desc(S.b3, kTcLbo, kTcSbo3);
#pragma unroll
    for (int k = 0; k < kHid / 16; ++k)
      tc_mma_f16(d, ad + k * (kTcKStep >> 4), bd + k * (kTcKStep >> 4),
                 tc_idesc(false, kTcRows, 16), k > 0 ? 1u : 0u);
  }
  if (!S.withhold) tc_commit(&S.bar[g]);
}

// Per-thread bookkeeping of the MMA group in flight on its warpgroup's
// mbarrier: the parity of the next phase, and whether a committed group has
// not been seen complete (with the parity it completes).
struct TcState {
  uint32_t phase = 0;
  uint32_t pend_par = 0;
  bool pend = false;
  bool bad = false;  // a wait of the group ran out
};

__device__ __forceinline__ void tc_note_issue(TcState& t) {
  t.pend = true;
  t.pend_par = t.phase;
}

// Waits for warpgroup g's last committed MMA group; marks every thread of
// the group bad if the wait runs out.  Group-collective: its warp 0 polls
// the mbarrier and its other warps wait at the group barrier, where they
// take no issue slots.
__device__ __forceinline__ void tc_wait(TcSmem& S, TcState& t, int g) {
  bool ok = true;
  if (tc_row() < 32) ok = tc_mbar_wait(&S.bar[g], t.phase, kTcWaitCycles);
  if (!tc_group_sync_or(g, !ok)) t.pend = false;
  else t.bad = true;
  t.phase ^= 1u;
  tc_fence_after_sync();
}

// The network over a sequence of 128-row tiles k = 0, 1, 2, ... of the
// thread's warpgroup (one row per thread).  Src supplies, uniformly over
// the group, whether tile k exists (has(k)), this thread's features of tile
// k (features(k): called once per tile, in order of k), and takes
// kOutScale * o of the thread's row (finish(k, o): not called for a tile
// whose waits ran out).  Block-collective (every warpgroup of the CTA runs
// its own tiles).  Returns true if a tensor-core wait ran out in any thread
// of the CTA (its warpgroup then stopped early).
template <class Src>
__device__ __forceinline__ bool tc_run(TcSmem& S, Src& src) {
  const int g = tc_group(), row = tc_row();
  // the warp's TMEM lanes (warp w of a warpgroup reads lanes 32w..32w+31),
  // the group's columns
  const uint32_t lanes = S.tmem + (static_cast<uint32_t>(row & ~31) << 16) +
                         static_cast<uint32_t>(g) * kHid;
  uint16_t* a2 = S.a2[g];
  TcState t;
  bool live = src.has(0);
  bool stop = false;
  if (live) tc_put_a1(a2, row, src.features(0));
  tc_sync_bad(g, false);
  if (live) {
    if (row == 0) tc_issue(S, g, 1);
    tc_note_issue(t);
  }
  for (long long k = 0; live && !stop; ++k) {
    // layers 2 and 3: SiLU of the accumulators, then the next layer
#pragma unroll
    for (int layer = 2; layer <= 3; ++layer) {
      if (stop) continue;
      tc_wait(S, t, g);
      tc_silu_to_a2(a2, row, lanes);
      if (tc_sync_bad(g, t.bad)) {
        stop = true;
        continue;
      }
      if (row == 0) tc_issue(S, g, layer);
      tc_note_issue(t);
    }
    if (stop) break;
    // output, then the next tile
    tc_wait(S, t, g);
    uint32_t o[1];
    tmem_ld_wait_32x32b_x1(lanes, o);
    if (!t.bad) src.finish(k, kOutScale * (__uint_as_float(o[0]) + S.b3s));
    const bool next = src.has(k + 1);
    if (next) tc_put_a1(a2, row, src.features(k + 1));
    if (tc_sync_bad(g, t.bad)) {
      stop = true;
      break;
    }
    if (next) {
      if (row == 0) tc_issue(S, g, 1);
      tc_note_issue(t);
    }
    live = next;
  }
  // tear-down: agree on a timeout; if there was one, wait (bounded) for
  // the group still in flight before the TMEM is released
  const bool any_bad = __syncthreads_or(t.bad) != 0;
  if (any_bad && t.pend) tc_mbar_wait(&S.bar[g], t.pend_par, kTcWaitCycles);
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  if (threadIdx.x < 32) tc_tmem_dealloc(S.tmem, kTcCols);
  return any_bad;
}

}  // namespace prad
