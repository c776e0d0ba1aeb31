// Deterministic two-pass Kahan-compensated FP64 reduction of the two
// per-particle ledgers (emitted synchrotron energy and Landau-Lifshitz loss),
// the global sums compared in Fig. 3 of arXiv:1409.5574.
//
// Pass 1: block b owns the fixed chunk [b*chunk, (b+1)*chunk); each thread
// keeps a Kahan (sum, compensation) pair over a fixed strided subset, then
// the block merges the pairs in a fixed tree with TwoSum.  Pass 2: one block
// merges the per-block pairs the same way.  The mapping of elements to
// threads and the merge order never depend on timing, so results are
// bit-reproducible for a given n and block count.
#include <cuda_runtime.h>
#include <stdint.h>

#include "prad_internal.h"

namespace prad {

struct KSum {
  double s, c;  // value = s + c
};

__device__ __forceinline__ void kahan_add(KSum& k, double v) {
  const double y = v - k.c;
  const double t = k.s + y;
  k.c = (t - k.s) - y;
  k.s = t;
}

// TwoSum merge of two compensated sums (Knuth): exact error of s1 + s2 is
// carried into the compensation.
__device__ __forceinline__ KSum merge(KSum a, KSum b) {
  const double s = a.s + b.s;
  const double bb = s - a.s;
  const double err = (a.s - (s - bb)) + (b.s - bb);
  KSum r;
  r.s = s;
  r.c = a.c + b.c - err;  // kahan convention: value = s - c
  return r;
}

constexpr int kRedThreads = 256;

__device__ void block_merge(KSum& ka, KSum& kb, KSum (*sh)[kRedThreads]) {
  sh[0][threadIdx.x] = ka;
  sh[1][threadIdx.x] = kb;
  __syncthreads();
  for (int off = kRedThreads / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) {
      sh[0][threadIdx.x] = merge(sh[0][threadIdx.x], sh[0][threadIdx.x + off]);
      sh[1][threadIdx.x] = merge(sh[1][threadIdx.x], sh[1][threadIdx.x + off]);
    }
    __syncthreads();
  }
  ka = sh[0][0];
  kb = sh[1][0];
}

__global__ void __launch_bounds__(kRedThreads)
    k_ledger_pass1(const double* __restrict__ a, const double* __restrict__ b,
                   int64_t n, double* __restrict__ partials) {
  __shared__ KSum sh[2][kRedThreads];
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t lo = static_cast<int64_t>(blockIdx.x) * chunk;
  const int64_t hi = lo + chunk < n ? lo + chunk : n;
  KSum ka{0.0, 0.0}, kb{0.0, 0.0};
  for (int64_t i = lo + threadIdx.x; i < hi; i += kRedThreads) {
    kahan_add(ka, a[i]);
    kahan_add(kb, b[i]);
  }
  block_merge(ka, kb, sh);
  if (threadIdx.x == 0) {
    partials[4 * blockIdx.x + 0] = ka.s;
    partials[4 * blockIdx.x + 1] = ka.c;
    partials[4 * blockIdx.x + 2] = kb.s;
    partials[4 * blockIdx.x + 3] = kb.c;
  }
}

__global__ void __launch_bounds__(kRedThreads)
    k_ledger_pass2(const double* __restrict__ partials, int nparts,
                   double* __restrict__ out) {
  __shared__ KSum sh[2][kRedThreads];
  KSum ka{0.0, 0.0}, kb{0.0, 0.0};
  for (int i = threadIdx.x; i < nparts; i += kRedThreads) {
    ka = merge(ka, KSum{partials[4 * i + 0], partials[4 * i + 1]});
    kb = merge(kb, KSum{partials[4 * i + 2], partials[4 * i + 3]});
  }
  block_merge(ka, kb, sh);
  if (threadIdx.x == 0) {
    out[0] = ka.s - ka.c;
    out[1] = kb.s - kb.c;
  }
}

cudaError_t launch_ledger_reduce(const double* a, const double* b, int64_t n,
                                 double* partials, int nblocks, double* out,
                                 cudaStream_t s) {
  k_ledger_pass1<<<nblocks, kRedThreads, 0, s>>>(a, b, n, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_ledger_pass2<<<1, kRedThreads, 0, s>>>(partials, nblocks, out);
  return cudaGetLastError();
}

}  // namespace prad
