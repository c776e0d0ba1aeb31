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

#include <cstdio>
#include <mutex>

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

// ---------------------------------------------------------------------------
// Allocation-free totals.  Some callers cannot allocate device memory at the
// point where they need the totals: a host code that owns a fixed device
// memory pool, or a time loop in which a cudaMalloc (which synchronises the
// device and may fail once the pool has claimed the memory) is not
// acceptable.  This variant of the two-pass reduction above keeps its
// per-block partials in a file-scope device array instead of context
// scratch, and calls no allocation routine.
// ---------------------------------------------------------------------------
namespace {

// Each block sums at most kStaticChunk consecutive entries; at most
// kStaticBlocks blocks (4 doubles of partials each: 128 KB, held by every
// GPU that loads the library until the process exits).
constexpr int64_t kStaticChunk = 65536;
constexpr int kStaticBlocks = 4096;
__device__ __align__(256) double g_static_partials[4 * kStaticBlocks];

// Device address of g_static_partials per device, looked up once per device
// (host code must not pass the array's host-side name to a kernel).  The
// address belongs to the device's primary context at the first call; a
// cudaDeviceReset later in the process invalidates it (calls after a reset
// are not supported).
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
double* g_static_addr[kMaxDevices] = {nullptr};

thread_local char g_static_err[256];

int static_fail(int code, const char* msg) {
  std::snprintf(g_static_err, sizeof(g_static_err), "%s", msg);
  return code;
}

}  // namespace

extern "C" const char* prad_ledger_totals_noalloc_error(void) { return g_static_err; }

extern "C" int prad_ledger_totals_noalloc(const double* emit, const double* rr, int64_t n,
                                          double* out, void* stream) {
  g_static_err[0] = '\0';  // the message describes this call's failure only
  if (!out || n < 0 || (n > 0 && (!emit || !rr)))
    return static_fail(PRAD_ERR_ARG, "ledger_totals_noalloc: null pointer or n < 0");
  if (n > kStaticChunk * kStaticBlocks)
    return static_fail(PRAD_ERR_ARG,
                       "ledger_totals_noalloc: n exceeds the static scratch limit of "
                       "268435456 entries (4096 blocks x 65536)");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return static_fail(PRAD_ERR_CUDA, "ledger_totals_noalloc: no usable current device");
  double* partials = nullptr;
  {
    // set-up on the first call per device, with that device current
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_static_partials) != cudaSuccess || !p)
        return static_fail(PRAD_ERR_CUDA, "ledger_totals_noalloc: cudaGetSymbolAddress failed");
      g_static_addr[dev] = static_cast<double*>(p);
    }
    partials = g_static_addr[dev];
  }
  if (n == 0) {  // nothing to read: zero totals without touching the inputs
    const cudaError_t ez = cudaMemsetAsync(out, 0, 2 * sizeof(double),
                                           static_cast<cudaStream_t>(stream));
    return ez == cudaSuccess ? PRAD_OK : static_fail(PRAD_ERR_CUDA, cudaGetErrorString(ez));
  }
  const int64_t nb64 = (n + kStaticChunk - 1) / kStaticChunk;
  const int nblocks = static_cast<int>(nb64);
  // every partial the second pass reads is written by the first: nothing
  // left from an earlier call is used
  const cudaError_t e = prad::launch_ledger_reduce(emit, rr, n, partials, nblocks, out,
                                                   static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return static_fail(PRAD_ERR_CUDA, cudaGetErrorString(e));
  return PRAD_OK;
}
