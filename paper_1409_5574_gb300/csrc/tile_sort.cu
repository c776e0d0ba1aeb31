// Counting sort of particles by the 32 x 32-cell tile of the 2D Yee grid that
// holds them (histogram -> exclusive scan -> scatter into a scratch copy), then
// by cell inside each tile (one block per tile, scattering back into the
// caller's arrays), and the work list of the tile-staged gather kernel: one
// item per chunk of at most kChunk particles of one tile.  In cell order the
// lanes of a warp read the same or neighbouring stencil values of the staged
// tile (broadcasts instead of shared-memory bank conflicts).  Particles keep
// their ids (pid array), so the Philox streams and ledger entries follow
// them.  The order inside a cell depends on atomic timing; results per
// particle do not.
#include <cuda_runtime.h>
#include <stdint.h>

#include "prad_internal.h"

namespace prad {

namespace {

// The grid cell (ix, iy) that holds (x, y): periodic, clamped (also for NaN)
// into range.
template <typename R>
__device__ __forceinline__ int2 cell_xy(R x, R y, int nx, int ny, R x0, R y0, R inv_dx,
                                        R inv_dy) {
  R xi = (x - x0) * inv_dx, yi = (y - y0) * inv_dy;
  const R fx = static_cast<R>(nx), fy = static_cast<R>(ny);
  xi -= fx * floor(xi / fx);
  yi -= fy * floor(yi / fy);
  int ix = static_cast<int>(fmin(fmax(xi, R(0)), fx - R(1)));
  int iy = static_cast<int>(fmin(fmax(yi, R(0)), fy - R(1)));
  ix = ix < 0 ? 0 : (ix >= nx ? nx - 1 : ix);
  iy = iy < 0 ? 0 : (iy >= ny ? ny - 1 : iy);
  return make_int2(ix, iy);
}

template <typename R>
__device__ __forceinline__ int tile_of(R x, R y, int nx, int ny, int ntx, R x0, R y0,
                                       R inv_dx, R inv_dy) {
  const int2 c = cell_xy(x, y, nx, ny, x0, y0, inv_dx, inv_dy);
  return (c.y / kTile) * ntx + (c.x / kTile);
}

// The cell's index inside its tile, row-major (0 .. kTile^2 - 1).
template <typename R>
__device__ __forceinline__ int cell_in_tile(R x, R y, int nx, int ny, R x0, R y0, R inv_dx,
                                            R inv_dy) {
  const int2 c = cell_xy(x, y, nx, ny, x0, y0, inv_dx, inv_dy);
  return (c.y % kTile) * kTile + (c.x % kTile);
}

// Warp-aggregated increment of counter[t] for every valid lane: lanes of the
// warp with the same tile form one group, its first lane adds the group's
// size with one atomic, and each lane receives base + its rank in the group.
// Particles stay nearly tile-ordered between sorts, so a warp usually holds
// one or two tiles: one or two atomics per 32 particles instead of 32 on the
// same counter.  Warp-collective (every lane calls it).
__device__ __forceinline__ unsigned int warp_claim(unsigned int* counter, int t, bool valid) {
  const int lane = threadIdx.x & 31;
  const unsigned vmask = __ballot_sync(0xffffffffu, valid);
  unsigned int slot = 0u;
  if (valid) {
    const unsigned peers = __match_any_sync(vmask, t);
    const int leader = __ffs(peers) - 1;
    const int rank = __popc(peers & ((1u << lane) - 1u));
    unsigned int base = 0u;
    if (lane == leader) base = atomicAdd(counter + t, static_cast<unsigned int>(__popc(peers)));
    slot = __shfl_sync(peers, base, leader) + static_cast<unsigned int>(rank);
  }
  return slot;
}

// Grid-stride over warps of 32 consecutive particles (every lane of a warp
// takes the same number of iterations).
template <typename R>
__global__ void k_tile_count(const R* __restrict__ x, const R* __restrict__ y, int64_t n,
                             int nx, int ny, int ntx, R x0, R y0, R inv_dx, R inv_dy,
                             unsigned int* __restrict__ counts) {
  const int lane = threadIdx.x & 31;
  const int64_t wstride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t w0 = blockIdx.x * static_cast<int64_t>(blockDim.x) + (threadIdx.x & ~31);
       w0 < n; w0 += wstride) {
    const int64_t i = w0 + lane;
    const bool valid = i < n;
    const int t = valid ? tile_of(x[i], y[i], nx, ny, ntx, x0, y0, inv_dx, inv_dy) : 0;
    (void)warp_claim(counts, t, valid);
  }
}

// One block: exclusive scan of the tile counts (starts, scatter cursors) and
// of the per-tile chunk counts (work list offsets); writes the work list.
constexpr int kScanThreads = 1024;

__global__ void __launch_bounds__(kScanThreads)
    k_tile_scan(const unsigned int* __restrict__ counts, int ntiles,
                unsigned int* __restrict__ starts, unsigned int* __restrict__ cursor,
                int4* __restrict__ work, unsigned int* __restrict__ work_count) {
  __shared__ unsigned int s_part[kScanThreads], s_chunk[kScanThreads];
  const int per = (ntiles + kScanThreads - 1) / kScanThreads;
  const int lo = threadIdx.x * per;
  const int hi = min(lo + per, ntiles);
  unsigned int sum = 0, csum = 0;
  for (int t = lo; t < hi; ++t) {
    sum += counts[t];
    csum += (counts[t] + kChunk - 1) / kChunk;
  }
  s_part[threadIdx.x] = sum;
  s_chunk[threadIdx.x] = csum;
  __syncthreads();
  // Hillis-Steele inclusive scan over the thread partials
  for (int off = 1; off < kScanThreads; off <<= 1) {
    const unsigned int a = threadIdx.x >= off ? s_part[threadIdx.x - off] : 0u;
    const unsigned int b = threadIdx.x >= off ? s_chunk[threadIdx.x - off] : 0u;
    __syncthreads();
    s_part[threadIdx.x] += a;
    s_chunk[threadIdx.x] += b;
    __syncthreads();
  }
  unsigned int run = s_part[threadIdx.x] - sum;
  unsigned int wrun = s_chunk[threadIdx.x] - csum;
  for (int t = lo; t < hi; ++t) {
    const unsigned int c = counts[t];
    starts[t] = run;
    cursor[t] = run;
    for (unsigned int f = 0; f < c; f += kChunk) {
      const unsigned int e = f + kChunk < c ? f + kChunk : c;
      work[wrun++] = make_int4(t, static_cast<int>(run + f), static_cast<int>(run + e), 0);
    }
    run += c;
  }
  if (threadIdx.x == kScanThreads - 1) {
    starts[ntiles] = run;
    *work_count = wrun;
  }
}

template <typename R>
struct Arrays7 {
  R* p[7];  // x y z ux uy uz w (z may be null)
};

template <typename R>
__global__ void k_tile_scatter(const Arrays7<R> src, const Arrays7<R> dst,
                               const uint32_t* __restrict__ pid, uint32_t* __restrict__ pid_out,
                               int64_t n, int nx, int ny, int ntx, R x0, R y0, R inv_dx,
                               R inv_dy, unsigned int* __restrict__ cursor) {
  const int lane = threadIdx.x & 31;
  const int64_t wstride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t w0 = blockIdx.x * static_cast<int64_t>(blockDim.x) + (threadIdx.x & ~31);
       w0 < n; w0 += wstride) {
    const int64_t i = w0 + lane;
    const bool valid = i < n;
    const int t =
        valid ? tile_of(src.p[0][i], src.p[1][i], nx, ny, ntx, x0, y0, inv_dx, inv_dy) : 0;
    const unsigned int d = warp_claim(cursor, t, valid);
    if (valid) {
#pragma unroll
      for (int k = 0; k < 7; ++k)
        if (src.p[k]) dst.p[k][d] = src.p[k][i];
      pid_out[d] = pid[i];
    }
  }
}

// Second pass, one block per tile: the tile's particles (a contiguous range
// of the tile-sorted scratch copy) are ordered by cell with a shared-memory
// histogram of the tile's kTile^2 cells, and written back to the caller's
// arrays.  The cell is computed with the same arithmetic as the tile, so
// every particle stays inside its tile's range.
constexpr int kCellThreads = kTile * kTile;

template <typename R>
__global__ void __launch_bounds__(kCellThreads)
    k_cell_scatter(const Arrays7<R> src, const Arrays7<R> dst,
                   const uint32_t* __restrict__ pid_src, uint32_t* __restrict__ pid_dst,
                   const unsigned int* __restrict__ starts, int nx, int ny, R x0, R y0,
                   R inv_dx, R inv_dy) {
  __shared__ unsigned int s_cnt[kCellThreads];
  __shared__ unsigned int s_warp[kCellThreads / 32];
  const unsigned int a = starts[blockIdx.x], b = starts[blockIdx.x + 1];
  if (a == b) return;  // the whole block leaves: no barrier is left waiting
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  s_cnt[tid] = 0u;
  __syncthreads();
  for (unsigned int i = a + tid; i < b; i += kCellThreads)
    atomicAdd(s_cnt + cell_in_tile(src.p[0][i], src.p[1][i], nx, ny, x0, y0, inv_dx, inv_dy),
              1u);
  __syncthreads();
  // exclusive scan of the cell counts: within warps, then over the warp sums
  const unsigned int c = s_cnt[tid];
  unsigned int v = c;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const unsigned int u = __shfl_up_sync(0xffffffffu, v, off);
    if (lane >= off) v += u;
  }
  if (lane == 31) s_warp[warp] = v;
  __syncthreads();
  if (warp == 0) {
    unsigned int w = s_warp[lane];
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const unsigned int u = __shfl_up_sync(0xffffffffu, w, off);
      if (lane >= off) w += u;
    }
    s_warp[lane] = w;
  }
  __syncthreads();
  s_cnt[tid] = (warp > 0 ? s_warp[warp - 1] : 0u) + v - c;  // cursor of cell tid
  __syncthreads();
  for (unsigned int i = a + tid; i < b; i += kCellThreads) {
    const int cl = cell_in_tile(src.p[0][i], src.p[1][i], nx, ny, x0, y0, inv_dx, inv_dy);
    const unsigned int d = a + atomicAdd(s_cnt + cl, 1u);
#pragma unroll
    for (int k = 0; k < 7; ++k)
      if (src.p[k]) dst.p[k][d] = src.p[k][i];
    pid_dst[d] = pid_src[i];
  }
}

}  // namespace

template <typename R>
cudaError_t launch_tile_sort(R* arr[7], uint32_t* pid, int64_t n, const SortBuffers& b,
                             int nx, int ny, double x0, double y0, double inv_dx,
                             double inv_dy, cudaStream_t s) {
  const int ntx = (nx + kTile - 1) / kTile;
  cudaError_t e = cudaMemsetAsync(b.counts, 0, sizeof(unsigned int) * b.ntiles, s);
  if (e != cudaSuccess) return e;
  const int block = 256;
  const int64_t want = (n + block - 1) / block;
  const int grid = static_cast<int>(want < 8192 ? (want > 0 ? want : 1) : 8192);
  k_tile_count<R><<<grid, block, 0, s>>>(arr[0], arr[1], n, nx, ny, ntx, R(x0), R(y0),
                                         R(inv_dx), R(inv_dy), b.counts);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_tile_scan<<<1, kScanThreads, 0, s>>>(b.counts, b.ntiles, b.starts, b.cursor, b.work,
                                          b.work_count);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  Arrays7<R> srcp, dstp;
  for (int k = 0; k < 7; ++k) {
    srcp.p[k] = arr[k];
    dstp.p[k] = arr[k] ? static_cast<R*>(b.tmp[k]) : nullptr;
  }
  k_tile_scatter<R><<<grid, block, 0, s>>>(srcp, dstp, pid, b.tmp_pid, n, nx, ny, ntx, R(x0),
                                           R(y0), R(inv_dx), R(inv_dy), b.cursor);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // back into the caller's arrays, in cell order inside each tile
  k_cell_scatter<R><<<b.ntiles, kCellThreads, 0, s>>>(dstp, srcp, b.tmp_pid, pid, b.starts, nx,
                                                      ny, R(x0), R(y0), R(inv_dx), R(inv_dy));
  return cudaGetLastError();
}

template cudaError_t launch_tile_sort<float>(float* [7], uint32_t*, int64_t, const SortBuffers&,
                                             int, int, double, double, double, double,
                                             cudaStream_t);
template cudaError_t launch_tile_sort<double>(double* [7], uint32_t*, int64_t,
                                              const SortBuffers&, int, int, double, double,
                                              double, double, cudaStream_t);

}  // namespace prad
