// Angular distribution of the emitted energy (Fig. 4 of arXiv:1409.5574: the
// emitted energy over the front hemisphere around the laser propagation
// direction).  Each held photon record adds energy x weight to the bin of
// its direction: polar angle theta from the axis (bins uniform over
// [0, theta_max]) and azimuth phi around it, measured from the projection of
// a reference vector (bins uniform over [0, 2 pi)).  Block-private FP64
// histograms in shared memory, added to the output with one atomic per bin
// and block (FP64 sums: the order of the adds varies between runs in the
// last bits).
#include <cuda_runtime.h>
#include <stdint.h>

#include "prad_internal.h"

namespace prad {

namespace {

__global__ void k_angular_hist(AngularArgs a) {
  extern __shared__ double hist[];
  const int nb = a.ntheta * a.nphi;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) hist[b] = 0.0;
  __syncthreads();
  const unsigned long long cur = *a.cursor;
  const unsigned long long held =
      cur < static_cast<unsigned long long>(a.cap) ? cur : static_cast<unsigned long long>(a.cap);
  const double kTwoPi = 6.283185307179586476925286766559;
  for (unsigned long long i = blockIdx.x * static_cast<unsigned long long>(blockDim.x) + threadIdx.x;
       i < held; i += static_cast<unsigned long long>(gridDim.x) * blockDim.x) {
    const double nx = a.nx[i], ny = a.ny[i], nz = a.nz[i];
    const double c = nx * a.axis[0] + ny * a.axis[1] + nz * a.axis[2];
    const double th = acos(fmin(fmax(c, -1.0), 1.0));
    if (!(th <= a.theta_max)) continue;  // also drops NaN directions
    const double p1 = nx * a.e1[0] + ny * a.e1[1] + nz * a.e1[2];
    const double p2 = nx * a.e2[0] + ny * a.e2[1] + nz * a.e2[2];
    double ph = atan2(p2, p1);
    if (ph < 0.0) ph += kTwoPi;
    int it = static_cast<int>(th * (a.ntheta / a.theta_max));
    int ip = static_cast<int>(ph * (a.nphi / kTwoPi));
    it = it < a.ntheta ? it : a.ntheta - 1;
    ip = ip < a.nphi ? (ip >= 0 ? ip : 0) : a.nphi - 1;
    atomicAdd(&hist[it * a.nphi + ip],
              static_cast<double>(a.eps[i]) * static_cast<double>(a.weight[i]));
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nb; b += blockDim.x)
    if (hist[b] != 0.0) atomicAdd(a.out + b, hist[b]);
}

}  // namespace

cudaError_t launch_angular_hist(const AngularArgs& a, int grid, cudaStream_t s) {
  const size_t smem = sizeof(double) * static_cast<size_t>(a.ntheta) * a.nphi;
  cudaError_t e = cudaFuncSetAttribute(k_angular_hist,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(a.out, 0, smem, s);
  if (e != cudaSuccess) return e;
  k_angular_hist<<<grid, 256, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace prad
