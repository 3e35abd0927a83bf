// Sub-voxel translation refinement (dses_refine_translation).
//
// Algorithm 2 returns the translation as a voxel centre t* = k* delta_t, so its
// error is up to (sqrt 3 / 2) delta_t. With the pose's correspondences fixed --
// every source point paired with its nearest target, kept when closer than
// epsilon as in Eq. 3 -- the translation that minimises the summed squared
// residual of those pairs is the mean of y_nn(i) - R x_i. One step is one
// launch of refine_step_kernel (sums in FP64) and one of refine_update_kernel
// (t <- mean, or unchanged with no pair), so repeated steps stay on the device.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>

#include "kernels.cuh"

namespace dses {

extern std::atomic<long long> g_launches;

namespace {

constexpr int kRefineThreads = 256;

// Nearest target strictly within epsilon of q through the cell list (cells at
// least epsilon wide, so the 3x3x3 neighbourhood holds every such point);
// returns its index in the cell-ordered target array, or -1.
__device__ __forceinline__ int nearest_within(const RefineDesc& d, float qx, float qy, float qz) {
  const float fx = (qx - d.cell_lo[0]) * d.cell_inv;
  const float fy = (qy - d.cell_lo[1]) * d.cell_inv;
  const float fz = (qz - d.cell_lo[2]) * d.cell_inv;
  const int cx = (int)floorf(fminf(fmaxf(fx, -2.f), (float)d.cell_dim[0] + 1.f));
  const int cy = (int)floorf(fminf(fmaxf(fy, -2.f), (float)d.cell_dim[1] + 1.f));
  const int cz = (int)floorf(fminf(fmaxf(fz, -2.f), (float)d.cell_dim[2] + 1.f));
  const int x0 = max(cx - 1, 0), x1 = min(cx + 1, d.cell_dim[0] - 1);
  const int y0 = max(cy - 1, 0), y1 = min(cy + 1, d.cell_dim[1] - 1);
  const int z0 = max(cz - 1, 0), z1 = min(cz + 1, d.cell_dim[2] - 1);
  float best = d.eps2;
  int jb = -1;
  if (x0 > x1 || y0 > y1 || z0 > z1) return -1;
  for (int z = z0; z <= z1; ++z)
    for (int y = y0; y <= y1; ++y) {
      const int row = (z * d.cell_dim[1] + y) * d.cell_dim[0];
      const int s = __ldg(d.cell_start + row + x0), e = __ldg(d.cell_start + row + x1 + 1);
      for (int j = s; j < e; ++j) {
        const float4 p = __ldg(d.Y + j);
        const float dx = p.x - qx, dy = p.y - qy, dz = p.z - qz;
        const float dd = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        if (dd < best) {
          best = dd;
          jb = j;
        }
      }
    }
  return jb;
}

__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// acc[0..2] += sum over this grid's inliers of (y_nn(i) - R x_i); acc[3] += count.
__global__ void __launch_bounds__(kRefineThreads) refine_step_kernel(RefineDesc d) {
  __shared__ double part[kRefineThreads / 32][4];
  const float tx = (float)d.t[0], ty = (float)d.t[1], tz = (float)d.t[2];
  double sx = 0.0, sy = 0.0, sz = 0.0, n = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.N; i += gridDim.x * blockDim.x) {
    const float x = __ldg(d.X + 3 * (size_t)i), y = __ldg(d.X + 3 * (size_t)i + 1), z = __ldg(d.X + 3 * (size_t)i + 2);
    const float ux = fmaf(d.R[0], x, fmaf(d.R[1], y, d.R[2] * z));
    const float uy = fmaf(d.R[3], x, fmaf(d.R[4], y, d.R[5] * z));
    const float uz = fmaf(d.R[6], x, fmaf(d.R[7], y, d.R[8] * z));
    const int j = nearest_within(d, ux + tx, uy + ty, uz + tz);
    if (j >= 0) {
      const float4 p = __ldg(d.Y + j);
      sx += (double)p.x - (double)ux;
      sy += (double)p.y - (double)uy;
      sz += (double)p.z - (double)uz;
      n += 1.0;
    }
  }
  sx = warp_sum_f64(sx);
  sy = warp_sum_f64(sy);
  sz = warp_sum_f64(sz);
  n = warp_sum_f64(n);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    part[warp][0] = sx;
    part[warp][1] = sy;
    part[warp][2] = sz;
    part[warp][3] = n;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double s = 0.0;
    for (int w = 0; w < kRefineThreads / 32; ++w) s += part[w][threadIdx.x];
    if (s != 0.0) atomicAdd(d.acc + threadIdx.x, s);
  }
}

// t <- acc[0..2] / acc[3] when some pair was kept; records the count and
// clears the sums for the next step.
__global__ void refine_update_kernel(double* t, double* acc, uint32_t* n_out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double n = acc[3];
  if (n > 0.0)
    for (int a = 0; a < 3; ++a) t[a] = acc[a] / n;
  *n_out = (uint32_t)n;
  acc[0] = acc[1] = acc[2] = acc[3] = 0.0;
}

}  // namespace

cudaError_t launch_refine_step(const RefineDesc& d, uint32_t* n_out, cudaStream_t s) {
  int sms = 148;
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = std::max(1, std::min((d.N + kRefineThreads - 1) / kRefineThreads, sms * 8));
  g_launches.fetch_add(2, std::memory_order_relaxed);
  refine_step_kernel<<<blocks, kRefineThreads, 0, s>>>(d);
  refine_update_kernel<<<1, 32, 0, s>>>(d.t, d.acc, n_out);
  return cudaGetLastError();
}

}  // namespace dses
