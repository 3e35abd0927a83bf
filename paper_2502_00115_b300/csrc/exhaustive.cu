// Algorithm 1 (pure exhaustive search) on the GPU, the validator of the DSES
// pass on small problems (dses_exhaustive_search).
//
// For every rotation r and every lattice translation t of the box,
//   e(r, t) = sum_i rho(min_j ||y_j - R_r x_i - t||),
// with exact nearest neighbours: the whole target is staged in shared memory
// and every (r, t, i) scans it. One block per (rotation, translation tile),
// rotation-major in a 1-D grid; each warp
// takes translations of the tile, its lanes take source points. Work is
// n_rot * n_t * N * M distance evaluations, so this is for small clouds.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>

#include "kernels.cuh"

namespace dses {

extern std::atomic<long long> g_launches;

namespace {

constexpr int kExThreads = 256;
constexpr int kExTilesPerBlock = 32;  // translations per block

__global__ void __launch_bounds__(kExThreads) exhaustive_kernel(ExhaustiveDesc d) {
  extern __shared__ float4 sY[];
  const int tiles = (d.n_t + kExTilesPerBlock - 1) / kExTilesPerBlock;
  const int r = (int)(blockIdx.x / (unsigned)tiles);
  const int tile = (int)(blockIdx.x % (unsigned)tiles);
  for (int j = threadIdx.x; j < d.M; j += kExThreads) sY[j] = __ldg(d.Y + j);
  float R[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) R[k] = __ldg(d.rot + 9 * (size_t)r + k);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int Eyz = d.E[1] * d.E[2];
  const int t0 = tile * kExTilesPerBlock;
  const int t1 = min(t0 + kExTilesPerBlock, d.n_t);
  for (int ti = t0 + warp; ti < t1; ti += kExThreads / 32) {
    const int kx = d.lo[0] + ti / Eyz, ky = d.lo[1] + (ti / d.E[2]) % d.E[1], kz = d.lo[2] + ti % d.E[2];
    const float tx = (float)kx * d.delta, ty = (float)ky * d.delta, tz = (float)kz * d.delta;
    float e = 0.f;
    int cnt = 0;
    for (int i = lane; i < d.N; i += 32) {
      const float x = __ldg(d.X + 3 * (size_t)i), y = __ldg(d.X + 3 * (size_t)i + 1),
                  z = __ldg(d.X + 3 * (size_t)i + 2);
      const float qx = fmaf(R[0], x, fmaf(R[1], y, R[2] * z)) + tx;
      const float qy = fmaf(R[3], x, fmaf(R[4], y, R[5] * z)) + ty;
      const float qz = fmaf(R[6], x, fmaf(R[7], y, R[8] * z)) + tz;
      float m2 = 3.4e38f;
      for (int j = 0; j < d.M; ++j) {
        const float4 p = sY[j];  // every lane reads the same word: broadcast
        const float dx = p.x - qx, dy = p.y - qy, dz = p.z - qz;
        m2 = fminf(m2, fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
      }
      const float dist = sqrtf(m2);
      e += robust_rho(d.metric, dist, d.eps, d.tau, d.huber_h, d.p_exp);
      cnt += dist < d.eps ? 1 : 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      e += __shfl_xor_sync(0xffffffffu, e, o);
      cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
    if (lane == 0) {
      const uint32_t idx = (uint32_t)r * (uint32_t)d.n_t + (uint32_t)ti;
      const float cost = d.metric == 0 ? (float)(d.N - cnt) : e;
      d.cost[idx] = cost;
      d.count[idx] = (uint32_t)cnt;
      atomicMin(d.best, ((unsigned long long)__float_as_uint(cost) << 32) | (unsigned long long)idx);
    }
  }
}

}  // namespace

cudaError_t launch_exhaustive(const ExhaustiveDesc& d, cudaStream_t s) {
  const size_t smem = sizeof(float4) * (size_t)d.M;
  if (smem > 48 * 1024) {
    const cudaError_t e =
        cudaFuncSetAttribute(exhaustive_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  // n_rot * n_t <= 2^28, so the block count stays below 2^31
  const long long tiles = (d.n_t + kExTilesPerBlock - 1) / kExTilesPerBlock;
  const unsigned grid = (unsigned)(tiles * d.n_rot);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  exhaustive_kernel<<<grid, kExThreads, smem, s>>>(d);
  return cudaGetLastError();
}

}  // namespace dses
