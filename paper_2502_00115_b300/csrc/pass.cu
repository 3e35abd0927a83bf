// Rotation pass: the hot loop of Direct Semi-Exhaustive Search (Algorithm 2).
//
// For every rotation R of a work item, one CTA (32 warps, one CTA per SM):
//   1. rotates the source cloud and stages per-point lattice offsets
//      c_i = 1/2 - (R x_i)/delta - lo in shared memory;
//   2. votes every pair (i, j): k = floor(y_j/delta + c_i) (the ROUND of
//      Algorithm 2 relative to the box corner); pairs inside the lattice box
//      increment a shared-memory histogram (Lemma 1, Eq. 5: the translation
//      mode of the rotated pairwise differences);
//   3. scans and clears the histogram for the mode: V = max count, k* = the
//      lexicographically smallest bin holding V;
//   4. counts the inliers of Eq. 3 at t* = k* delta through the target cell
//      list (exact Euclidean test against epsilon), and, when every rotation
//      is a candidate, also sums the robust cost from the target's truncated
//      distance grid;
//   5. publishes (k*, V, M, cost) and folds M*, max V and the argmin key into
//      per-problem accumulators.
// Work items are (problem, rotation tile) pairs taken from a global counter, so
// one persistent launch serves one problem or a batch of uneven problems.
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.cuh"

#include <atomic>

namespace dses {

extern std::atomic<long long> g_launches;

namespace {

// floor(v) for |v| < 2^22: adding 1.5 * 2^23 rounding toward -inf leaves
// floor(v) in the low mantissa bits. Out-of-range v map to huge unsigned
// values, i.e. outside every box.
constexpr float kMagic = 12582912.0f;
constexpr int kMagicBits = 0x4B400000;

__device__ __forceinline__ unsigned floor_bits(float v) {
  return (unsigned)(__float_as_int(__fadd_rd(v, kMagic)) - kMagicBits);
}

__device__ __forceinline__ float rho(int metric, float d, float eps, float tau, float h, float p) {
  switch (metric) {
    case 0:
      return d < eps ? 0.f : 1.f;
    case 1:
      return fminf(d, tau);
    case 2: {
      const float e = fminf(d, tau);
      return e * e;
    }
    case 3: {
      const float e = fminf(d, tau);
      return e <= h ? 0.5f * e * e : h * (e - 0.5f * h);
    }
    default:
      return powf(d, p);
  }
}

// Trilinear interpolation between voxel centres of the truncated distance
// grid, clamped at the outermost centres; outside the grid box: the cap.
__device__ __forceinline__ float grid_lookup(const PassDesc& d, float qx, float qy, float qz) {
  const float G = (float)d.G;
  float gx = (qx - d.glo[0]) * d.ginv_h[0];
  float gy = (qy - d.glo[1]) * d.ginv_h[1];
  float gz = (qz - d.glo[2]) * d.ginv_h[2];
  if (!(gx >= 0.f && gx <= G && gy >= 0.f && gy <= G && gz >= 0.f && gz <= G)) return d.gcap;
  gx = fminf(fmaxf(gx - 0.5f, 0.f), G - 1.f);
  gy = fminf(fmaxf(gy - 0.5f, 0.f), G - 1.f);
  gz = fminf(fmaxf(gz - 0.5f, 0.f), G - 1.f);
  const int ix = min((int)gx, d.G - 2), iy = min((int)gy, d.G - 2), iz = min((int)gz, d.G - 2);
  const float fx = gx - (float)ix, fy = gy - (float)iy, fz = gz - (float)iz;
  const float* b = d.D + ((size_t)ix * d.G + iy) * d.G + iz;
  const size_t sy = d.G, sx = (size_t)d.G * d.G;
  const float c00 = b[0] + fz * (b[1] - b[0]);
  const float c01 = b[sy] + fz * (b[sy + 1] - b[sy]);
  const float c10 = b[sx] + fz * (b[sx + 1] - b[sx]);
  const float c11 = b[sx + sy] + fz * (b[sx + sy + 1] - b[sx + sy]);
  const float c0 = c00 + fy * (c01 - c00);
  const float c1 = c10 + fy * (c11 - c10);
  return c0 + fx * (c1 - c0);
}

// Is some target point strictly within epsilon of q? (Eq. 3, one source point.)
// Cells are at least epsilon wide, so the 3x3x3 cell neighbourhood suffices.
__device__ __forceinline__ bool has_inlier(const PassDesc& d, float qx, float qy, float qz) {
  const float fx = (qx - d.cell_lo[0]) * d.cell_inv;
  const float fy = (qy - d.cell_lo[1]) * d.cell_inv;
  const float fz = (qz - d.cell_lo[2]) * d.cell_inv;
  // clamp before converting so far-away queries stay well defined
  const int cx = (int)floorf(fminf(fmaxf(fx, -2.f), (float)d.cell_dim[0] + 1.f));
  const int cy = (int)floorf(fminf(fmaxf(fy, -2.f), (float)d.cell_dim[1] + 1.f));
  const int cz = (int)floorf(fminf(fmaxf(fz, -2.f), (float)d.cell_dim[2] + 1.f));
  const int x0 = max(cx - 1, 0), x1 = min(cx + 1, d.cell_dim[0] - 1);
  const int y0 = max(cy - 1, 0), y1 = min(cy + 1, d.cell_dim[1] - 1);
  const int z0 = max(cz - 1, 0), z1 = min(cz + 1, d.cell_dim[2] - 1);
  if (x0 > x1 || y0 > y1 || z0 > z1) return false;
  for (int z = z0; z <= z1; ++z)
    for (int y = y0; y <= y1; ++y) {
      const int row = (z * d.cell_dim[1] + y) * d.cell_dim[0];
      const int s = __ldg(d.cell_start + row + x0), e = __ldg(d.cell_start + row + x1 + 1);
      for (int j = s; j < e; ++j) {
        const float4 p = __ldg(d.Y + j);
        const float dx = p.x - qx, dy = p.y - qy, dz = p.z - qz;
        if (fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < d.eps2) return true;
      }
    }
  return false;
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

// Vote all (source in this chunk) x (target) pairs of the CTA's items into the
// slab histogram. Item = (target chunk of 32 P points, source group); a warp
// holds its P targets per lane in registers and streams the source offsets
// from shared memory (broadcast reads).
template <int P, bool U16>
__device__ __forceinline__ void vote_chunk(const PassDesc& d, const float4* __restrict__ srcc, int nsrc,
                                           unsigned SX, uint32_t* __restrict__ hist, int warp, int lane) {
  const int n_tchunks = d.n_tchunks, n_sgroups = d.n_sgroups;
  const int n_items = n_tchunks * n_sgroups;
  const int spg = (nsrc + n_sgroups - 1) / n_sgroups;
  const unsigned Ey = (unsigned)d.E[1], Ez = (unsigned)d.E[2];
  const float inv = d.inv_delta;
  const int M = d.M;
  const float4* __restrict__ Y = d.Y;
  for (int it = warp; it < n_items; it += kPassThreads / 32) {
    const int tc = it % n_tchunks, sg = it / n_tchunks;
    float ty[P][3];
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const int j = (tc * P + p) * 32 + lane;
      if (j < M) {
        const float4 q = __ldg(Y + j);
        ty[p][0] = q.x; ty[p][1] = q.y; ty[p][2] = q.z;
      } else {  // padding lane: lands far outside every box
        ty[p][0] = 1e30f; ty[p][1] = 1e30f; ty[p][2] = 1e30f;
      }
    }
    const int i0 = sg * spg, i1 = min(i0 + spg, nsrc);
    for (int i = i0; i < i1; ++i) {
      const float4 c = srcc[i];
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const unsigned bx = floor_bits(fmaf(ty[p][0], inv, c.x));
        const unsigned by = floor_bits(fmaf(ty[p][1], inv, c.y));
        const unsigned bz = floor_bits(fmaf(ty[p][2], inv, c.z));
        if (bx < SX && by < Ey && bz < Ez) {
          const unsigned bin = (bx * Ey + by) * Ez + bz;
          if (U16)
            atomicAdd(&hist[bin >> 1], 1u << ((bin & 1u) << 4));
          else
            atomicAdd(&hist[bin], 1u);
        }
      }
    }
  }
}

template <int P>
__global__ void __launch_bounds__(kPassThreads, 1) rotation_pass_kernel(PassLaunch L) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ PassDesc sd;
  __shared__ unsigned long long red64[32];
  __shared__ float redf[32];
  __shared__ int redi[32];
  __shared__ int s_item, s_prob;

  uint32_t* hist = reinterpret_cast<uint32_t*>(smem);
  float4* srcc = reinterpret_cast<float4*>(smem + L.hist_bytes);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  for (int w = tid; w < L.hist_bytes / 4; w += kPassThreads) hist[w] = 0u;
  int cur_prob = -1;
  const int total_tiles = L.tile_prefix[L.n_probs];

  for (;;) {
    if (tid == 0) {
      const int item = atomicAdd(L.work_counter, 1);
      int p = -1;
      if (item < total_tiles) {
        int lo = 0, hi = L.n_probs - 1;  // last p with tile_prefix[p] <= item
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (L.tile_prefix[mid] <= item) lo = mid; else hi = mid - 1;
        }
        p = lo;
      }
      s_item = item;
      s_prob = p;
    }
    __syncthreads();
    const int item = s_item, p = s_prob;
    if (p < 0) break;
    if (p != cur_prob) {
      const int words = (int)(sizeof(PassDesc) / 4);
      if (tid < words)
        reinterpret_cast<int*>(&sd)[tid] = reinterpret_cast<const int*>(&L.probs[p])[tid];
      cur_prob = p;
    }
    __syncthreads();
    const PassDesc& d = sd;
    const int r0 = (item - L.tile_prefix[p]) * L.tile_rot;
    const int r1 = min(r0 + L.tile_rot, d.n_rot);

    for (int r = r0; r < r1; ++r) {
      float R[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) R[k] = __ldg(d.rot + 9 * (size_t)r + k);
      const unsigned Ey = (unsigned)d.E[1], Ez = (unsigned)d.E[2];
      unsigned long long best = 0ull;  // (count << 32) | ~global_bin, max wins

      for (int s = 0; s < d.n_slabs; ++s) {
        const int x0 = s * d.slab_x;
        const unsigned SX = (unsigned)min(d.slab_x, d.E[0] - x0);
        const float off0 = 0.5f - (float)(d.lo[0] + x0);
        const float off1 = 0.5f - (float)d.lo[1];
        const float off2 = 0.5f - (float)d.lo[2];
        for (int c0 = 0; c0 < d.N; c0 += kSrcChunk) {
          const int c1 = min(c0 + kSrcChunk, d.N);
          __syncthreads();  // previous chunk's readers are done
          for (int i = c0 + tid; i < c1; i += kPassThreads) {
            const float x = __ldg(d.X + 3 * (size_t)i), y = __ldg(d.X + 3 * (size_t)i + 1),
                        z = __ldg(d.X + 3 * (size_t)i + 2);
            const float ux = fmaf(R[0], x, fmaf(R[1], y, R[2] * z));
            const float uy = fmaf(R[3], x, fmaf(R[4], y, R[5] * z));
            const float uz = fmaf(R[6], x, fmaf(R[7], y, R[8] * z));
            srcc[i - c0] = make_float4(fmaf(-ux, d.inv_delta, off0), fmaf(-uy, d.inv_delta, off1),
                                       fmaf(-uz, d.inv_delta, off2), 0.f);
          }
          __syncthreads();
          if (d.hist_u16)
            vote_chunk<P, true>(d, srcc, c1 - c0, SX, hist, warp, lane);
          else
            vote_chunk<P, false>(d, srcc, c1 - c0, SX, hist, warp, lane);
        }
        __syncthreads();
        // mode of this slab: scan and clear; each thread walks increasing bins
        const unsigned nbins = SX * Ey * Ez;
        unsigned bc = 0, bb = 0;
        if (d.hist_u16) {
          const unsigned words = (nbins + 1) >> 1;
          for (unsigned w = tid; w < words; w += kPassThreads) {
            const uint32_t v = hist[w];
            hist[w] = 0u;
            const unsigned a = v & 0xffffu, b = v >> 16;
            if (a > bc) { bc = a; bb = 2 * w; }
            if (b > bc) { bc = b; bb = 2 * w + 1; }
          }
        } else {
          for (unsigned w = tid; w < nbins; w += kPassThreads) {
            const uint32_t v = hist[w];
            hist[w] = 0u;
            if (v > bc) { bc = v; bb = w; }
          }
        }
        const unsigned gbin = (unsigned)x0 * Ey * Ez + bb;
        unsigned long long key = ((unsigned long long)bc << 32) | (unsigned long long)(0xffffffffu - gbin);
        key = warp_max_u64(key);
        if (lane == 0) red64[warp] = key;
        __syncthreads();
        if (warp == 0) {
          const unsigned long long k2 = warp_max_u64(red64[lane]);
          if (lane == 0) red64[0] = k2;
        }
        __syncthreads();
        const unsigned long long sk = red64[0];
        // strict: an earlier slab holds smaller bins and keeps ties
        if (s == 0 || (sk >> 32) > (best >> 32)) best = sk;
        __syncthreads();
      }

      const unsigned V = (unsigned)(best >> 32);
      const unsigned gbin = 0xffffffffu - (unsigned)(best & 0xffffffffull);
      const int kx = d.lo[0] + (int)(gbin / (Ey * Ez));
      const int ky = d.lo[1] + (int)((gbin / Ez) % Ey);
      const int kz = d.lo[2] + (int)(gbin % Ez);
      const float tx = (float)kx * d.delta, ty = (float)ky * d.delta, tz = (float)kz * d.delta;

      // inlier count (Eq. 3) and, on the fused path, the robust cost
      int cnt = 0;
      float csum = 0.f;
      const bool grid_cost = d.fuse_score && d.metric != 0;
      for (int i = tid; i < d.N; i += kPassThreads) {
        const float x = __ldg(d.X + 3 * (size_t)i), y = __ldg(d.X + 3 * (size_t)i + 1),
                    z = __ldg(d.X + 3 * (size_t)i + 2);
        const float qx = fmaf(R[0], x, fmaf(R[1], y, R[2] * z)) + tx;
        const float qy = fmaf(R[3], x, fmaf(R[4], y, R[5] * z)) + ty;
        const float qz = fmaf(R[6], x, fmaf(R[7], y, R[8] * z)) + tz;
        cnt += has_inlier(d, qx, qy, qz) ? 1 : 0;
        if (grid_cost) csum += rho(d.metric, grid_lookup(d, qx, qy, qz), d.eps, d.tau, d.huber_h, d.p_exp);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        csum += __shfl_xor_sync(0xffffffffu, csum, o);
      }
      if (lane == 0) { redi[warp] = cnt; redf[warp] = csum; }
      __syncthreads();
      if (warp == 0) {
        int c2 = redi[lane];
        float f2 = redf[lane];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          c2 += __shfl_xor_sync(0xffffffffu, c2, o);
          f2 += __shfl_xor_sync(0xffffffffu, f2, o);
        }
        if (lane == 0) {
          const uint32_t gidx = d.rot_base + (uint32_t)r;
          const uint32_t o = gidx - d.out_base;
          d.kv[o] = make_int4(kx, ky, kz, (int)V);
          d.Mout[o] = (uint32_t)c2;
          atomicMax(d.acc + 0, (uint32_t)c2);
          atomicMax(d.acc + 1, V);
          if (d.fuse_score) {
            const float cost = d.metric == 0 ? (float)(d.N - c2) : f2;
            d.cost[o] = cost;
            const unsigned long long bkey =
                ((unsigned long long)__float_as_uint(cost) << 32) | (unsigned long long)gidx;
            atomicMin(d.best, bkey);
          }
        }
      }
      __syncthreads();
    }
  }
}

template <int P>
cudaError_t launch_p(const PassLaunch& L, int grid_ctas, cudaStream_t s) {
  const int smem = pass_smem_bytes(L.hist_bytes);
  static int configured = 0;
  if (configured < smem) {
    cudaError_t e =
        cudaFuncSetAttribute(rotation_pass_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  g_launches.fetch_add(1, std::memory_order_relaxed);
  rotation_pass_kernel<P><<<grid_ctas, kPassThreads, smem, s>>>(L);
  return cudaGetLastError();
}

}  // namespace

int pass_smem_bytes(int hist_bytes) { return hist_bytes + kSrcChunk * (int)sizeof(float4); }

cudaError_t launch_rotation_pass(const PassLaunch& L, int points_per_thread, int grid_ctas, cudaStream_t s) {
  switch (points_per_thread) {
    case 1: return launch_p<1>(L, grid_ctas, s);
    case 2: return launch_p<2>(L, grid_ctas, s);
    case 4: return launch_p<4>(L, grid_ctas, s);
    case 8: return launch_p<8>(L, grid_ctas, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dses
