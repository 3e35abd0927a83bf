// Allocation-free vote entry point (dses_vote_static, declared in dses.h).
//
// Some callers cannot allocate device memory while they run: code inside a
// CUDA-graph-driven real-time loop, a host that pre-reserves all device memory
// at start-up, or a plugin whose host application owns the allocator. For them
// the rotation vote can run with its scratch (the work-queue descriptor, the
// work counter, the accumulators and a packed copy of the target) in one
// file-scope device array instead of memory from cudaMalloc. Every GPU that
// loads this library holds that array until the process exits.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <climits>
#include <cstring>
#include <mutex>

#include "dses.h"
#include "kernels.cuh"

namespace dses {

extern std::atomic<long long> g_launches;

namespace {

// Largest target accepted by dses_vote_static (points).
constexpr int kStaticMaxTargets = 8192;

// Scratch layout (bytes): packed targets, then the descriptor, tile prefix,
// rotation prefix, work counter and accumulators.
constexpr size_t kOffY = 0;
constexpr size_t kOffDesc = kOffY + sizeof(float4) * kStaticMaxTargets;
constexpr size_t kOffTiles = kOffDesc + ((sizeof(PassDesc) + 255) / 256) * 256;
constexpr size_t kOffRots = kOffTiles + 256;
constexpr size_t kOffCounter = kOffRots + 256;
constexpr size_t kOffAcc = kOffCounter + 256;
constexpr size_t kScratchBytes = kOffAcc + 256;

static __device__ __align__(256) unsigned char g_vote_scratch[kScratchBytes];

// Host view: the array's device address per device, looked up once with that
// device current (the host symbol itself is not a device address). The cache
// lives as long as the process: a cudaDeviceReset of a device (which drops the
// context that address belongs to) leaves it stale, as dses.h states.
std::mutex g_addr_mu;
void* g_addr[64] = {nullptr};

// Packs xyz targets into the scratch and writes the launch descriptor and
// prefixes; zeroes the work counter and accumulators.
__global__ void static_setup_kernel(const float* __restrict__ xyz, int m, PassDesc d, int tiles, int n_rot) {
  float4* Y = reinterpret_cast<float4*>(g_vote_scratch + kOffY);
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x)
    Y[j] = make_float4(xyz[3 * j], xyz[3 * j + 1], xyz[3 * j + 2], 0.f);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *reinterpret_cast<PassDesc*>(g_vote_scratch + kOffDesc) = d;
    int* tp = reinterpret_cast<int*>(g_vote_scratch + kOffTiles);
    tp[0] = 0;
    tp[1] = tiles;
    int* rp = reinterpret_cast<int*>(g_vote_scratch + kOffRots);
    rp[0] = 0;
    rp[1] = n_rot;
    *reinterpret_cast<int*>(g_vote_scratch + kOffCounter) = 0;
    uint32_t* acc = reinterpret_cast<uint32_t*>(g_vote_scratch + kOffAcc);
    acc[0] = acc[1] = acc[2] = acc[3] = 0u;
  }
}

int gcd_i(int a, int b) { return b ? gcd_i(b, a % b) : a; }

}  // namespace
}  // namespace dses

using namespace dses;

extern "C" dses_status dses_vote_static(int device, void* cuda_stream, const float* src_dev, int64_t n_src,
                                        const float* tgt_dev, int64_t n_tgt, const float* rot_dev, int64_t n_rot,
                                        const dses_params* params, int32_t* kv_dev) {
  if (!src_dev || !tgt_dev || !rot_dev || !params || !kv_dev) return DSES_ERR_INVALID_ARG;
  if (n_src < 1 || n_src > (1 << 24) || n_rot < 1 || n_rot > (1LL << 31) - 1) return DSES_ERR_INVALID_ARG;
  if (n_tgt < 1 || n_tgt > kStaticMaxTargets) return DSES_ERR_INVALID_ARG;  // beyond the static scratch
  // one bin can collect every pair: its count (and V in kv_dev) must fit an int32
  if (n_src * n_tgt > INT32_MAX) return DSES_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(kv_dev) & 15u) != 0) return DSES_ERR_INVALID_ARG;
  if (device < 0 || device >= 64) return DSES_ERR_INVALID_ARG;
  const dses_params& P = *params;
  if (!(P.epsilon > 0) || !std::isfinite(P.epsilon)) return DSES_ERR_INVALID_ARG;
  const float delta = P.delta_t > 0 ? P.delta_t : P.epsilon;
  if (!std::isfinite(delta)) return DSES_ERR_INVALID_ARG;
  int lo[3], E[3];
  for (int a = 0; a < 3; ++a) {
    if (!(P.t_half[a] > 0) || !std::isfinite(P.t_half[a]) || !std::isfinite(P.t_center[a])) return DSES_ERR_INVALID_ARG;
    const double l = std::ceil(((double)P.t_center[a] - (double)P.t_half[a]) / (double)delta);
    const double h = std::floor(((double)P.t_center[a] + (double)P.t_half[a]) / (double)delta);
    if (h < l || l < -(1 << 20) || h > (1 << 20)) return DSES_ERR_INVALID_ARG;
    lo[a] = (int)l;
    E[a] = (int)(h - l + 1);
  }
  // histogram plan: 16-bit counters only where N * M cannot overflow them
  const bool u16 = n_src * n_tgt <= 65535 && (int64_t)E[0] * E[1] * E[2] * 4 > kHistBudget;
  const int64_t per_plane = (int64_t)E[1] * E[2] * (u16 ? 2 : 4);
  if (per_plane + 8 > kHistBudget) return DSES_ERR_INVALID_ARG;
  const int sx = (int)std::min<int64_t>(E[0], (kHistBudget - 8) / per_plane);
  const int64_t bins = (int64_t)sx * E[1] * E[2];
  const int hist_bytes = (int)(((u16 ? ((bins + 1) / 2) * 4 : bins * 4) + 15) & ~15LL);

  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) {
    cudaGetLastError();
    return DSES_ERR_CUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return DSES_ERR_INVALID_ARG;
  }
  dses_status st = DSES_OK;
  do {
    unsigned char* base = nullptr;
    {
      std::lock_guard<std::mutex> lk(g_addr_mu);
      if (!g_addr[device]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_vote_scratch) != cudaSuccess || !p) {
          cudaGetLastError();
          st = DSES_ERR_CUDA;
          break;
        }
        g_addr[device] = p;
      }
      base = static_cast<unsigned char*>(g_addr[device]);
    }
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int M = (int)n_tgt, N = (int)n_src;
    const int ppt = M <= 128 ? 1 : (M <= 512 ? 2 : 4);
    PassDesc d;
    std::memset(&d, 0, sizeof(d));
    d.X = src_dev;
    d.Y = reinterpret_cast<const float4*>(base + kOffY);
    d.Yv = d.Y;
    d.N = N;
    set_chunks(d, kSrcChunk * 16);
    d.M = M;
    d.rot = rot_dev;
    d.n_rot = (int)n_rot;
    d.inv_delta = 1.0f / delta;
    d.delta = delta;
    for (int a = 0; a < 3; ++a) {
      d.lo[a] = lo[a];
      d.E[a] = E[a];
      d.Ev[a] = E[a];
    }
    d.hs[0] = (uint32_t)(E[1] * E[2]);
    d.hs[1] = (uint32_t)E[2];
    d.slab_x = sx;
    d.n_slabs = (E[0] + sx - 1) / sx;
    d.hist_u16 = u16 ? 1 : 0;
    d.n_tchunks = (M + 32 * ppt - 1) / (32 * ppt);
    d.n_sgroups = 32 / gcd_i(d.n_tchunks, 32);
    d.kv = reinterpret_cast<int4*>(kv_dev);
    d.acc = reinterpret_cast<uint32_t*>(base + kOffAcc);
    const int tile = (int)std::max<int64_t>(1, std::min<int64_t>(16, n_rot / ((int64_t)sms * 8)));
    const int tiles = (int)((n_rot + tile - 1) / tile);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    g_launches.fetch_add(1, std::memory_order_relaxed);
    static_setup_kernel<<<(M + 255) / 256, 256, 0, s>>>(tgt_dev, M, d, tiles, (int)n_rot);
    if (cudaGetLastError() != cudaSuccess) {
      st = DSES_ERR_CUDA;
      break;
    }
    PassLaunch L;
    L.probs = reinterpret_cast<const PassDesc*>(base + kOffDesc);
    L.tile_prefix = reinterpret_cast<const int*>(base + kOffTiles);
    L.rot_prefix = reinterpret_cast<const int*>(base + kOffRots);
    L.n_probs = 1;
    L.tile_rot = tile;
    L.work_counter = reinterpret_cast<int*>(base + kOffCounter);
    L.hist_bytes = hist_bytes;
    L.src_bytes = kSrcChunk * 16;
    L.blk_bytes = 0;
    L.list_bytes = 0;
    L.padded = 0;
    if (launch_vote(L, ppt, 0, std::max(1, std::min(sms, tiles)), s) != cudaSuccess) {
      cudaGetLastError();
      st = DSES_ERR_CUDA;
      break;
    }
  } while (false);
  cudaSetDevice(prev);
  return st;
}
