// Device-side data structures and kernel launchers of the DSES library.
// Host code (engine.cu) fills these descriptors; the kernels in pass.cu and
// aux.cu read them. Nothing here is part of the public C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

namespace dses {

// Robust per-point error rho(d) of a nearest-target distance d (the norm of
// Eq. 1): 0 inlier indicator [d >= eps] (Eq. 3), 1 truncated L1 min(d, tau),
// 2 truncated L2 min(d, tau)^2, 3 Huber with knee h on min(d, tau), 4 d^p.
__device__ __forceinline__ float robust_rho(int metric, float d, float eps, float tau, float h, float p) {
  switch (metric) {
    case 0: return d < eps ? 0.f : 1.f;
    case 1: return fminf(d, tau);
    case 2: { const float e = fminf(d, tau); return e * e; }
    case 3: { const float e = fminf(d, tau); return e <= h ? 0.5f * e * e : h * (e - 0.5f * h); }
    default: return powf(d, p);
  }
}

// Threads of the rotation-pass CTA (one CTA per SM, 32 warps).
constexpr int kPassThreads = 1024;
// Source points staged per chunk in shared memory (a float4 each; the packed
// vote stages two, so half as many per chunk): 32 KB of staging.
constexpr int kSrcChunk = 2048;
// Target points per bounding-box group of the vote-ordered targets.
constexpr int kGroup = 32;
// Largest dynamic shared memory a CTA may request on sm_103a (227 KB).
constexpr int kMaxSmem = 232448;
// Static shared memory of the pass kernel (descriptor, reductions, per-warp
// culling thresholds) plus headroom.
constexpr int kPassStaticSmem = 2048 + 32 * 8 * 8 * 4;
// Paired culled vote: per warp, three lists of kPairedListCap shared addresses
// of kept sources' staged offsets (sources kept by the item's first group only,
// by its second only, by both), flushed at kPairedListFlush entries (a block
// of 32 sources adds at most 32, so the cap is the flush count + 32). Measured
// on the robot-like vote at N_side 12: flushing at 16 / 24 / 32 / 40 entries
// ran 393.9 / 392.0 / 390.6 / 390.1 ms (at 8: 397.1 against 394.4 at 16 in
// another run); 32 keeps at least 8 KB of staging beside a histogram at
// kHistBudget.
constexpr int kPairedListFlush = 32;
constexpr int kPairedListCap = kPairedListFlush + 32;
constexpr int kPairedListBytes = (kPassThreads / 32) * 3 * kPairedListCap * 4;
// Tiled staging of the paired culled vote: 8 sources per 192-byte tile, the
// pairs (c_x, c_x) of its sources at bytes 0-63, (c_y, c_y) at 64-127 and
// (c_z, c_z) at 128-191.
constexpr int kTileSources = 8;
constexpr int kTileBytes = 192;
static_assert(kTileBytes == 3 * 8 * kTileSources, "one 8-byte pair per axis and source");
// the list loop reads four entries as one 16-byte load from a list start,
// and a block of 32 sources may add 32 entries to a list holding up to
// kPairedListFlush - 1
static_assert(kPairedListCap % 4 == 0, "16-byte aligned lists");
static_assert(kPairedListCap >= kPairedListFlush - 1 + 32, "room for a block's pushes before the flush");
// Histogram budget: what is left after the source chunk and static storage.
constexpr int kHistBudget = kMaxSmem - kSrcChunk * 16 - kPassStaticSmem;

// Everything the rotation pass (vote + count kernels) needs for one problem.
struct PassDesc {
  // inputs (device)
  const float* X;        // N x 3 source points
  const int* Xperm;      // culled paths: the order the vote stages the sources in
                         // (compact runs of 32), or NULL for the input order
  const float4* Y;       // M target points (cell-sorted; .w unused), inlier count
  const float4* Yv;      // M target points in the vote's order (compact runs)
  const float4* gbox;    // per group of kGroup consecutive targets of Yv: min, max
  int n_groups;
  // culled paths: keep windows widen by this many lattice units (1e-3 plus
  // 2^-20 of the largest lattice coordinate of the target and the box: far
  // above the FP32 roundings of the staged offsets, w and the thresholds)
  float cull_margin;
  const float* rot;      // rotations of this pass, 9 floats each (row-major)
  int N, M;
  int n_rot;             // rotations in this pass
  int tile_rot;          // rotations per work item of this problem (0: the launch's tile_rot)
  uint32_t rot_base;     // global rotation index of rot[0]
  // translation lattice (Lemma 1 discretised): k = floor((y - R x)/delta + 1/2)
  float inv_delta, delta;
  int lo[3];             // lattice box lower corner
  int E[3];              // histogram layout extent per axis (odd; >= Ev)
  int Ev[3];             // lattice box extent per axis (bins beyond it are padding)
  uint32_t hs[2];        // layout strides in bins: per x-plane (>= E[1] hs[1]) and per
                         // y-row (>= E[2]); bin of (kx, ky, kz) = kx hs[0] + ky hs[1] + kz
  int slab_x;            // x-planes per histogram slab
  int n_slabs;
  int hist_u16;          // 1: two 16-bit counters per 32-bit word
  int hist_lanes;        // 1: 32-bit counters, one copy per lane: word bin * 32 + lane
  int chunk[3];          // sources staged per chunk: [0] plain (16 bytes each), [1]
                         // packed (32 bytes each), [2] tiled (paired culled vote: 24
                         // bytes each, whole tiles of 8); equal chunks that fit the staging
  int sparse;            // culled vote: 0 no, 1 32-point groups, 2 paired 64-point
                         // groups (gbox / n_groups hold that mode's group boxes)
  // vote work decomposition per rotation: items = n_tchunks x n_sgroups
  int n_tchunks;         // target chunks of 32 * P points
  int n_sgroups;         // source groups
  // inlier count of Eq. 3 through the target cell list (cell size >= epsilon)
  float eps2;
  const int* cell_start; // ncells + 1 prefix offsets into Y
  float cell_lo[3];
  float cell_inv;
  int cell_dim[3];
  // robust cost
  int fuse_score;        // 1: score every rotation inside the pass (grid path)
  int metric;            // dses_metric
  float eps, tau, huber_h, p_exp;
  const float* D;        // G^3 truncated distance grid
  const float4* D4;      // per voxel its (y, z) 2 x 2 corner block (see launch_dist_grid)
  int G;
  float glo[3], ginv_h[3], gcap;
  float grid_err;        // FP32 margin of the distance bounds from the grid
  // outputs, indexed by (global rotation index - out_base)
  uint32_t out_base;
  int4* kv;              // (kx, ky, kz, V)
  uint32_t* Mout;        // inlier count M
  float* cost;           // robust cost (fused path)
  // per-problem accumulators
  uint32_t* acc;         // [0] = M*, [1] = max V
  unsigned long long* best;  // argmin key (cost bits << 32 | rotation index)
  unsigned long long* votes_total;  // sum of all histogram counts (in-box pair votes)
};

struct PassLaunch {
  const PassDesc* probs;   // device array
  const int* tile_prefix;  // device, n_probs + 1 prefix sums of tiles
  const int* rot_prefix;   // device, n_probs + 1 prefix sums of rotations
  int n_probs;
  int tile_rot;            // rotations per work item
  int* work_counter;       // device, zeroed before the launch
  int hist_bytes;          // histogram bytes of shared memory (max over problems)
  int src_bytes;           // source staging bytes (a multiple of 32)
  int blk_bytes;           // culled launches: per 32-source block bounds of the staged
                           // offsets (8 floats each) after the staging; else 0
  int list_bytes;          // paired culled launches: the warps' lists of kept sources
                           // (kPairedListBytes) after the block bounds; else 0
  int padded;              // 1: some problem's layout is padded (E != Ev): the
                           // instance whose mode scan skips padding bins
};

// Hot path, kernel 1: vote -> mode (k*, V) per rotation (persistent, one CTA per SM).
// sparse: 0 dense; 1 the instance that also carries the culled path (points
// per thread 1, 2, 4); 2 the paired culled path (2, 4). Problems of the launch
// with d.sparse set must use that mode; dense launches take 1, 2, 4 or 8.
cudaError_t launch_vote(const PassLaunch& L, int points_per_thread, int sparse, int grid_ctas, cudaStream_t s);
// Kernel 2: inlier count M at t* and, on the fused path, grid score + argmin.
cudaError_t launch_count(const PassLaunch& L, int total_rot, cudaStream_t s);
int pass_smem_bytes(int hist_bytes, int src_bytes);
// Shared memory of a rotation-pass launch past the histogram: the source
// staging (32 bytes per source of the largest problem, and for a paired
// launch at least its whole 192-byte tiles, as far as shared memory allows),
// for a culled launch with block bounds the bounds of every block of 32
// staged sources (32 bytes each, sized for the plain layout's largest chunk),
// and for a paired culled launch the warps' kept-source lists.
inline void pass_staging(int hist_bytes, int n_src_max, bool culled, bool paired, int* src_bytes, int* blk_bytes,
                         int* list_bytes) {
  const int list = paired ? kPairedListBytes : 0;
  // what shared memory leaves for the staging (and the block bounds): at
  // least kSrcChunk * 16 - list, since the histogram keeps to kHistBudget
  const int avail = (kMaxSmem - kPassStaticSmem - hist_bytes - list) & ~31;
  // a tile holds 8 sources in 192 bytes, 24 per source, but a partial tile
  // of r sources still spans 128 + 8 r bytes (its z pairs start at byte
  // 128): more than 32 per source for 1-5, 9 and 10 sources
  long long need = 32LL * n_src_max;
  if (paired) need = std::max<long long>(need, (long long)((n_src_max + kTileSources - 1) / kTileSources) * kTileBytes);
  int src = (int)std::min<long long>(need, avail);
  int blk = 0;
  if (culled) {
    blk = ((src / 16 + 31) / 32) * 32;
    if (src + blk > avail) {
      src = ((avail - 32) / 17 * 16) & ~31;
      blk = ((src / 16 + 31) / 32) * 32;
    }
  }
  *src_bytes = src;
  *blk_bytes = blk;
  *list_bytes = list;
}
// Equal chunks of the problem's sources that fit src_bytes of staging, plain,
// packed and tiled (d.chunk).
inline void set_chunks(PassDesc& d, int src_bytes) {
  for (int k = 0; k < 3; ++k) {
    const int cap = k == 2 ? std::max(1, src_bytes / kTileBytes) * kTileSources : src_bytes / (k ? 32 : 16);
    const int n = (d.N + cap - 1) / cap;
    d.chunk[k] = (d.N + n - 1) / n;
  }
}

// --- rotation grids (FP64 arithmetic, FP32 output) -------------------------
cudaError_t launch_hopf_grid(int n, float* out, cudaStream_t s);
// Euler boxes around `count` centres given as FP32 matrices (centres[c*9]).
cudaError_t launch_euler_boxes(const float* centres, int count, int K, double delta_r, float* out, cudaStream_t s);
// Euler boxes around Hopf-grid centres named by the low 32 bits of sorted keys
// (recomputed in FP64); all-ones padding keys repeat the previous centre.
cudaError_t launch_euler_boxes_hopf(int n, const unsigned long long* keys, int count, int K, double delta_r,
                                    float* out, cudaStream_t s);
// Euler boxes around centres picked from an FP32 rotation array by key.
cudaError_t launch_euler_boxes_keyed(const float* rot, const unsigned long long* keys, int count, int K,
                                     double delta_r, float* out, cudaStream_t s);
// Euler box around one FP64 centre held in device memory.
cudaError_t launch_euler_box_single(const double* R0_dev, int K, double delta_r, float* out, cudaStream_t s);

// --- target preprocessing ---------------------------------------------------
cudaError_t launch_pack_points(const float* xyz, int m, float4* out, cudaStream_t s);
// D: G^3 truncated distances (x-major); D4[v] for voxel v = (a, b, c) holds
// D at (a, b, c), (a, b, c+1), (a, b+1, c), (a, b+1, c+1) (indices clamped at
// G - 1), so a trilinear lookup reads its 8 corners as two 16-byte loads.
cudaError_t launch_dist_grid(const float4* Y, int m, int G, const float* lo, const float* h, float cap, float* D,
                             float4* D4, cudaStream_t s);
// cell list: counts -> prefix -> scatter. counts: ncells ints; scratch: ncells + m ints.
cudaError_t launch_cell_list(const float4* Y, int m, const float* cell_lo, float cell_inv, const int* dim,
                             int* counts, int* cell_start, int* scratch, float4* sorted, cudaStream_t s);

// --- candidate stage ----------------------------------------------------------
struct ScoreDesc {
  const float* X;
  const float4* Y;
  const float* rot;       // rotations of the pass (indexed by global index - rot_base)
  int N, M;
  float delta;
  int metric;
  float eps, tau, huber_h, p_exp;
  const float* D;
  const float4* D4;
  int G;
  float glo[3], ginv_h[3], gcap;
  const int4* kv;         // per-rotation outputs, indexed by global index - out_base
  const uint32_t* Mout;
  float* cost;
  uint32_t rot_base;
  uint32_t out_base;
};

// candidates (output slots, i.e. global index - out_base) with 1000 M >= q_milli M*
cudaError_t launch_select_q(const uint32_t* Mout, uint32_t first, int n, const uint32_t* acc, int q_milli,
                            uint32_t* cand, uint32_t* n_cand, cudaStream_t s);
// keys (0xffffffff - M) << 32 | global index for slots [first, first + n)
cudaError_t launch_keys_from_M(const uint32_t* Mout, uint32_t first, int n, uint32_t out_base,
                               unsigned long long* keys, cudaStream_t s);
// keys cost_bits << 32 | global index over a candidate list (cand == NULL:
// every slot of [0, n_max))
cudaError_t launch_keys_from_cost(const float* cost, const uint32_t* cand, const uint32_t* n_cand, int n_max,
                                  uint32_t out_base, unsigned long long* keys, cudaStream_t s);
// the k smallest of n keys (n read from n_dev when not NULL, else n_max), ascending into out[k];
// scratch holds 2 * ceil(n_max / 4096) * k keys
cudaError_t launch_k_smallest(const unsigned long long* keys, int n_max, const uint32_t* n_dev, int k,
                              unsigned long long* scratch, unsigned long long* out, cudaStream_t s);
size_t k_smallest_scratch(int n_max, int k);
// candidate slots from keys (global index - out_base), skipping padding keys
cudaError_t launch_cand_from_keys(const unsigned long long* keys, int k, uint32_t out_base, uint32_t* cand,
                                  uint32_t* n_cand, cudaStream_t s);
cudaError_t launch_score_grid(const ScoreDesc& d, const uint32_t* cand, const uint32_t* n_cand, int n_max,
                              cudaStream_t s);
cudaError_t launch_score_brute(const ScoreDesc& d, const uint32_t* cand, const uint32_t* n_cand, int n_max,
                               cudaStream_t s);
// argmin over candidates of (cost bits << 32 | global index); INLIER metric uses N - M
cudaError_t launch_argmin(float* cost, const uint32_t* Mout, int N, int metric, const uint32_t* cand,
                          const uint32_t* n_cand, int n_max, uint32_t out_base, unsigned long long* best,
                          cudaStream_t s);

struct FinalDesc {
  const unsigned long long* best;
  const uint32_t* acc;    // [1]: max V of the first pass, [3]: of the second pass
  const int4* kv;         // indexed by global index - out_base
  const uint32_t* Mout;
  const float* rot;       // first-pass rotations (global index < n_first)
  const float* rot_fine;  // second-pass rotations (global index - n_first)
  uint32_t n_first;
  uint32_t out_base;
  float delta;
  void* result;           // device dses_result
};
cudaError_t launch_finalize(const FinalDesc* d_dev, int count, cudaStream_t s);

// One step of the sub-voxel translation refinement at (R, t): the mean of
// y_nn(i) - R x_i over source points whose nearest target (cell-list search)
// is closer than epsilon. t (3 doubles, device) is read and replaced by that
// mean (kept when no pair qualifies); acc (4 doubles, device) must be zero and
// is left zero; *n_out (device) receives the number of pairs.
struct RefineDesc {
  const float* X;         // source, N x 3
  int N;
  const float4* Y;        // target in cell order
  const int* cell_start;  // cells + 1
  float cell_lo[3];
  float cell_inv;
  int cell_dim[3];
  float eps2;
  float R[9];
  double* t;
  double* acc;
};
cudaError_t launch_refine_step(const RefineDesc& d, uint32_t* n_out, cudaStream_t s);

// Algorithm 1 over a rotation list and the lattice box: cost[r n_t + t] and
// count[r n_t + t] (inliers of Eq. 3) for every pair, atomicMin of
// (cost bits << 32 | r n_t + t) into *best (initialised to ~0 by the caller).
// t = ((kx - lo_x) E_y + (ky - lo_y)) E_z + (kz - lo_z). The target (M float4)
// is staged in shared memory: M <= kExhaustiveMaxTargets.
constexpr int kExhaustiveMaxTargets = 12288;
struct ExhaustiveDesc {
  const float* X;     // source, N x 3
  int N;
  const float4* Y;    // target, M points
  int M;
  const float* rot;   // n_rot x 9
  int n_rot;
  int lo[3], E[3];
  int n_t;            // E_x E_y E_z
  float delta;
  int metric;
  float eps, tau, huber_h, p_exp;
  float* cost;
  uint32_t* count;
  unsigned long long* best;
};
cudaError_t launch_exhaustive(const ExhaustiveDesc& d, cudaStream_t s);

// Kernels launched by this library since it was loaded (all launch sites count).
long long kernel_launch_count();

cudaError_t launch_fill_u32(uint32_t* p, uint32_t v, size_t n, cudaStream_t s);
cudaError_t launch_fill_f32(float* p, float v, size_t n, cudaStream_t s);
cudaError_t launch_fill_u64(unsigned long long* p, unsigned long long v, size_t n, cudaStream_t s);

}  // namespace dses
