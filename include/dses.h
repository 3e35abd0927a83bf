/*
 * dses.h - C ABI of the B300 (sm_103a) implementation of Direct Semi-Exhaustive
 * Search (DSES) for partial-to-full point-cloud registration, arXiv 2502.00115.
 *
 * The method (Section IV-B, Algorithm 2): for every rotation R of a rotation
 * grid, the translation that maximises inliers is the mode of the rotated
 * pairwise differences y_j - R x_i on a delta_t lattice (Lemma 1, Eq. 5); the
 * inlier count M of Eq. 3 is taken at that translation; candidates whose M is
 * at least q times the best M* are scored under a robust distance metric (the
 * norm p of Eq. 1: Sum_i rho(min_j ||y_j - R x_i - t||)); the lowest-cost
 * candidate is returned.
 *
 * Conventions shared by every entry point:
 *  - Points are FP32, xyz interleaved, row-major (n x 3). A pointer is a host
 *    pointer unless the call's "is_device" flag says it is a device pointer of
 *    the context's device; device pointers are read in the order of the
 *    context's stream.
 *  - The caller owns every buffer it passes; no call keeps a caller pointer
 *    after it returns (dses_submit copies the source cloud before returning).
 *  - Targets belong to the library from dses_create_target until
 *    dses_destroy_target.
 *  - No C++ exception crosses this boundary. Every call returns a dses_status;
 *    dses_last_error(ctx) gives a one-line description of the last failure on
 *    that context (overwritten by the next failure).
 *  - A context serialises its calls with a mutex; dses_poll may be called from
 *    any thread.
 *  - A CUDA error inside a call is reported as DSES_ERR_CUDA; after a sticky
 *    CUDA error the context must be destroyed and recreated.
 */
#ifndef DSES_H_
#define DSES_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dses_ctx dses_ctx;
typedef struct dses_target dses_target;

typedef enum {
  DSES_OK = 0,
  DSES_NOT_READY = 1,            /* dses_poll: the request is still running */
  DSES_ERR_INVALID_ARG = -1,     /* bad pointer, size, parameter or handle */
  DSES_ERR_OOM = -2,             /* device or pinned-host allocation failed */
  DSES_ERR_CUDA = -3,            /* a CUDA runtime call failed */
  DSES_ERR_QUEUE_FULL = -4,      /* dses_submit: the request queue is at capacity */
  DSES_ERR_TIMEOUT = -5,         /* a bounded wait ran out */
  DSES_ERR_NO_CANDIDATE = -6,    /* no point pair voted inside the translation box */
  DSES_ERR_UNKNOWN_TICKET = -7,  /* dses_poll: ticket never issued or already collected */
  DSES_ERR_EXCHANGE = -8         /* dses_register_sharded: the all-gather callback failed */
} dses_status;

/* Robust per-point error rho(d) on the nearest-target distance d (the norm p of
 * Eq. 1 and the ERROR of Algorithm 2; Section IV-B names the truncated L1):
 *   INLIER    rho = [d >= epsilon]           (cost = N - M, the saturated L0 of Eq. 3)
 *   TRUNC_L1  rho = min(d, tau)
 *   TRUNC_L2  rho = min(d, tau)^2
 *   HUBER     e = min(d, tau); rho = e^2/2 if e <= h else h (e - h/2)
 *   LP        rho = d^p, p in (0, 1]                                        */
typedef enum {
  DSES_METRIC_INLIER = 0,
  DSES_METRIC_TRUNC_L1 = 1,
  DSES_METRIC_TRUNC_L2 = 2,
  DSES_METRIC_HUBER = 3,
  DSES_METRIC_LP = 4
} dses_metric;

typedef enum {
  /* Dense SO(3) grid of 72 n^3 rotations: Hopf coordinates from the HEALPix
   * RING pixel centres at N_side = n (theta, phi) and psi_k = 2 pi (k + 1/2)/(6n);
   * quaternion (cos(t/2)cos(s/2), cos(t/2)sin(s/2), sin(t/2)cos(f+s/2),
   * sin(t/2)sin(f+s/2)); index = pixel * 6n + k.                            */
  DSES_GRID_HOPF = 0,
  /* Euler box of Algorithm 2's rotation loops: R = R0 Rz(a) Ry(b) Rx(c), each
   * angle in {-K, ..., K} * delta_r, index ((a (2K+1)) + b)(2K+1) + c.       */
  DSES_GRID_EULER_BOX = 1,
  /* Caller-supplied FP32 row-major 3x3 matrices (host memory, n_explicit x 9). */
  DSES_GRID_EXPLICIT = 2
} dses_grid_kind;

typedef enum {
  DSES_NN_GRID = 0,  /* trilinear lookup in the target's truncated distance grid */
  DSES_NN_BRUTE = 1  /* exact brute-force nearest neighbour over all target points */
} dses_nn_mode;

typedef struct {
  int32_t kind;             /* dses_grid_kind */
  int32_t hopf_n;           /* HOPF: N_side >= 1 */
  int32_t K;                /* EULER_BOX: half-size >= 0 */
  double delta_r;           /* EULER_BOX: angular step, radians */
  double R0[9];             /* EULER_BOX: centre rotation, row-major */
  const float* explicit_R;  /* EXPLICIT: host pointer, n_explicit x 9 */
  int64_t n_explicit;       /* EXPLICIT: number of rotations */
} dses_rotation_grid;

typedef struct {
  int32_t metric;           /* dses_metric */
  float epsilon;            /* inlier threshold of Eq. 3 (> 0) */
  float delta_t;            /* lattice step of the translation mode; 0 => epsilon */
  float tau;                /* truncation of TRUNC_L1/TRUNC_L2/HUBER; 0 => 2 epsilon */
  float huber_h;            /* Huber knee; 0 => epsilon */
  float p;                  /* LP exponent in (0, 1] */
  float t_center[3];        /* translation search range [c - s, c + s] per axis ... */
  float t_half[3];          /* ... (s > 0); the lattice points k delta_t inside it */
  int32_t q_milli;          /* candidate filter 1000 M >= q_milli M*, 0..1000 (0: all) */
  int32_t top_k;            /* > 0: candidates are the top_k by (M desc, index asc) */
  int32_t nn_mode;          /* dses_nn_mode */
  int32_t refine_top_k;     /* > 0: second pass on Euler boxes around this many best */
  int32_t refine_K;         /* Euler box half-size of the second pass */
  double refine_delta_r;    /* Euler box step of the second pass, radians */
} dses_params;

typedef struct {
  float R[9];               /* best rotation, row-major: y ~ R x + t */
  float t[3];               /* its translation t* = k* delta_t */
  int64_t rot_index;        /* index in the grid; a second-pass rotation has index
                               n_grid + c (2K+1)^3 + local, c = rank of its centre */
  uint32_t inliers;         /* M at the best rotation (Eq. 3) */
  uint32_t votes;           /* V: the mode's frequency at the best rotation */
  float cost;               /* Sum_i rho(d_i) at the best pose */
  int32_t status;           /* dses_status of this registration */
} dses_result;

typedef struct {
  const dses_target* target; /* resident target (full model) Y */
  const float* src;          /* source (partial observation) X, n_src x 3 */
  int64_t n_src;             /* N >= 1 */
  int32_t src_is_device;     /* 1: src is a device pointer */
  dses_rotation_grid grid;
  dses_params params;
} dses_problem;

/* Context on `device`. cuda_stream: a cudaStream_t to run on (NULL: the context
 * creates its own non-blocking stream). Errors: INVALID_ARG (bad device or out
 * NULL), CUDA. */
dses_status dses_create(int device, void* cuda_stream, dses_ctx** out);

/* Stops the serving worker, frees every target and buffer of the context. */
dses_status dses_destroy(dses_ctx* ctx);

/* Resident target (Section III's reference cloud Y, the full model): copies the
 * m x 3 points to the device and builds its truncated distance grid of
 * grid_res^3 FP32 voxels (grid_res in [8, 512]; 0 => 128), truncated at
 * grid_cap (> 0; the TRUNC/HUBER metrics need grid_cap >= tau). Voxel size per
 * axis h = (extent + 2 cap)/(grid_res - 2), origin min - cap - h; voxel centre
 * values are min(cap, exact nearest-target distance). Device memory: 20
 * bytes per voxel (the grid, and a copy holding each voxel's 2 x 2 corner
 * block for the lookups: 40 MB at 128^3, 2.7 GB at 512^3) plus the points.
 * Errors: INVALID_ARG (m < 1, non-finite point, bad size), OOM, CUDA. */
dses_status dses_create_target(dses_ctx* ctx, const float* xyz, int64_t m, int32_t ptr_is_device,
                               float grid_cap, int32_t grid_res, dses_target** out);

/* Frees a target. INVALID_ARG while a submitted request still uses it. */
dses_status dses_destroy_target(dses_ctx* ctx, dses_target* target);

/* One registration (Algorithm 2), blocking until the result is written to
 * *out (host memory). Errors: INVALID_ARG, OOM, CUDA, NO_CANDIDATE (the result
 * is still filled, with votes = 0). */
dses_status dses_register(dses_ctx* ctx, const dses_problem* problem, dses_result* out);

/* n registrations run as one persistent launch over a (problem, rotation-tile)
 * work queue; out[i] (host) receives problem i's result. Each result equals the
 * result of dses_register on the same problem. Returns the first non-OK
 * per-problem status, or OK. */
dses_status dses_register_batch(dses_ctx* ctx, const dses_problem* problems, int32_t n, dses_result* out);

/* Rotation sharding of one registration (Algorithm 2 treats every rotation of
 * the grid on its own): shard `rank` of `world` takes the contiguous range
 * [begin, end) of a grid of n_rot rotations in index order, begin =
 * floor(n_rot rank / world), end = floor(n_rot (rank + 1) / world). Host
 * only. INVALID_ARG for a NULL pointer, n_rot < 0, world < 1 or rank outside
 * [0, world). */
dses_status dses_shard_range(int64_t n_rot, int32_t rank, int32_t world, int64_t* begin, int64_t* end);

/* Registers shard `rank` of `world` of the problem's grid (the range of
 * dses_shard_range) on this context's GPU, blocking, with the same rotations
 * (FP32 values, the device grid sliced in place) as the whole grid;
 * out->rot_index is the rotation's index in the whole grid. Every rotation of
 * the range is scored, so combining the shards (dses_combine_results) gives
 * dses_register's result only when every rotation is a candidate: q_milli,
 * top_k and refine_top_k must be 0 (INVALID_ARG otherwise: a q filter, top-k
 * or second pass across shards needs the global M* or the K best keys first,
 * which dses_register_sharded exchanges). A shard with no rotations (world
 * above the grid size) returns NO_CANDIDATE with rot_index = -1. Errors as
 * dses_register. */
dses_status dses_register_shard(dses_ctx* ctx, const dses_problem* problem, int32_t rank, int32_t world,
                                dses_result* out);

/* The result of a sharded registration from its n shards' results (any
 * order, each from dses_register_shard): the lexicographic minimum of (cost,
 * rotation index), the order of the kernels' argmin (the last step of
 * Algorithm 2); status OK when any shard voted inside the translation box,
 * else NO_CANDIDATE (rot_index = -1 when no shard had a candidate). Host
 * only: results travel between processes as plain structs (an all-gather).
 * INVALID_ARG for n < 1, a NULL pointer or a part with another error. */
dses_status dses_combine_results(const dses_result* parts, int32_t n, dses_result* out);

/* All-gather used by dses_register_sharded: every shard passes `bytes` bytes
 * in `send`; `recv` (world * bytes, provided by the library) receives shard
 * r's bytes at offset r * bytes. Returns 0 on success, anything else on
 * failure. Called from the thread that called dses_register_sharded. */
typedef int32_t (*dses_allgather_fn)(void* user, const void* send, int64_t bytes, void* recv);

/* One registration sharded over `world` processes (one GPU each) by rotation
 * ranges, with every step of Algorithm 2: shard `rank` runs the ranges
 * dses_shard_range gives it of the grid and of the second pass, and the
 * shards meet, through `allgather`, only where Algorithm 2 reduces over all
 * rotations: the best inlier count M* before the q filter (4 bytes per
 * shard), the top_k keys (M desc, index asc; 8 top_k bytes), the
 * refine_top_k best first-pass candidates by (cost, index) that centre the
 * second pass's Euler boxes (8 refine_top_k bytes), the second pass's own M*
 * or top_k keys, and the shards' results (one dses_result each). Every shard
 * receives the combined result, equal to dses_register's on the whole
 * problem. Every shard must make the call with the same problem and world;
 * the callback is called the same number of times on every shard, with the
 * same sizes. A shard that fails before an exchange leaves the others waiting
 * in their callbacks: give the collective behind it a timeout. Blocking.
 * Errors: INVALID_ARG (NULL argument, bad rank or world, bad problem),
 * EXCHANGE (the callback returned non-zero), others as dses_register. */
dses_status dses_register_sharded(dses_ctx* ctx, const dses_problem* problem, int32_t rank, int32_t world,
                                  dses_allgather_fn allgather, void* user, dses_result* out);

/* Asynchronous registration: copies the problem (and the source cloud) and
 * queues it for the serving worker, which admits requests when device memory
 * and batch slots free up and runs admitted requests together (continuous
 * batching). *ticket identifies the request. Errors: INVALID_ARG, QUEUE_FULL. */
dses_status dses_submit(dses_ctx* ctx, const dses_problem* problem, uint64_t* ticket);

/* DSES_NOT_READY while the request runs; otherwise copies the result to *out,
 * forgets the ticket and returns the registration's status. UNKNOWN_TICKET for
 * a ticket never issued or already collected. */
dses_status dses_poll(dses_ctx* ctx, uint64_t ticket, dses_result* out);

/* Test hook: runs the registration and copies per-rotation intermediates to
 * host arrays of length n_rot (grid size, plus the second pass if any): k_star
 * (n_rot x 3, lattice index of t*), votes (V), inliers (M) and cost (NaN for a
 * rotation that was not a candidate). Any output pointer may be NULL. out
 * (optional) receives the result. */
dses_status dses_debug_per_rotation(dses_ctx* ctx, const dses_problem* problem, int32_t* k_star,
                                    uint32_t* votes, uint32_t* inliers, float* cost, dses_result* out);

/* Test hook, batched: the n problems run as dses_register_batch runs them (one
 * persistent launch over their (problem, rotation-tile) work queue, without
 * graph replay); problem b's per-rotation intermediates go to k_star[b],
 * votes[b], inliers[b] and cost[b] (host arrays of that problem's n_rot
 * entries, as dses_debug_per_rotation writes them) and its result to out[b].
 * Any of the four pointer arrays, or any entry of one, may be NULL. */
dses_status dses_debug_per_rotation_batch(dses_ctx* ctx, const dses_problem* problems, int32_t n,
                                          int32_t* const* k_star, uint32_t* const* votes,
                                          uint32_t* const* inliers, float* const* cost, dses_result* out);

/* Builds a rotation grid on the device and copies it to out_R (host,
 * capacity x 9 floats). *count receives the grid size; INVALID_ARG if it
 * exceeds capacity (out_R may be NULL to query the size). */
dses_status dses_rotation_grid_build(dses_ctx* ctx, const dses_rotation_grid* grid, float* out_R,
                                     int64_t capacity, int64_t* count);

/* Copies a target's distance grid (res^3 floats, index (a res + b) res + c)
 * and its geometry to host memory. D may be NULL to query res. */
dses_status dses_target_distance_grid(dses_ctx* ctx, const dses_target* target, float* D, float lo[3],
                                      float h[3], int32_t* res, float* cap);

/* Sub-voxel translation refinement (a step after Algorithm 2, which returns
 * the voxel centre t* = k* delta_t, up to (sqrt 3 / 2) delta_t from the
 * optimum). At the pose (R, t) every source point is paired with its nearest
 * target point and the pair is kept when that distance is below epsilon (the
 * inlier test of Eq. 3); the translation minimising the summed squared
 * residual of the kept pairs is their mean of y_nn(i) - R x_i, which replaces
 * t. `iterations` (1..64) such steps run, each re-pairing at the new t. src:
 * n_src x 3 FP32 (host, or a device pointer of the context's device with
 * src_is_device = 1). R (row-major 3x3, y ~ R x + t), t and t_out (3 floats)
 * are host memory; t_out may alias t. *n_inliers (may be NULL) receives the
 * number of pairs kept in the last step; with none kept t is left as it was.
 * Blocking. Errors: INVALID_ARG (NULL or non-finite input, epsilon <= 0,
 * iterations out of range, a target of another context), OOM, CUDA. */
dses_status dses_refine_translation(dses_ctx* ctx, const dses_target* target, const float* src, int64_t n_src,
                                    int32_t src_is_device, const float R[9], const float t[3], float epsilon,
                                    int32_t iterations, float t_out[3], uint32_t* n_inliers);

/* Algorithm 1 (pure exhaustive search), the validator of Algorithm 2 on small
 * problems: for every rotation of problem->grid and every lattice translation
 * k delta_t of the params' translation box, the error
 *   e(R, t) = sum_i rho(min_j ||y_j - R x_i - t||)
 * with exact nearest neighbours (nn_mode, q_milli, top_k and the refinement
 * fields are ignored). out receives the pose of the smallest error (the first
 * in index order on ties): R, t = k delta_t, rot_index, cost = e, inliers =
 * M of Eq. 3 at that pose, votes = 0. cost_out (host, may be NULL) receives
 * every e at [r * n_t + t], t = ((kx - lo_x) E_y + (ky - lo_y)) E_z +
 * (kz - lo_z) over the box's lattice extents E, and needs cost_capacity >=
 * n_rot * n_t. Work is n_rot * n_t * N * M distances: target m <= 12288 and
 * n_rot * n_t <= 2^28 (else INVALID_ARG). Blocking. Errors: as dses_register. */
dses_status dses_exhaustive_search(dses_ctx* ctx, const dses_problem* problem, float* cost_out,
                                   int64_t cost_capacity, dses_result* out);

/* Tuning and engine options (key = value). Keys:
 *   "hist_mode"            0 auto, 1 force 32-bit counters, 2 force packed 16-bit,
 *                          3 lane-private 32-bit counters (a copy of every bin
 *                          per lane, 128 bytes per bin; never chosen by 0; they
 *                          take the scalar dense or the 32-point culled vote)
 *   "hist_budget_bytes"    shared-memory bytes for the vote histogram (slabs below it)
 *   "points_per_thread"    0 auto, or 1, 2, 4, 8 target points held per lane
 *                          (a problem on the culled vote uses 4 for 8)
 *   "fuse_score"           1 (default) score inside the rotation pass when every
 *                          rotation is a candidate; 0 always score in a second kernel
 *   "tile_rotations"       rotations per work item of the persistent launch (0 auto)
 *   "autotune"             1 (default): time the vote's launch shapes once per
 *                          problem-size bucket (points per thread 1/2/4/8, then
 *                          rotations per work item 1/2/4/8/16 for that shape) on an
 *                          even-stride sample of the problem's own rotations; 0:
 *                          fixed heuristics. Results do not depend on the shape.
 *                          The serving worker never runs trials (they would stall
 *                          the requests in flight): a bucket first seen there takes
 *                          the heuristic shape until a blocking call tunes it.
 *   "use_graphs"           1 (default) replay repeated batches through CUDA graphs
 *   "serve_max_batch"      requests the serving worker runs together
 *   "serve_queue_cap"      submitted requests waiting for admission
 *   "serve_mem_budget"     device bytes the serving worker may hold for requests
 *   "serve_tile_rotations" most rotations one request takes per serving iteration
 *   "serve_iter_pairs"     pair votes per serving iteration (requests in arrival
 *                          order fill it; default 1.5e11, ~100 ms of vote work:
 *                          about one request of the serving workload)
 *   "vote_sparse"          0 auto, 1 dense vote, 2 cull (source, 32-point target
 *                          group) pairs outside the translation window (pays for
 *                          small boxes), 3 the same with 64-point groups voted as
 *                          packed pairs (pays when the window spans many groups;
 *                          with lane-private counters the 32-point form is used)
 *   "record_timing"        1: time every rotation pass with CUDA events on the
 *                          context's stream
 *   "target_order"         the vote's order of a target's points, fixed at
 *                          dses_create_target: 0 (default) recursive bisection
 *                          along the longest side of the bounding box, cut at
 *                          multiples of 64 points (compact culling groups); 1
 *                          Morton order. Results do not depend on it.
 *   "hist_strides"         1 (default): the vote histogram's row and plane strides
 *                          are padded past the box extents where that spreads
 *                          neighbouring lattice bins over more shared-memory banks
 *                          without costing a histogram slab or a source chunk; 0:
 *                          compact strides. Results do not depend on it.
 *   "fail_next_allocs"     test hook: the next this-many registrations (blocking or
 *                          served) fail at their scratch allocation with
 *                          DSES_ERR_OOM, as if the device allocator had refused,
 *                          without touching the device; the context stays usable
 *   "serve_max_active"     most requests the serving worker has held admitted at
 *                          once (set to 0 to reset; no other value)
 *   "serve_busy_ns"        summed device time of the serving worker's iterations, from
 *                          events at each iteration's first and last queued work
 *                          (set to 0 to reset)
 *   "serve_iterations"     serving iterations retired (set to 0 to reset)
 *   "last_pass_ns"         (read-only) summed duration of the vote kernels of the
 *                          last blocking call, in nanoseconds
 *   "last_count_ns"        (read-only) the same for its inlier-count / score kernels
 *   "last_pass_launches"   (read-only) how many rotation passes that call made
 *   "last_votes_total"     (read-only) histogram increments (pairs voting inside
 *                          the translation box) of the last blocking call
 *   "last_vote_sparse"     (read-only) how many problems of the last blocking call
 *                          ran the culled (windowed) vote
 *   "last_vote_paired"     (read-only) ... of which its 64-point-group form
 *   "last_p_mask"          (read-only) points-per-thread shapes the last pipeline run
 *                          launched its rotation passes with (bit P set for each)
 *   "last_tile_max"        (read-only) the largest rotations per work item among them
 *   "graphs_cached"        (read-only) captured CUDA graphs held by the context
 *                          (dses_destroy_target drops those that read the target)
 *   "kernel_launches"      (read-only) kernels this library has launched in the
 *                          process so far (all contexts)
 * INVALID_ARG for an unknown key or a value out of range. */
dses_status dses_set_option(dses_ctx* ctx, const char* key, int64_t value);
dses_status dses_get_option(dses_ctx* ctx, const char* key, int64_t* value);

/* Rotation vote without any device allocation (the paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc while they
 * run, e.g. a real-time loop driven by pre-built CUDA graphs, a host that
 * reserves all device memory at start-up, or a plugin whose application owns
 * the allocator). For every rotation it computes what dses_debug_per_rotation
 * reports as k_star and votes: the lattice index k* of the translation mode
 * and its frequency V. All inputs and outputs are device pointers of `device`
 * owned by the caller: src_dev (n_src x 3), tgt_dev (n_tgt x 3), rot_dev
 * (n_rot x 9 row-major FP32 rotations), kv_dev (n_rot x 4 int32: kx, ky, kz, V;
 * 16-byte aligned). Only params->epsilon, delta_t, t_center and t_half are read.
 * Work is queued on cuda_stream (NULL: the legacy default stream); outputs are
 * valid once that stream has reached this point. Scratch lives in one static
 * device array of about 129 KB per GPU (held until exit), so n_tgt is limited to
 * 8192 points (larger: INVALID_ARG), and n_src * n_tgt to 2^31 - 1 (a bin may
 * collect every pair and V is an int32). The first call on a device looks up
 * the array's device address with that device made current, keeps it for the
 * life of the process, then restores the caller's current device; make that
 * first call before any stream capture. A cudaDeviceReset of that device
 * invalidates the kept address: do not call this entry point on the device
 * after resetting it.
 * Calls share the array: calls that overlap on the GPU (other streams, other
 * host threads) race and must be serialised by the caller. Each call clears
 * the counters it needs. Errors: INVALID_ARG, CUDA. */
dses_status dses_vote_static(int device, void* cuda_stream, const float* src_dev, int64_t n_src,
                             const float* tgt_dev, int64_t n_tgt, const float* rot_dev, int64_t n_rot,
                             const dses_params* params, int32_t* kv_dev);

/* Last error text of the context (empty string if none; never NULL). */
const char* dses_last_error(dses_ctx* ctx);

/* Static name of a status code. */
const char* dses_status_string(dses_status status);

#ifdef __cplusplus
}
#endif

#endif /* DSES_H_ */
