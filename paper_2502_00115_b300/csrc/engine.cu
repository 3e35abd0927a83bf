// Host side of the DSES library: contexts, resident targets, the launch
// planner, the single / batched registration pipeline, the serving worker and
// the C ABI declared in include/dses.h.
//
// Pipeline of one registration (Algorithm 2):
//   rotation grid (cached per Hopf resolution, or built per call)
//   -> rotation pass over every rotation (vote, mode, inlier count and, when
//      every rotation is a candidate, the fused grid score + argmin)
//   -> otherwise: candidate selection (q filter or top-k), scoring of the
//      candidates (distance-grid lookup or exact brute-force nearest
//      neighbour), argmin
//   -> optional second pass on Euler boxes around the best candidates
//   -> finaliser writes the dses_result on the device, one copy to the host.
// Everything runs asynchronously on the context's stream; a call synchronises
// once, at the end.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <limits>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "bounds.h"
#include "dses.h"
#include "exchange.h"
#include "kernels.cuh"
#include "strides.h"

using namespace dses;

namespace {

struct Error {
  dses_status code;
  std::string msg;
};

#define CK(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) {                                                                  \
      cudaGetLastError(); /* a non-sticky error must not poison the next launch check */      \
      if (e_ == cudaErrorMemoryAllocation) {                                                  \
        throw Error{DSES_ERR_OOM, std::string(#call) + ": " + cudaGetErrorString(e_)};        \
      }                                                                                       \
      throw Error{DSES_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)};         \
    }                                                                                         \
  } while (0)

[[noreturn]] void invalid(const std::string& m) { throw Error{DSES_ERR_INVALID_ARG, m}; }

inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Stream-ordered device allocation (the pool keeps freed blocks cached).
struct DevMem {
  void* p = nullptr;
  cudaStream_t s = nullptr;
  void alloc(size_t bytes, cudaStream_t stream) {
    s = stream;
    CK(cudaMallocAsync(&p, std::max<size_t>(bytes, 256), stream));
  }
  void release() {
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
  }
  ~DevMem() { release(); }
};

struct CellList {
  float cs = 0, inv = 0;
  float lo[3] = {0, 0, 0};
  int dim[3] = {0, 0, 0};
  int* start = nullptr;     // ncells + 1
  float4* sorted = nullptr; // m points in cell order
};

// Pinned host staging for host-to-device uploads of one pipeline run (the
// copies read it asynchronously, and a captured graph replays from it).
struct Stage {
  char* host = nullptr;
  size_t cap = 0, used = 0;
  void reserve(size_t bytes) {
    if (bytes <= cap) return;
    if (host) cudaFreeHost(host);
    host = nullptr;
    cap = 0;
    CK(cudaMallocHost((void**)&host, bytes));
    cap = bytes;
  }
  void release() {
    if (host) cudaFreeHost(host);
    host = nullptr;
    cap = used = 0;
  }
};

struct Options {
  int64_t hist_mode = 0;
  int64_t hist_budget = kHistBudget;
  int64_t points_per_thread = 0;
  int64_t fuse_score = 1;
  int64_t tile_rotations = 0;
  int64_t autotune = 1;
  int64_t use_graphs = 1;
  int64_t serve_max_batch = 16;
  int64_t serve_queue_cap = 100000;
  int64_t serve_mem_budget = 8LL << 30;
  int64_t serve_tile_rotations = 1LL << 30;
  int64_t serve_iter_pairs = 150000000000LL;
  int64_t record_timing = 0;
  int64_t vote_sparse = 0;
  // test hook: the next this-many registrations (blocking or served) are
  // refused at their scratch allocation as if the device allocator had
  // failed (DSES_ERR_OOM), without touching the device
  int64_t fail_next_allocs = 0;
  // the vote's target order, fixed when a target is created: 0 recursive
  // bisection along the longest side (compact groups), 1 Morton
  int64_t target_order = 0;
  // histogram strides: 1 (default) spread a lattice neighbourhood over the
  // shared-memory banks where the padding costs no slab and no source chunk;
  // 0 compact (row and plane strides equal to the extents)
  int64_t hist_strides = 1;
};

}  // namespace

struct dses_target {
  dses_ctx* ctx = nullptr;
  uint64_t uid = 0;         // never reused within a context (graph-cache key)
  int m = 0;
  std::vector<float> host;  // m x 3
  float bbmin[3], bbmax[3];
  float4* Y = nullptr;      // packed, input order
  float4* Ym = nullptr;     // the vote's order (recursive bisection, or Morton)
  float4* gbox = nullptr;   // per group of kGroup consecutive points of Ym: min, max
  int n_groups = 0;
  float gext[3] = {0, 0, 0};  // mean group bounding-box extent per axis
  float4* gbox2 = nullptr;  // the same for groups of 2 kGroup points (paired culled vote)
  int n_groups2 = 0;
  float gext2[3] = {0, 0, 0};
  float* D = nullptr;       // G^3 distance grid
  float4* D4 = nullptr;     // its 2 x 2 (y, z) corner blocks, one per voxel
  int G = 0;
  float glo[3], gh[3], gcap = 0;
  std::map<uint32_t, CellList> cells;  // by bit pattern of epsilon
  std::map<uint32_t, int> capY;        // by bit pattern of delta_t
  std::atomic<int> inflight{0};
};

namespace {

struct Request;  // serving

}  // namespace

struct dses_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int sms = 148;
  std::recursive_mutex mu;
  std::string err;
  std::map<int, float*> hopf;  // cached Hopf grids by N_side
  std::vector<dses_target*> targets;
  uint64_t next_target_uid = 1;
  Options opt;
  // serving
  std::mutex smu;
  std::condition_variable scv;
  std::deque<std::shared_ptr<Request>> queue;
  std::unordered_map<uint64_t, std::shared_ptr<Request>> tickets;
  uint64_t next_ticket = 1;
  std::thread worker;
  bool stop = false;
  bool worker_started = false;
  dses_result* pinned_res = nullptr;  // result staging for blocking calls
  size_t pinned_cap = 0;
  // optional event timing of rotation-pass launches (record_timing = 1)
  struct PassEvents {
    cudaEvent_t start, voted, counted;
  };
  std::vector<PassEvents> pass_events;
  int64_t pass_ns = 0;     // summed duration of the last call's vote launches
  int64_t count_ns = 0;    // ... and of its inlier-count / score launches
  int64_t pass_launches = 0;
  int64_t launch_snapshot = 0;
  int64_t votes_total = 0;  // in-box pair votes of the last blocking call
  int64_t vote_sparse_jobs = 0;  // problems of the last blocking call on the culled vote
  int64_t vote_paired_jobs = 0;  // ... of which on its paired 64-point-group form
  int64_t graph_count = 0;       // snapshot for the "graphs_cached" option
  int64_t serve_max_active = 0;  // most requests the serving worker held at once (resettable to 0)
  int64_t serve_busy_ns = 0;     // summed device time of the serving iterations (resettable to 0)
  int64_t serve_iterations = 0;  // serving iterations retired (resettable to 0)
  // pinned result slots of submitted requests, handed out and returned under
  // smu; allocated in chunks and freed only with the context (pinned frees
  // synchronise the device, which would stall the serving pipeline)
  std::vector<dses_result*> res_chunks;
  std::vector<dses_result*> res_free;
  // host staging: blocking calls, the serving worker, and the one in use
  Stage stage, serve_stage[2];  // the serving worker alternates two (two iterations in flight)
  Stage* cur_stage = nullptr;
  bool capturing = false;
  // captured batch graphs by problem signature
  struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    Stage stage;
    dses_result* res = nullptr;  // pinned results written by the graph
    std::vector<std::pair<size_t, size_t>> src_slots;  // (stage offset, bytes) per problem, host sources
  };
  std::map<std::string, GraphEntry> graphs;
  std::map<std::string, int> graph_seen;
  // autotuner: problem-size bucket -> (points per thread, rotations per work item)
  std::map<std::string, std::pair<int, int>> tuned;
  int64_t last_p_mask = 0;   // points-per-thread shapes of the last blocking call's passes (bit P)
  int64_t last_tile_max = 0; // largest rotations per work item among them
};

namespace {

// ---------------------------------------------------------------------------
// small helpers

uint32_t fbits(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return u;
}

bool finite3(const float* p, int64_t n) {
  for (int64_t i = 0; i < 3 * n; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}

void set_device(dses_ctx* c) { CK(cudaSetDevice(c->device)); }

const float* hopf_grid(dses_ctx* c, int n) {
  auto it = c->hopf.find(n);
  if (it != c->hopf.end()) return it->second;
  float* p = nullptr;
  CK(cudaMalloc(&p, sizeof(float) * 9 * (size_t)72 * n * n * n));
  CK(launch_hopf_grid(n, p, c->stream));
  c->hopf[n] = p;
  return p;
}

// Bound on the target points in any cube of side delta (bounds.h), cached per
// delta: N times it bounds every vote-histogram counter.
int cap_points_in_cube(dses_target* T, float delta) {
  auto it = T->capY.find(fbits(delta));
  if (it != T->capY.end()) return it->second;
  const int best = points_in_cube_bound(T->host.data(), (int64_t)T->m, T->bbmin, delta);
  T->capY[fbits(delta)] = best;
  return best;
}

// The vote's order of the target points and the bounding box of every run of
// kGroup (and 2 kGroup) consecutive points: the culled vote's groups. Order 0
// (default) bisects the cloud recursively along the longest side of its
// bounding box, cutting at a multiple of 2 kGroup points, so every aligned
// run of 2 kGroup points (and each half of one) is a compact box; order 1 is
// Morton (Z-order) over the bounding box. On the robot-like problem the
// bisection keeps 27% fewer (source, 64-point group) pairs than Morton runs
// (whose runs jump between distant cells) at the same window.
void kd_bisect(const std::vector<float>& xyz, std::vector<int>& idx, int lo, int hi, int g) {
  const int n = hi - lo;
  if (n <= g) return;
  float mn[3], mx[3];
  for (int a = 0; a < 3; ++a) {
    mn[a] = mx[a] = xyz[3 * (size_t)idx[lo] + a];
    for (int k = lo + 1; k < hi; ++k) {
      const float v = xyz[3 * (size_t)idx[k] + a];
      mn[a] = std::min(mn[a], v);
      mx[a] = std::max(mx[a], v);
    }
  }
  int ax = 0;
  for (int a = 1; a < 3; ++a)
    if (mx[a] - mn[a] > mx[ax] - mn[ax]) ax = a;
  std::stable_sort(idx.begin() + lo, idx.begin() + hi,
                   [&](int p, int q) { return xyz[3 * (size_t)p + ax] < xyz[3 * (size_t)q + ax]; });
  const int cut = lo + ((n + g - 1) / g / 2) * g;  // the first part a multiple of g: the partial group comes last
  kd_bisect(xyz, idx, lo, cut, g);
  kd_bisect(xyz, idx, cut, hi, g);
}

void build_vote_groups(dses_ctx* c, dses_target* T) {
  const int m = T->m;
  std::vector<std::pair<uint64_t, int>> code((size_t)m);
  if (c->opt.target_order == 1) {
    for (int j = 0; j < m; ++j) {
      uint64_t q[3];
      for (int a = 0; a < 3; ++a) {
        const double ext = (double)T->bbmax[a] - T->bbmin[a];
        const double u = ext > 0 ? ((double)T->host[3 * j + a] - T->bbmin[a]) / ext : 0.0;
        q[a] = (uint64_t)std::min(1023.0, std::max(0.0, std::floor(u * 1024.0)));
      }
      uint64_t k = 0;
      for (int b = 0; b < 10; ++b)
        for (int a = 0; a < 3; ++a) k |= ((q[a] >> b) & 1ull) << (3 * b + a);
      code[(size_t)j] = {k, j};
    }
    std::stable_sort(code.begin(), code.end());
  } else {
    std::vector<int> idx((size_t)m);
    for (int j = 0; j < m; ++j) idx[(size_t)j] = j;
    kd_bisect(T->host, idx, 0, m, 2 * kGroup);
    for (int j = 0; j < m; ++j) code[(size_t)j] = {0, idx[(size_t)j]};
  }
  std::vector<float4> ym((size_t)m);
  for (int j = 0; j < m; ++j) {
    const float* p = &T->host[3 * (size_t)code[(size_t)j].second];
    ym[(size_t)j] = make_float4(p[0], p[1], p[2], 0.f);
  }
  // group boxes for groups of kGroup and of 2 kGroup consecutive points
  auto boxes = [&](int gsize, int* n_out, float* ext, std::vector<float4>& box) {
    const int n = (m + gsize - 1) / gsize;
    *n_out = n;
    box.assign(2 * (size_t)n, make_float4(0.f, 0.f, 0.f, 0.f));
    ext[0] = ext[1] = ext[2] = 0.f;
    for (int g = 0; g < n; ++g) {
      float4 lo = ym[(size_t)g * gsize], hi = lo;
      for (int j = g * gsize; j < std::min(m, (g + 1) * gsize); ++j) {
        lo.x = std::min(lo.x, ym[j].x); lo.y = std::min(lo.y, ym[j].y); lo.z = std::min(lo.z, ym[j].z);
        hi.x = std::max(hi.x, ym[j].x); hi.y = std::max(hi.y, ym[j].y); hi.z = std::max(hi.z, ym[j].z);
      }
      box[2 * (size_t)g] = lo;
      box[2 * (size_t)g + 1] = hi;
      ext[0] += (hi.x - lo.x) / n;
      ext[1] += (hi.y - lo.y) / n;
      ext[2] += (hi.z - lo.z) / n;
    }
  };
  std::vector<float4> box, box2;
  boxes(kGroup, &T->n_groups, T->gext, box);
  boxes(2 * kGroup, &T->n_groups2, T->gext2, box2);
  CK(cudaMalloc(&T->Ym, sizeof(float4) * (size_t)m));
  CK(cudaMalloc(&T->gbox, sizeof(float4) * box.size()));
  CK(cudaMalloc(&T->gbox2, sizeof(float4) * box2.size()));
  CK(cudaMemcpyAsync(T->Ym, ym.data(), sizeof(float4) * (size_t)m, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(T->gbox, box.data(), sizeof(float4) * box.size(), cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(T->gbox2, box2.data(), sizeof(float4) * box2.size(), cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
}

// Target cell list for inlier counting at tolerance eps: cells at least
// eps * 1.001 wide (so a query's 3x3x3 neighbourhood holds every point within
// eps even after FP32 rounding), at most ~4M cells.
CellList* cell_list(dses_ctx* c, dses_target* T, float eps) {
  auto it = T->cells.find(fbits(eps));
  if (it != T->cells.end()) return &it->second;
  CellList cl;
  double ext = 0;
  for (int a = 0; a < 3; ++a) ext = std::max(ext, (double)T->bbmax[a] - T->bbmin[a]);
  double cs = std::max((double)eps * 1.001, ext / 128.0);
  if (cs <= 0) cs = 1e-6;
  int dim[3];
  for (;;) {
    int64_t total = 1;
    for (int a = 0; a < 3; ++a) {
      dim[a] = (int)std::floor(((double)T->bbmax[a] - T->bbmin[a]) / cs) + 3;
      total *= dim[a];
    }
    if (total <= (4 << 20)) break;
    cs *= 1.26;
  }
  cl.cs = (float)cs;
  cl.inv = (float)(1.0 / cs);
  for (int a = 0; a < 3; ++a) {
    cl.lo[a] = (float)((double)T->bbmin[a] - cs);
    cl.dim[a] = dim[a];
  }
  const int ncells = dim[0] * dim[1] * dim[2];
  CK(cudaMalloc(&cl.start, sizeof(int) * ((size_t)ncells + 1)));
  CK(cudaMalloc(&cl.sorted, sizeof(float4) * (size_t)T->m));
  DevMem tmp;
  tmp.alloc(sizeof(int) * ((size_t)2 * ncells + T->m), c->stream);
  int* counts = (int*)tmp.p;
  CK(launch_cell_list(T->Y, T->m, cl.lo, cl.inv, cl.dim, counts, cl.start, counts + ncells, cl.sorted, c->stream));
  tmp.release();
  return &(T->cells[fbits(eps)] = cl);
}

// ---------------------------------------------------------------------------
// one registration problem, resolved and planned

struct Job {
  const dses_problem* prob = nullptr;
  dses_target* T = nullptr;
  CellList* cl = nullptr;
  int N = 0;
  const float* X = nullptr;  // device
  int metric = 0, q = 0, topk = 0, nn = 0, rtop = 0, rK = 0;
  float eps = 0, delta = 0, tau = 0, hh = 0, pexp = 1;
  double rdr = 0;
  int lo[3], E[3];
  const float* rot = nullptr;  // first-pass rotations (device)
  int64_t n_first = 0, n_fine = 0, n_total = 0;
  int hopf_n = 0;
  // plan
  int u16 = 0, lanes = 0, slab_x = 0, n_slabs = 1, hist_bytes = 0;
  int Ep[3] = {0, 0, 0};  // vote layout extents: E padded to odd values
  int64_t hs[2] = {0, 0};  // vote layout strides in bins: per x-plane, per y-row
  bool fused = false;
  int sparse = 0;  // culled vote: 0 no, 1 32-point groups, 2 paired 64-point groups
  int tile = 0;    // rotations per work item picked by the autotuner (0: the launch's default)
  int* Xperm = nullptr;  // culled vote: sources in bisection order (device), or NULL
  // device scratch
  DevMem mem;
  int4* kv = nullptr;
  uint32_t* M = nullptr;
  float* cost = nullptr;
  uint32_t* cand = nullptr;
  uint32_t* n_cand = nullptr;  // [0] first pass, [1] second pass
  uint32_t* acc = nullptr;     // [0] M* first, [1] max V first, [2] M* second, [3] max V second
  unsigned long long* best = nullptr;  // [0] argmin key, [1] total in-box pair votes
  unsigned long long* keys = nullptr;
  unsigned long long* ks_scratch = nullptr;
  unsigned long long* ksel = nullptr;
  float* rot_fine = nullptr;
  float* rot_own = nullptr;  // Euler-box / explicit first-pass grid
  double* R0 = nullptr;
  float* Xown = nullptr;
  dses_result* res = nullptr;
  size_t bytes = 0;
  int ksel_k = 0;
  size_t src_stage_off = 0;  // where the host source sits in the pinned stage
};

// Copies bytes into the current pinned stage; returns the staged pointer.
const void* stage_put(dses_ctx* c, const void* src, size_t bytes, size_t* offset = nullptr) {
  Stage* st = c->cur_stage;
  const size_t off = (st->used + 63) & ~(size_t)63;
  if (!st->host || off + bytes > st->cap) throw Error{DSES_ERR_CUDA, "internal: host staging too small"};
  std::memcpy(st->host + off, src, bytes);
  st->used = off + bytes;
  if (offset) *offset = off;
  return st->host + off;
}

// Upper bound of the staging bytes one pipeline run over `jobs` uses.
size_t stage_bytes(const std::vector<Job*>& jobs) {
  size_t b = 4096;
  for (auto* j : jobs) {
    b += 64 * 16 + 6 * sizeof(PassDesc) + 2 * 16 + sizeof(FinalDesc) + 72;
    if (!j->prob->src_is_device) b += 12 * (size_t)j->N;
    if (j->sparse) b += 4 * (size_t)j->N + 64;  // the culled source order, when staged
    if (j->prob->grid.kind == DSES_GRID_EXPLICIT) b += 36 * (size_t)j->n_first;
  }
  return b;
}

void resolve(dses_ctx* c, const dses_problem* pb, Job& j) {
  if (!pb) invalid("problem is NULL");
  j.prob = pb;
  dses_target* T = const_cast<dses_target*>(pb->target);
  if (!T || T->ctx != c) invalid("target is NULL or belongs to another context");
  j.T = T;
  if (!pb->src) invalid("src is NULL");
  if (pb->n_src < 1 || pb->n_src > (1 << 24)) invalid("n_src must be in [1, 2^24]");
  j.N = (int)pb->n_src;
  if (!pb->src_is_device && !finite3(pb->src, pb->n_src)) invalid("source cloud has a non-finite coordinate");
  const dses_params& P = pb->params;
  if (P.metric < 0 || P.metric > 4) invalid("unknown metric");
  j.metric = P.metric;
  if (!(P.epsilon > 0) || !std::isfinite(P.epsilon)) invalid("epsilon must be positive and finite");
  j.eps = P.epsilon;
  j.delta = P.delta_t > 0 ? P.delta_t : P.epsilon;
  if (!std::isfinite(j.delta)) invalid("delta_t must be finite");
  j.tau = P.tau > 0 ? P.tau : 2.f * P.epsilon;
  j.hh = P.huber_h > 0 ? P.huber_h : P.epsilon;
  j.pexp = P.p;
  if (j.metric == DSES_METRIC_LP && !(P.p > 0 && P.p <= 1)) invalid("LP metric needs p in (0, 1]");
  if (P.q_milli < 0 || P.q_milli > 1000) invalid("q_milli must be in [0, 1000]");
  if (P.top_k < 0 || P.top_k > 1024) invalid("top_k must be in [0, 1024]");
  if (P.nn_mode != DSES_NN_GRID && P.nn_mode != DSES_NN_BRUTE) invalid("unknown nn_mode");
  j.q = P.q_milli;
  j.topk = P.top_k;
  j.nn = P.nn_mode;
  if (P.refine_top_k < 0 || P.refine_top_k > 1024) invalid("refine_top_k must be in [0, 1024]");
  j.rtop = P.refine_top_k;
  if (j.rtop > 0) {
    if (P.refine_K < 0 || P.refine_K > 16) invalid("refine_K must be in [0, 16]");
    if (!(P.refine_delta_r > 0) || !std::isfinite(P.refine_delta_r)) invalid("refine_delta_r must be positive");
  }
  j.rK = P.refine_K;
  j.rdr = P.refine_delta_r;
  if (j.metric != DSES_METRIC_INLIER && j.nn == DSES_NN_GRID && j.metric != DSES_METRIC_LP && T->gcap < j.tau)
    invalid("the target's distance-grid cap is below tau; recreate the target with grid_cap >= tau");
  // translation box: lattice points k delta inside [c - s, c + s]
  for (int a = 0; a < 3; ++a) {
    if (!(P.t_half[a] > 0) || !std::isfinite(P.t_half[a]) || !std::isfinite(P.t_center[a]))
      invalid("t_half must be positive and t_center finite");
    const double lo = std::ceil(((double)P.t_center[a] - (double)P.t_half[a]) / (double)j.delta);
    const double hi = std::floor(((double)P.t_center[a] + (double)P.t_half[a]) / (double)j.delta);
    if (hi < lo) invalid("translation box holds no lattice point");
    if (lo < -(1 << 20) || hi > (1 << 20)) invalid("translation box too large for delta_t");
    j.lo[a] = (int)lo;
    j.E[a] = (int)(hi - lo + 1);
  }
  // rotation grid
  const dses_rotation_grid& g = pb->grid;
  if (g.kind == DSES_GRID_HOPF) {
    if (g.hopf_n < 1 || g.hopf_n > 48) invalid("hopf_n must be in [1, 48]");
    j.hopf_n = g.hopf_n;
    j.n_first = 72LL * g.hopf_n * g.hopf_n * g.hopf_n;
  } else if (g.kind == DSES_GRID_EULER_BOX) {
    if (g.K < 0 || g.K > 100) invalid("Euler box K must be in [0, 100]");
    if (!(g.delta_r > 0)) invalid("Euler box delta_r must be positive");
    j.n_first = (int64_t)(2 * g.K + 1) * (2 * g.K + 1) * (2 * g.K + 1);
  } else if (g.kind == DSES_GRID_EXPLICIT) {
    if (!g.explicit_R || g.n_explicit < 1) invalid("explicit grid needs explicit_R and n_explicit >= 1");
    j.n_first = g.n_explicit;
  } else {
    invalid("unknown rotation grid kind");
  }
  const int B = (2 * j.rK + 1) * (2 * j.rK + 1) * (2 * j.rK + 1);
  j.n_fine = j.rtop > 0 ? (int64_t)j.rtop * B : 0;
  j.n_total = j.n_first + j.n_fine;
  if (j.n_total >= (1LL << 31)) invalid("too many rotations");
}

// Histogram slabs over the x planes: (slab width, slab count, padded x extent)
// such that every slab is an odd number of planes (the centred vote needs odd
// extents); at most one padding plane is added.
static void odd_slabs(int64_t Ex, int64_t max_planes, int64_t* sx, int64_t* n, int64_t* Exp) {
  if (Ex + (Ex % 2 == 0 ? 1 : 0) <= max_planes) {
    *sx = *Exp = Ex | 1;
    *n = 1;
    return;
  }
  int64_t w = max_planes % 2 == 0 ? max_planes - 1 : max_planes;
  *sx = w;
  *n = (Ex + w - 1) / w;
  const int64_t last = Ex - (*n - 1) * w;
  *Exp = Ex + (last % 2 == 0 ? 1 : 0);
}

bool culled_source_order(const Job& j);

// Source chunks a launch of this job alone stages per rotation with a
// histogram of hist_bytes (pass_staging and set_chunks of the launch).
int source_chunks(const Job& j, int hist_bytes) {
  int src = 0, blk = 0, list = 0;
  const bool blocks = j.sparse && culled_source_order(j);
  pass_staging(hist_bytes, j.N, blocks, j.sparse == 2, &src, &blk, &list);
  const int cap = j.sparse == 2 ? std::max(1, src / kTileBytes) * kTileSources : std::max(1, src / (j.sparse ? 16 : 32));
  return (j.N + cap - 1) / cap;
}

// Row and plane strides (in bins) of the 32-bit vote histogram, padded past
// the extents where that spreads a lattice neighbourhood over more banks
// (pick_strides, strides.h) without costing a slab or a source chunk: the
// slab keeps its x-planes within the budget and the launch stages the sources
// in as many chunks as with the compact layout. 16-bit counters keep the
// compact layout: their conflicts come mostly from the two halves of one
// word, which padding does not separate. The choice depends on the extents
// and the byte limit only, and is cached.
void spread_strides(Job& j, int64_t budget) {
  if (j.u16) return;
  const int64_t Ey = j.Ep[1], Ez = j.Ep[2], sx = j.slab_x;
  // the largest histogram that keeps the budget and the source chunks
  const int chunks0 = source_chunks(j, j.hist_bytes);
  int64_t lo = j.hist_bytes, hi = budget - 8;
  if (hi < lo) return;
  if (source_chunks(j, (int)hi) > chunks0) {
    while (hi - lo > 16) {
      const int64_t mid = (lo + hi) / 2;
      if (source_chunks(j, (int)mid) > chunks0) hi = mid; else lo = mid;
    }
    hi = lo;
  }
  const int64_t limit = hi;
  static std::mutex mu;
  static std::map<std::array<int64_t, 4>, std::pair<int64_t, int64_t>> cache;
  const std::array<int64_t, 4> key{Ey, Ez, sx, limit};
  std::pair<int64_t, int64_t> pick;
  {
    std::lock_guard<std::mutex> g(mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
      pick = it->second;
    } else {
      pick = pick_strides(Ey, Ez, sx, limit);
      // a process that plans many box shapes keeps at most 4,096 choices
      // (~0.3 ms of host search each to redo)
      if (cache.size() >= 4096) cache.clear();
      cache[key] = pick;
    }
  }
  j.hs[0] = pick.first;
  j.hs[1] = pick.second;
  j.hist_bytes = layout_bytes(sx, pick.first, false);
}

void plan(dses_ctx* c, Job& j) {
  // vote layout: the lattice box padded to odd extents (the centred vote
  // paths need them); the scan of a padded layout skips the padding bins
  const int64_t Ey = j.E[1] | 1, Ez = j.E[2] | 1, Ex = j.E[0];
  const int64_t budget = c->opt.hist_budget;
  const int64_t M = j.T->m;
  bool u16_ok = (int64_t)j.N * M <= 65535;
  if (!u16_ok) u16_ok = (int64_t)j.N * cap_points_in_cube(j.T, j.delta) <= 65535;
  bool u16;
  if (c->opt.hist_mode == 1) {
    u16 = false;
  } else if (c->opt.hist_mode == 2) {
    if (!u16_ok) invalid("16-bit vote counters could overflow for this problem");
    u16 = true;
  } else {
    u16 = ((Ex | 1) * Ey * Ez * 4 > budget) && u16_ok;
  }
  const int64_t per_plane = Ey * Ez * (u16 ? 2 : 4);
  if (per_plane + 8 > budget) invalid("translation box too large: one lattice plane exceeds the histogram budget");
  int64_t sx, ns, Exp;
  odd_slabs(Ex, (budget - 8) / per_plane, &sx, &ns, &Exp);
  j.u16 = u16;
  j.slab_x = (int)sx;
  j.n_slabs = (int)ns;
  j.Ep[0] = (int)Exp;
  j.Ep[1] = (int)Ey;
  j.Ep[2] = (int)Ez;
  j.hs[0] = Ey * Ez;
  j.hs[1] = Ez;
  j.hist_bytes = layout_bytes(sx, j.hs[0], u16);
  j.lanes = 0;
  // One 32-bit copy of every bin per lane (word bin * 32 + lane, so a warp's
  // increments never share a bank), on request only: measured slower than
  // shared 32-bit counters on every small box tried (dense 9^3: 13.2 vs
  // 12.4 ms; culled ModelNet-shaped and robot boxes: 1-13%), the scan of
  // 32 copies per bin costing more than the bank conflicts it removes.
  const int64_t all = (Ex | 1) * Ey * Ez;
  const bool lanes_fit = all * 128 + 8 <= budget;
  const bool lanes = c->opt.hist_mode == 3;
  if (lanes) {
    if (!lanes_fit) invalid("lane-private counters need 128 bytes per lattice bin within the histogram budget");
    j.u16 = 0;
    j.lanes = 1;
    j.slab_x = (int)(Ex | 1);
    j.n_slabs = 1;
    j.Ep[0] = (int)(Ex | 1);
    j.hist_bytes = (int)(all * 128);
  }
  j.fused = c->opt.fuse_score && j.q == 0 && j.topk == 0 && (j.metric == DSES_METRIC_INLIER || j.nn == DSES_NN_GRID);
  // Culling pays when the translation window (plus a target group's extent)
  // covers a small part of the target: estimated fraction of (source, group)
  // pairs that survive, per axis (window + group extent) / target extent.
  double keep = 1.0;
  for (int a = 0; a < 3; ++a) {
    const double ext = (double)j.T->bbmax[a] - j.T->bbmin[a];
    const double win = (double)j.E[a] * j.delta + j.T->gext[a];
    keep *= ext > 0 ? std::min(1.0, win / ext) : 1.0;
  }
  const bool cull = c->opt.vote_sparse >= 2 || (c->opt.vote_sparse == 0 && keep < 0.35);
  // paired 64-point groups when the window is at least 0.6 mean group extents
  // wide on every axis (each kept source then votes 64 targets in one packed
  // step). Measured: paired faster at 0.73 (robot search ranges, 11%) and 2.2
  // (robot-like, 9%); 32-point groups faster at 0.14-0.5 (ModelNet-shaped
  // small boxes, 8-10%).
  double span = 1e300;
  for (int a = 0; a < 3; ++a)
    span = std::min(span, (double)j.E[a] * j.delta / std::max(1e-12, (double)j.T->gext2[a]));
  j.sparse = !cull ? 0 : c->opt.vote_sparse == 2 ? 1 : c->opt.vote_sparse == 3 ? 2 : (span >= 0.6 ? 2 : 1);
  // the paired form votes into shared counters only: lane-private counters
  // take the 32-point culled path
  if (j.lanes && j.sparse == 2) j.sparse = 1;
  if (c->opt.hist_strides && !j.lanes) spread_strides(j, budget);
}

int choose_p(dses_ctx* c, const std::vector<Job*>& jobs) {
  if (c->opt.points_per_thread > 0) return (int)c->opt.points_per_thread;
  int64_t mmax = 0;
  for (auto* j : jobs) mmax = std::max<int64_t>(mmax, j->T->m);
  const int P = mmax <= 128 ? 1 : (mmax <= 512 ? 2 : 4);
  bool paired = false;
  for (auto* j : jobs) paired |= j->sparse == 2;
  return paired && P == 1 ? 2 : P;  // the paired culled vote is built for 2 and 4
}

int gcd(int a, int b) { return b ? gcd(b, a % b) : a; }

// Set on the serving worker's thread (no autotuner trials there).
thread_local bool t_serving_worker = false;

// Vote items per source chunk the sparse path aims for (a few per warp).
constexpr int c_sparse_items = 128;

// Does the culled vote stage this job's sources in bisection order? When its
// items walk at least 256 sources each (sized here with the largest culled
// shape, 4 points per lane: 128 targets per item).
bool culled_source_order(const Job& j) {
  if (!j.sparse) return false;
  const int64_t chunks = ((int64_t)j.T->m + 127) / 128;
  const int64_t groups = std::max<int64_t>(1, c_sparse_items / std::max<int64_t>(1, chunks));
  return j.N / groups >= 256;
}

void carve(Job& j) {
  size_t off = 0;
  auto take = [&](size_t b) {
    const size_t o = off;
    off += align256(b);
    return o;
  };
  const size_t n = (size_t)j.n_total;
  const int kmax = std::max({j.topk, j.rtop, 1});
  j.ksel_k = kmax;
  const size_t o_kv = take(16 * n), o_M = take(4 * n), o_cost = take(4 * n), o_cand = take(4 * n),
               o_nc = take(8), o_acc = take(16), o_best = take(16), o_keys = take(8 * n),
               o_ks = take(8 * k_smallest_scratch((int)j.n_total, kmax)), o_ksel = take(8 * (size_t)kmax),
               o_fine = take(36 * (size_t)j.n_fine + 4), o_res = take(sizeof(dses_result));
  const bool own_rot = j.prob->grid.kind != DSES_GRID_HOPF;
  const size_t o_rot = own_rot ? take(36 * (size_t)j.n_first) : 0, o_R0 = own_rot ? take(72) : 0;
  const size_t o_X = j.prob->src_is_device ? 0 : take(12 * (size_t)j.N);
  const bool perm = culled_source_order(j);
  const size_t o_perm = perm ? take(4 * (size_t)j.N) : 0;
  j.bytes = off;
  j.mem.alloc(off, j.mem.s ? j.mem.s : nullptr);
  char* b = (char*)j.mem.p;
  j.kv = (int4*)(b + o_kv);
  j.M = (uint32_t*)(b + o_M);
  j.cost = (float*)(b + o_cost);
  j.cand = (uint32_t*)(b + o_cand);
  j.n_cand = (uint32_t*)(b + o_nc);
  j.acc = (uint32_t*)(b + o_acc);
  j.best = (unsigned long long*)(b + o_best);
  j.keys = (unsigned long long*)(b + o_keys);
  j.ks_scratch = (unsigned long long*)(b + o_ks);
  j.ksel = (unsigned long long*)(b + o_ksel);
  j.rot_fine = (float*)(b + o_fine);
  j.res = (dses_result*)(b + o_res);
  if (own_rot) {
    j.rot_own = (float*)(b + o_rot);
    j.R0 = (double*)(b + o_R0);
  }
  if (!j.prob->src_is_device) j.Xown = (float*)(b + o_X);
  j.Xperm = perm ? (int*)(b + o_perm) : nullptr;
}

// Device memory one job needs (for serving admission).
size_t job_bytes(const Job& j) {
  const size_t n = (size_t)j.n_total;
  const int kmax = std::max({j.topk, j.rtop, 1});
  size_t b = 40 * n + 8 * k_smallest_scratch((int)j.n_total, kmax) + 36 * (size_t)j.n_fine + 16 * (size_t)j.N +
             (j.prob->grid.kind != DSES_GRID_HOPF ? 36 * (size_t)j.n_first : 0) + 16 * 256;
  return b;
}

// Scratch and inputs of a job: carve its device scratch, the target's cell
// list at its epsilon, and the source cloud on the device.
void stage_inputs(dses_ctx* c, Job& j) {
  cudaStream_t s = c->stream;
  j.mem.s = s;
  if (c->opt.fail_next_allocs > 0) {
    --c->opt.fail_next_allocs;
    throw Error{DSES_ERR_OOM, "scratch allocation refused (fail_next_allocs test hook)"};
  }
  carve(j);
  j.cl = cell_list(c, j.T, j.eps);
  if (j.Xown) {
    const void* st = stage_put(c, j.prob->src, 12 * (size_t)j.N, &j.src_stage_off);
    CK(cudaMemcpyAsync(j.Xown, st, 12 * (size_t)j.N, cudaMemcpyHostToDevice, s));
    j.X = j.Xown;
  } else {
    j.X = j.prob->src;
  }
  if (j.Xperm) {
    // the culled vote stages the sources in bisection order: a block of 32
    // staged sources is then compact, and a block whose bounds miss an item's
    // window is skipped whole (the vote's counts do not depend on the order)
    std::vector<float> xyz(3 * (size_t)j.N);
    if (j.prob->src_is_device) {
      if (c->capturing) {  // no host copy inside a capture: the input order
        j.Xperm = nullptr;
        return;
      }
      CK(cudaMemcpyAsync(xyz.data(), j.prob->src, 12 * (size_t)j.N, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
    } else {
      std::memcpy(xyz.data(), j.prob->src, 12 * (size_t)j.N);
    }
    std::vector<int> idx((size_t)j.N);
    for (int i = 0; i < j.N; ++i) idx[(size_t)i] = i;
    kd_bisect(xyz, idx, 0, j.N, 32);
    CK(cudaMemcpyAsync(j.Xperm, stage_put(c, idx.data(), 4 * (size_t)j.N), 4 * (size_t)j.N, cudaMemcpyHostToDevice,
                       s));
  }
}

// Zeroed accumulators (M*, max V, candidate counts, votes), an empty argmin
// key and NaN costs (a rotation that is never scored keeps NaN).
void stage_reset(dses_ctx* c, Job& j) {
  cudaStream_t s = c->stream;
  CK(cudaMemsetAsync(j.acc, 0, 16, s));
  CK(cudaMemsetAsync(j.n_cand, 0, 8, s));
  CK(launch_fill_u64(j.best, ~0ull, 1, s));
  CK(cudaMemsetAsync(j.best + 1, 0, 8, s));
  if (j.n_total > 0) CK(launch_fill_f32(j.cost, NAN, (size_t)j.n_total, s));
}

// Allocate scratch, upload inputs, build per-call grids, reset accumulators.
void stage_setup(dses_ctx* c, Job& j) {
  cudaStream_t s = c->stream;
  stage_inputs(c, j);
  const dses_rotation_grid& g = j.prob->grid;
  if (g.kind == DSES_GRID_HOPF) {
    j.rot = hopf_grid(c, g.hopf_n);
  } else if (g.kind == DSES_GRID_EULER_BOX) {
    CK(cudaMemcpyAsync(j.R0, stage_put(c, g.R0, sizeof(double) * 9), sizeof(double) * 9, cudaMemcpyHostToDevice, s));
    CK(launch_euler_box_single(j.R0, g.K, g.delta_r, j.rot_own, s));
    j.rot = j.rot_own;
  } else {
    if (!finite3(g.explicit_R, 3 * g.n_explicit)) invalid("explicit rotations have a non-finite entry");
    CK(cudaMemcpyAsync(j.rot_own, stage_put(c, g.explicit_R, 36 * (size_t)g.n_explicit), 36 * (size_t)g.n_explicit,
                       cudaMemcpyHostToDevice, s));
    j.rot = j.rot_own;
  }
  stage_reset(c, j);
}


PassDesc make_desc(const Job& j, int P, bool second) {
  PassDesc d;
  std::memset(&d, 0, sizeof(d));
  d.X = j.X;
  d.Xperm = j.Xperm;
  d.Y = j.cl->sorted;
  d.Yv = j.T->Ym;
  d.gbox = j.sparse == 2 ? j.T->gbox2 : j.T->gbox;
  d.n_groups = j.sparse == 2 ? j.T->n_groups2 : j.T->n_groups;
  d.N = j.N;
  d.M = j.T->m;
  if (!second) {
    d.rot = j.rot;
    d.n_rot = (int)j.n_first;
    d.rot_base = 0;
    d.acc = j.acc;
  } else {
    d.rot = j.rot_fine;
    d.n_rot = (int)j.n_fine;
    d.rot_base = (uint32_t)j.n_first;
    d.acc = j.acc + 2;
  }
  d.inv_delta = 1.0f / j.delta;
  d.delta = j.delta;
  for (int a = 0; a < 3; ++a) {
    d.lo[a] = j.lo[a];
    d.E[a] = j.Ep[a];
    d.Ev[a] = j.E[a];
  }
  d.hs[0] = (uint32_t)j.hs[0];
  d.hs[1] = (uint32_t)j.hs[1];
  {
    // the magnitudes the culled paths' FP32 keep tests round at: target
    // coordinates and the box's lattice offsets, in lattice units
    double big = 0;
    for (int a = 0; a < 3; ++a)
      big = std::max({big, std::fabs((double)j.T->bbmin[a]) / j.delta, std::fabs((double)j.T->bbmax[a]) / j.delta,
                      std::fabs((double)j.lo[a]) + (double)j.Ep[a]});
    d.cull_margin = (float)(1e-3 + std::ldexp(big, -20));
  }
  d.slab_x = j.slab_x;
  d.n_slabs = j.n_slabs;
  d.hist_u16 = j.u16;
  d.hist_lanes = j.lanes;
  d.sparse = j.sparse;
  d.n_tchunks = (j.T->m + 32 * P - 1) / (32 * P);
  // dense: items a multiple of the 32 warps (equal work per item); sparse:
  // items are uneven anyway and the CTA's item counter balances them, so keep
  // each item's target loads and thresholds amortised over many sources
  d.n_sgroups = j.sparse ? std::max(1, (int)(c_sparse_items / std::max(1, d.n_tchunks)))
                         : 32 / gcd(d.n_tchunks, 32);
  d.eps2 = j.eps * j.eps;
  d.cell_start = j.cl->start;
  for (int a = 0; a < 3; ++a) {
    d.cell_lo[a] = j.cl->lo[a];
    d.cell_dim[a] = j.cl->dim[a];
    d.glo[a] = j.T->glo[a];
    d.ginv_h[a] = 1.0f / j.T->gh[a];
  }
  d.cell_inv = j.cl->inv;
  d.fuse_score = j.fused ? 1 : 0;
  d.metric = j.metric;
  d.eps = j.eps;
  d.tau = j.tau;
  d.huber_h = j.hh;
  d.p_exp = j.pexp;
  d.D = j.T->D;
  d.D4 = j.T->D4;
  d.G = j.T->G;
  d.gcap = j.T->gcap;
  {
    // margin of the grid distance bounds: far above the FP32 error of the
    // stored distances and of the corner distances
    d.grid_err = (float)(1e-5 + 1e-5 * j.T->gcap);
  }
  d.out_base = 0;
  d.kv = j.kv;
  d.Mout = j.M;
  d.cost = j.cost;
  d.best = j.best;
  d.votes_total = j.best + 1;
  return d;
}

// Rotations per work item: enough items to balance the SMs, few enough to
// keep the work counter cold.
int tile_rotations(dses_ctx* c, int64_t total_rot) {
  if (c->opt.tile_rotations > 0) return (int)c->opt.tile_rotations;
  // at least ~32 tiles per SM, so the launch's tail (SMs idle while the last
  // tiles finish) stays a few percent of the launch; at most 16 rotations
  const int64_t t = total_rot / ((int64_t)c->sms * 32);
  return (int)std::max<int64_t>(1, std::min<int64_t>(16, t));
}

// One persistent launch over the given (job, rotation range) work.
struct PassPart {
  Job* job;
  bool second;
  int64_t r0, r1;  // rotation range of the pass (local indices)
};

// The culled instances of the vote kernel carry only their culled path,
// which needs odd layout extents on every axis and slab (the centred vote;
// plan() pads every layout so).
void check_culled_layout(const Job& j) {
  const int last = j.Ep[0] - (j.n_slabs - 1) * j.slab_x;
  if (j.sparse && !((j.Ep[1] & 1) && (j.Ep[2] & 1) && (j.slab_x & 1) && (last & 1)))
    throw Error{DSES_ERR_CUDA, "internal: culled vote planned with an even layout extent"};
}

// The culled vote skips whole blocks of 32 staged sources by their bounds
// when its items walk many sources, the sources staged in bisection order
// (the robot-like problem: 5,000 per item, vote 22.7% faster). With few
// sources per item (a ModelNet-shaped source against a small box: ~45) there
// is little to skip, and the spatially ordered sources alone made that vote
// 6% slower (consecutive kept sources increment nearby bins), so such
// problems keep the input order and the launch stages no bounds.
bool block_bounds_pay(const PassDesc& d) { return d.sparse && d.Xperm && d.N / std::max(1, d.n_sgroups) >= 256; }

void launch_pass(dses_ctx* c, const std::vector<PassPart>& parts, int P) {
  if (parts.empty()) return;
  cudaStream_t s = c->stream;
  std::vector<PassDesc> descs;
  std::vector<int> prefix(1, 0), rprefix(1, 0);
  int64_t total_rot = 0;
  int hist = 16;
  for (auto& pp : parts) total_rot += pp.r1 - pp.r0;
  const int tile = tile_rotations(c, total_rot);
  // a tuned tile is kept below the size that leaves fewer than ~32 tiles per
  // SM in this launch (the launch's tail)
  const int tile_cap = (int)std::max<int64_t>(1, total_rot / ((int64_t)c->sms * 32));
  c->last_p_mask |= 1LL << P;
  for (auto& pp : parts) {
    PassDesc d = make_desc(*pp.job, P, pp.second);
    d.rot += 9 * pp.r0;
    d.rot_base += (uint32_t)pp.r0;
    d.n_rot = (int)(pp.r1 - pp.r0);
    d.tile_rot = c->opt.tile_rotations > 0 ? (int)c->opt.tile_rotations
                 : pp.job->tile > 0         ? std::min(pp.job->tile, tile_cap)
                                            : tile;
    c->last_tile_max = std::max<int64_t>(c->last_tile_max, d.tile_rot);
    descs.push_back(d);
    prefix.push_back(prefix.back() + (int)((d.n_rot + d.tile_rot - 1) / d.tile_rot));
    rprefix.push_back(rprefix.back() + d.n_rot);
    hist = std::max(hist, pp.job->hist_bytes);
  }
  int max_n = 1;
  bool blocks = true;
  for (auto& pp : parts) max_n = std::max(max_n, pp.job->N);
  for (auto& d : descs) blocks &= block_bounds_pay(d);
  bool paired = false;
  for (auto& pp : parts) paired |= pp.job->sparse == 2;
  int src_bytes = 0, blk_bytes = 0, list_bytes = 0;
  pass_staging(hist, max_n, blocks, paired, &src_bytes, &blk_bytes, &list_bytes);
  for (auto& d : descs) set_chunks(d, src_bytes);
  const size_t db = align256(sizeof(PassDesc) * descs.size()), pb = align256(sizeof(int) * prefix.size());
  DevMem m;
  m.alloc(db + 2 * pb + 256, s);
  char* base = (char*)m.p;
  CK(cudaMemcpyAsync(base, stage_put(c, descs.data(), sizeof(PassDesc) * descs.size()),
                     sizeof(PassDesc) * descs.size(), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(base + db, stage_put(c, prefix.data(), sizeof(int) * prefix.size()), sizeof(int) * prefix.size(),
                     cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(base + db + pb, stage_put(c, rprefix.data(), sizeof(int) * rprefix.size()),
                     sizeof(int) * rprefix.size(), cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(base + db + 2 * pb, 0, 4, s));
  PassLaunch L;
  L.probs = (const PassDesc*)base;
  L.tile_prefix = (const int*)(base + db);
  L.rot_prefix = (const int*)(base + db + pb);
  L.n_probs = (int)descs.size();
  L.tile_rot = tile;
  L.work_counter = (int*)(base + db + 2 * pb);
  L.hist_bytes = hist;
  L.src_bytes = src_bytes;
  L.blk_bytes = blk_bytes;
  L.list_bytes = list_bytes;
  L.padded = 0;
  for (auto& pp : parts)
    for (int a = 0; a < 3; ++a) L.padded |= pp.job->Ep[a] != pp.job->E[a] ? 1 : 0;
  const int ctas = std::max(1, std::min(c->sms, prefix.back()));
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  if (c->opt.record_timing && !c->capturing) {
    for (auto& e : ev) CK(cudaEventCreate(&e));
    CK(cudaEventRecord(ev[0], s));
  }
  // one culled mode per launch (the engine groups launches by shape and mode)
  int mode = 0;
  for (auto& pp : parts) mode = std::max(mode, pp.job->sparse);
  // a culled instance carries only its culled path, which needs odd layout
  // extents (the centred vote): every problem of the launch must be of that
  // mode and have them
  for (auto& pp : parts) {
    if (pp.job->sparse != mode) throw Error{DSES_ERR_CUDA, "internal: mixed culled modes"};
    check_culled_layout(*pp.job);
  }
  if ((mode == 1 && P == 8) || (mode == 2 && P != 2 && P != 4))
    throw Error{DSES_ERR_CUDA, "internal: culled vote planned with an unsupported points-per-thread shape"};
  CK(launch_vote(L, P, mode, ctas, s));
  if (ev[0]) CK(cudaEventRecord(ev[1], s));
  CK(launch_count(L, (int)total_rot, s));
  if (ev[0]) {
    CK(cudaEventRecord(ev[2], s));
    c->pass_events.push_back({ev[0], ev[1], ev[2]});
  }
  m.release();
}

ScoreDesc make_score(const Job& j, bool second) {
  ScoreDesc d;
  std::memset(&d, 0, sizeof(d));
  d.X = j.X;
  d.Y = j.cl->sorted;
  d.rot = second ? j.rot_fine : j.rot;
  d.rot_base = second ? (uint32_t)j.n_first : 0;
  d.out_base = 0;
  d.N = j.N;
  d.M = j.T->m;
  d.delta = j.delta;
  d.metric = j.metric;
  d.eps = j.eps;
  d.tau = j.tau;
  d.huber_h = j.hh;
  d.p_exp = j.pexp;
  d.D = j.T->D;
  d.D4 = j.T->D4;
  d.G = j.T->G;
  for (int a = 0; a < 3; ++a) {
    d.glo[a] = j.T->glo[a];
    d.ginv_h[a] = 1.0f / j.T->gh[a];
  }
  d.gcap = j.T->gcap;
  d.kv = j.kv;
  d.Mout = j.M;
  d.cost = j.cost;
  return d;
}

// Candidate selection, scoring and argmin of one pass (skipped when fused).
void stage_candidates(dses_ctx* c, Job& j, bool second) {
  if (j.fused) return;
  cudaStream_t s = c->stream;
  const uint32_t first = second ? (uint32_t)j.n_first : 0;
  const int n = (int)(second ? j.n_fine : j.n_first);
  uint32_t* cand = j.cand + first;
  uint32_t* ncand = j.n_cand + (second ? 1 : 0);
  if (j.topk > 0) {
    CK(launch_keys_from_M(j.M, first, n, 0, j.keys, s));
    const int k = std::min(j.topk, n);
    CK(launch_k_smallest(j.keys, n, nullptr, k, j.ks_scratch, j.ksel, s));
    CK(launch_cand_from_keys(j.ksel, k, 0, cand, ncand, s));
  } else {
    CK(launch_select_q(j.M, first, n, j.acc + (second ? 2 : 0), j.q, cand, ncand, s));
  }
  const ScoreDesc sd = make_score(j, second);
  if (j.metric != DSES_METRIC_INLIER) {
    if (j.nn == DSES_NN_GRID)
      CK(launch_score_grid(sd, cand, ncand, n, s));
    else
      CK(launch_score_brute(sd, cand, ncand, n, s));
  }
  CK(launch_argmin(j.cost, j.M, j.N, j.metric, cand, ncand, n, 0, j.best, s));
}

// Euler boxes around the refine_top_k best first-pass candidates.
void stage_refine_grid(dses_ctx* c, Job& j) {
  cudaStream_t s = c->stream;
  const int n = (int)j.n_first;
  if (j.fused)
    CK(launch_keys_from_cost(j.cost, nullptr, nullptr, n, 0, j.keys, s));
  else
    CK(launch_keys_from_cost(j.cost, j.cand, j.n_cand, n, 0, j.keys, s));
  const int k = j.rtop;
  CK(launch_k_smallest(j.keys, n, j.fused ? nullptr : j.n_cand, k, j.ks_scratch, j.ksel, s));
  if (j.hopf_n > 0)
    CK(launch_euler_boxes_hopf(j.hopf_n, j.ksel, k, j.rK, j.rdr, j.rot_fine, s));
  else
    CK(launch_euler_boxes_keyed(j.rot, j.ksel, k, j.rK, j.rdr, j.rot_fine, s));
}

void stage_finalize(dses_ctx* c, std::vector<Job*>& jobs) {
  cudaStream_t s = c->stream;
  std::vector<FinalDesc> fd(jobs.size());
  for (size_t i = 0; i < jobs.size(); ++i) {
    Job& j = *jobs[i];
    fd[i].best = j.best;
    fd[i].acc = j.acc;
    fd[i].kv = j.kv;
    fd[i].Mout = j.M;
    fd[i].rot = j.rot;
    fd[i].rot_fine = j.rot_fine;
    fd[i].n_first = (uint32_t)j.n_first;
    fd[i].out_base = 0;
    fd[i].delta = j.delta;
    fd[i].result = j.res;
  }
  DevMem m;
  m.alloc(sizeof(FinalDesc) * fd.size(), s);
  CK(cudaMemcpyAsync(m.p, stage_put(c, fd.data(), sizeof(FinalDesc) * fd.size()), sizeof(FinalDesc) * fd.size(),
                     cudaMemcpyHostToDevice, s));
  CK(launch_finalize((const FinalDesc*)m.p, (int)fd.size(), s));
  m.release();
}

// Autotuner: the vote's launch shape for a problem-size bucket, chosen once
// per bucket by timing trial launches on an even-stride sample of the
// problem's own rotations (the trials rewrite only per-rotation values that
// the pass rewrites identically): first the points per thread (1, 2, 4, 8)
// with one rotation per work item, then, for that shape, the rotations per
// work item (1, 2, 4, 8, 16) on a sample holding at least 16 items per SM at
// the largest. Sets j.tile (capped per launch, see launch_pass) and returns
// the points per thread.
float time_vote_trial(dses_ctx* c, Job& j, const float* rot, int64_t n, int P, int tile) {
  check_culled_layout(j);
  std::vector<PassDesc> d{make_desc(j, P, false)};
  d[0].rot = rot;
  d[0].n_rot = (int)n;
  d[0].tile_rot = tile;
  d[0].votes_total = nullptr;  // a trial's votes are not the registration's
  int src_bytes = 0, blk_bytes = 0, list_bytes = 0;
  pass_staging(j.hist_bytes, j.N, block_bounds_pay(d[0]), j.sparse == 2, &src_bytes, &blk_bytes, &list_bytes);
  set_chunks(d[0], src_bytes);
  const int tiles = (int)((n + tile - 1) / tile);
  std::vector<int> tp{0, tiles}, rp{0, (int)n};
  DevMem m;
  m.alloc(4096, c->stream);
  char* base = (char*)m.p;
  CK(cudaMemcpyAsync(base, stage_put(c, d.data(), sizeof(PassDesc)), sizeof(PassDesc), cudaMemcpyHostToDevice,
                     c->stream));
  CK(cudaMemcpyAsync(base + 1024, stage_put(c, tp.data(), 8), 8, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(base + 2048, stage_put(c, rp.data(), 8), 8, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemsetAsync(base + 3072, 0, 4, c->stream));
  PassLaunch L;
  L.probs = (const PassDesc*)base;
  L.tile_prefix = (const int*)(base + 1024);
  L.rot_prefix = (const int*)(base + 2048);
  L.n_probs = 1;
  L.tile_rot = tile;
  L.work_counter = (int*)(base + 3072);
  L.hist_bytes = j.hist_bytes;
  L.src_bytes = src_bytes;
  L.blk_bytes = blk_bytes;
  L.list_bytes = list_bytes;
  L.padded = 0;
  for (int a = 0; a < 3; ++a) L.padded |= j.Ep[a] != j.E[a] ? 1 : 0;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaEventRecord(e0, c->stream));
  CK(launch_vote(L, P, j.sparse, std::min<int>(c->sms, tiles), c->stream));
  CK(cudaEventRecord(e1, c->stream));
  CK(cudaEventSynchronize(e1));
  float ms = 0;
  CK(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  m.release();
  return ms;
}

int pick_p(dses_ctx* c, Job& j) {
  // the culled vote has no 8-points-per-thread instance: the shape is settled
  // here, before any descriptor is built for it
  if (c->opt.points_per_thread > 0) {
    const int P = (int)c->opt.points_per_thread;
    if (j.sparse == 2) return P >= 4 ? 4 : 2;
    return j.sparse && P == 8 ? 4 : P;
  }
  std::vector<Job*> one{&j};
  if (!c->opt.autotune || j.n_first < 1) return choose_p(c, one);
  auto lg = [](int64_t v) { int b = 0; while ((1LL << b) < v) ++b; return b; };
  char key[96];
  snprintf(key, sizeof(key), "m%d n%d b%d r%d s%d u%d l%d", lg(j.T->m), lg(j.N),
           lg((int64_t)j.E[0] * j.E[1] * j.E[2]), lg(j.n_first), (int)j.sparse, j.u16, j.lanes);
  auto it = c->tuned.find(key);
  if (it != c->tuned.end()) {
    j.tile = it->second.second;
    return it->second.first;
  }
  // no trial launches inside a capture, nor in the serving worker (they
  // synchronise the device and would stall every request in flight): an
  // untuned bucket takes the heuristic shape there
  if (c->capturing || t_serving_worker) return choose_p(c, one);
  // an even-stride sample of the grid (its first rotations are one corner of
  // SO(3), which can favour another shape)
  auto sample = [&](int64_t want, DevMem& buf) -> std::pair<const float*, int64_t> {
    const int64_t n = std::min<int64_t>(j.n_first, want);
    const int64_t stride = j.n_first / n;
    if (stride <= 1) return {j.rot, n};
    buf.alloc(36 * (size_t)n, c->stream);
    CK(cudaMemcpy2DAsync(buf.p, 36, j.rot, 36 * (size_t)stride, 36, (size_t)n, cudaMemcpyDeviceToDevice,
                         c->stream));
    return {(const float*)buf.p, n};
  };
  DevMem s1, s2;
  const auto a = sample((int64_t)c->sms * 16, s1);
  float best_ms = 1e30f;
  int best_p = choose_p(c, one);
  for (int P : {1, 2, 4, 8}) {
    if ((j.sparse && P == 8) || (j.sparse == 2 && P == 1)) continue;
    const float ms = time_vote_trial(c, j, a.first, a.second, P, 1);
    if (ms < best_ms) {
      best_ms = ms;
      best_p = P;
    }
  }
  const auto b = sample((int64_t)c->sms * 16 * 16, s2);
  int best_tile = 1;
  best_ms = 1e30f;
  for (int tile : {1, 2, 4, 8, 16}) {
    if (tile > 1 && b.second / tile < (int64_t)c->sms * 4) break;  // too few items per SM to tell
    const float ms = time_vote_trial(c, j, b.first, b.second, best_p, tile);
    if (ms < best_ms * 0.99f) {  // a larger tile must win by 1%
      best_ms = ms;
      best_tile = tile;
    }
  }
  c->tuned[key] = {best_p, best_tile};
  j.tile = best_tile;
  return best_p;
}

// The whole pipeline for a set of jobs; results land in each job's device
// result slot. No host synchronisation inside (except autotuner trials).
void run_pipeline(dses_ctx* c, std::vector<Job*>& jobs) {
  c->last_p_mask = 0;
  c->last_tile_max = 0;
  for (auto* j : jobs) stage_setup(c, *j);
  // one persistent launch per (points-per-thread shape, culled mode): key
  // 4 P + mode (normally one launch)
  std::map<int, std::vector<PassPart>> first, fine;
  std::map<Job*, int> shape;
  for (auto* j : jobs) shape[j] = 4 * pick_p(c, *j) + j->sparse;
  for (auto* j : jobs) first[shape[j]].push_back({j, false, 0, j->n_first});
  for (auto& kv : first) launch_pass(c, kv.second, kv.first / 4);
  for (auto* j : jobs) stage_candidates(c, *j, false);
  for (auto* j : jobs)
    if (j->rtop > 0) {
      stage_refine_grid(c, *j);
      fine[shape[j]].push_back({j, true, 0, j->n_fine});
    }
  for (auto& kv : fine) launch_pass(c, kv.second, kv.first / 4);
  for (auto* j : jobs)
    if (j->rtop > 0) stage_candidates(c, *j, true);
  stage_finalize(c, jobs);
}

void collect_timing(dses_ctx* c);

// ---------------------------------------------------------------------------
// Rotation sharding of one registration. Algorithm 2 treats every rotation on
// its own, so shard `rank` of `world` runs the contiguous ranges of the grid
// and of the second pass that dses_shard_range gives it; the shards meet only
// where the algorithm reduces over all rotations (exchange.h): M* for the q
// filter, the top-k keys, the second pass's centres and the final argmin. An
// exchange is an all-gather of a few bytes per shard through the caller's
// callback; without one (dses_register_shard) no reduction may cross shards.

struct Exchange {
  dses_allgather_fn fn = nullptr;
  void* user = nullptr;
  int world = 1;
  template <class T>
  std::vector<T> all(const T* send, size_t count) {
    std::vector<T> recv(count * (size_t)world);
    if (fn(user, send, (int64_t)(sizeof(T) * count), recv.data()) != 0)
      throw Error{DSES_ERR_EXCHANGE, "the all-gather callback of a sharded registration failed"};
    return recv;
  }
};

// Candidate stage of one pass of a shard: the q filter against the M* of all
// shards, or the top-k by (M desc, index asc) over all shards; then scoring
// and the argmin of the shard's own candidates.
void shard_candidates(dses_ctx* c, Job& j, bool second, const ShardMap& map, Exchange* X) {
  if (j.fused) return;
  cudaStream_t s = c->stream;
  const uint32_t first = second ? (uint32_t)j.n_first : 0;
  const int n = (int)(second ? j.n_fine : j.n_first);
  uint32_t* cand = j.cand + first;
  uint32_t* ncand = j.n_cand + (second ? 1 : 0);
  uint32_t* acc = j.acc + (second ? 2 : 0);
  if (j.topk > 0) {
    const int k = j.topk;
    std::vector<uint64_t> mine((size_t)k, kPadKey);
    if (n > 0) {
      CK(launch_keys_from_M(j.M, first, n, 0, j.keys, s));
      CK(launch_k_smallest(j.keys, n, nullptr, k, j.ks_scratch, j.ksel, s));
      CK(cudaMemcpyAsync(mine.data(), j.ksel, 8 * (size_t)k, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      for (auto& key : mine) key = key_to_global(key, map);
    }
    const std::vector<uint64_t> glob = X ? merge_k_smallest(X->all(mine.data(), (size_t)k).data(), X->world, k) : mine;
    std::vector<uint32_t> slots;
    for (uint64_t key : glob) {
      uint32_t l = 0;
      if (key != kPadKey && map.to_local((uint32_t)(key & 0xffffffffull), &l)) slots.push_back(l);
    }
    const uint32_t cnt = (uint32_t)slots.size();
    if (cnt) CK(cudaMemcpyAsync(cand, slots.data(), 4 * (size_t)cnt, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ncand, &cnt, 4, cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
  } else {
    if (X && j.q > 0) {  // M* over all shards (with q = 0 every rotation passes)
      uint32_t m = 0;
      if (n > 0) {
        CK(cudaMemcpyAsync(&m, acc, 4, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
      }
      m = merge_max(X->all(&m, 1).data(), X->world);
      CK(cudaMemcpyAsync(acc, &m, 4, cudaMemcpyHostToDevice, s));
      CK(cudaStreamSynchronize(s));
    }
    if (n > 0) CK(launch_select_q(j.M, first, n, acc, j.q, cand, ncand, s));
  }
  if (n < 1) return;
  const ScoreDesc sd = make_score(j, second);
  if (j.metric != DSES_METRIC_INLIER) {
    if (j.nn == DSES_NN_GRID)
      CK(launch_score_grid(sd, cand, ncand, n, s));
    else
      CK(launch_score_brute(sd, cand, ncand, n, s));
  }
  CK(launch_argmin(j.cost, j.M, j.N, j.metric, cand, ncand, n, 0, j.best, s));
}

// The second pass's Euler boxes (all of them, every shard the same): centred
// on the refine_top_k best first-pass candidates by (cost, index) over all
// shards, picked from the whole first-pass grid by global index.
void shard_refine_grid(dses_ctx* c, Job& j, const ShardMap& map, Exchange* X, const float* rot_full,
                       float* fine_full) {
  cudaStream_t s = c->stream;
  const int k = j.rtop;
  const int n = (int)j.n_first;
  std::vector<uint64_t> mine((size_t)k, kPadKey);
  if (n > 0) {
    if (j.fused)
      CK(launch_keys_from_cost(j.cost, nullptr, nullptr, n, 0, j.keys, s));
    else
      CK(launch_keys_from_cost(j.cost, j.cand, j.n_cand, n, 0, j.keys, s));
    CK(launch_k_smallest(j.keys, n, j.fused ? nullptr : j.n_cand, k, j.ks_scratch, j.ksel, s));
    CK(cudaMemcpyAsync(mine.data(), j.ksel, 8 * (size_t)k, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (auto& key : mine) key = key_to_global(key, map);
  }
  const std::vector<uint64_t> glob = X ? merge_k_smallest(X->all(mine.data(), (size_t)k).data(), X->world, k) : mine;
  CK(cudaMemcpyAsync(j.ksel, glob.data(), 8 * (size_t)k, cudaMemcpyHostToDevice, s));
  if (j.hopf_n > 0)
    CK(launch_euler_boxes_hopf(j.hopf_n, j.ksel, k, j.rK, j.rdr, fine_full, s));
  else
    CK(launch_euler_boxes_keyed(rot_full, j.ksel, k, j.rK, j.rdr, fine_full, s));
  CK(cudaStreamSynchronize(s));
}

// One shard of a registration. Returns the shard's own result (rotation index
// in the whole registration); with an exchange, every shard receives the
// combined result of all shards instead.
dses_status run_sharded(dses_ctx* c, const dses_problem* problem, int rank, int world, Exchange* X,
                        dses_result* out) {
  Job j;
  resolve(c, problem, j);
  plan(c, j);
  const int64_t n1 = j.n_first, nf = j.n_fine;
  ShardMap map;
  int64_t e1 = 0, e2 = 0;
  dses_shard_range(n1, rank, world, &map.b1, &e1);
  dses_shard_range(nf, rank, world, &map.b2, &e2);
  map.n1 = e1 - map.b1;
  map.n1_total = n1;
  map.n2 = e2 - map.b2;
  cudaStream_t s = c->stream;
  std::vector<Job*> jobs{&j};
  c->cur_stage = &c->stage;
  c->stage.reserve(stage_bytes(jobs));  // sized for the whole grid (an explicit one is uploaded whole)
  c->stage.used = 0;
  // the whole first-pass grid on the device: the shard's range is a slice of
  // it, and the second pass picks its centres from it by global index
  DevMem full1, fine;
  const float* rot_full = nullptr;
  const dses_rotation_grid& g = problem->grid;
  if (g.kind == DSES_GRID_HOPF) {
    rot_full = hopf_grid(c, g.hopf_n);
  } else {
    full1.alloc(align256(36 * (size_t)n1) + 256, s);
    if (g.kind == DSES_GRID_EULER_BOX) {
      double* R0 = (double*)((char*)full1.p + align256(36 * (size_t)n1));
      CK(cudaMemcpyAsync(R0, stage_put(c, g.R0, 72), 72, cudaMemcpyHostToDevice, s));
      CK(launch_euler_box_single(R0, g.K, g.delta_r, (float*)full1.p, s));
    } else {
      if (!finite3(g.explicit_R, 3 * g.n_explicit)) invalid("explicit rotations have a non-finite entry");
      CK(cudaMemcpyAsync(full1.p, stage_put(c, g.explicit_R, 36 * (size_t)n1), 36 * (size_t)n1,
                         cudaMemcpyHostToDevice, s));
    }
    rot_full = (const float*)full1.p;
  }
  j.n_first = map.n1;
  j.n_fine = map.n2;
  j.n_total = j.n_first + j.n_fine;
  stage_inputs(c, j);
  j.rot = rot_full + 9 * map.b1;
  stage_reset(c, j);
  const int P = pick_p(c, j);
  if (j.n_first > 0) launch_pass(c, {{&j, false, 0, j.n_first}}, P);
  shard_candidates(c, j, false, map, X);
  if (j.rtop > 0) {
    fine.alloc(36 * (size_t)nf + 256, s);
    shard_refine_grid(c, j, map, X, rot_full, (float*)fine.p);
    j.rot_fine = (float*)fine.p + 9 * map.b2;
    if (j.n_fine > 0) launch_pass(c, {{&j, true, 0, j.n_fine}}, P);
    shard_candidates(c, j, true, map, X);
  }
  stage_finalize(c, jobs);
  dses_result r;
  CK(cudaMemcpyAsync(&r, j.res, sizeof(r), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  collect_timing(c);
  if (r.rot_index >= 0) r.rot_index = map.to_global((uint32_t)r.rot_index);
  if (!X) {
    *out = r;
    return (dses_status)r.status;
  }
  const std::vector<dses_result> parts = X->all(&r, 1);
  const dses_status st = dses_combine_results(parts.data(), world, out);
  if (st != DSES_OK && st != DSES_ERR_NO_CANDIDATE) throw Error{DSES_ERR_EXCHANGE, "a shard's result was an error"};
  return st;
}

// ---------------------------------------------------------------------------
// serving: continuous batching. Admitted requests are processed in
// iterations; each iteration is one persistent pass launch over the next
// slice of rotations of every active request. A request whose first pass
// completes runs its candidate stage, second pass and finaliser, and leaves;
// queued requests join at the next iteration when slots and memory allow.

}  // namespace

namespace {

struct Request {
  dses_problem prob;
  std::vector<float> src;          // owned copy of the source cloud
  std::vector<float> explicit_R;   // owned copy of an explicit grid
  Job job;
  int64_t next = 0;                // next first-pass rotation to schedule
  bool admitted = false;
  std::atomic<int> state{0};       // 0 queued, 1 running, 2 done
  dses_result result;
  dses_status status = DSES_OK;
  std::string err;
  dses_result* host_res = nullptr;  // pinned
};

void fail_request(Request& r, const Error& e) {
  r.status = e.code;
  r.err = e.msg;
  std::memset(&r.result, 0, sizeof(r.result));
  r.result.status = e.code;
  r.result.rot_index = -1;
}

void worker_loop(dses_ctx* c) {
  cudaSetDevice(c->device);
  t_serving_worker = true;
  std::vector<std::shared_ptr<Request>> active;
  size_t mem_used = 0;
  // Iterations in flight (at most two): the host admits requests and builds and
  // launches the next iteration while the device runs the current one. Each
  // iteration records an event; once it has completed, the requests that
  // finished in it are retired. Iterations alternate between two pinned stages,
  // so a stage is refilled only after the iteration that read it has completed.
  struct Flight {
    cudaEvent_t ev = nullptr;
    cudaEvent_t start = nullptr;  // where the iteration's device work begins
    std::vector<std::shared_ptr<Request>> done;
  };
  std::deque<Flight> flights;
  int cur = 0;
  auto release = [&](const std::shared_ptr<Request>& r) {
    mem_used -= std::min(mem_used, job_bytes(r->job));
    {
      std::lock_guard<std::recursive_mutex> g(c->mu);
      r->job.mem.release();  // stream-ordered: after the work already queued
    }
    r->job.T->inflight--;
    r->state = 2;  // visible to dses_poll only now
  };
  auto retire_oldest = [&]() {
    Flight f = flights.front();
    flights.pop_front();
    const cudaError_t e = cudaEventSynchronize(f.ev);
    if (e == cudaSuccess && f.start) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, f.start, f.ev) == cudaSuccess) {
        std::lock_guard<std::recursive_mutex> g(c->mu);
        c->serve_busy_ns += (int64_t)(ms * 1e6);
        c->serve_iterations += 1;
      }
    }
    cudaGetLastError();
    if (f.start) cudaEventDestroy(f.start);
    cudaEventDestroy(f.ev);
    for (auto& r : f.done) {
      if (e != cudaSuccess) {
        fail_request(*r, Error{DSES_ERR_CUDA, std::string("serving iteration: ") + cudaGetErrorString(e)});
      } else {
        r->result = *r->host_res;
        r->status = (dses_status)r->result.status;
      }
      release(r);
      const auto it = std::find(active.begin(), active.end(), r);
      if (it != active.end()) active.erase(it);
    }
  };
  auto schedulable = [&]() {
    for (auto& r : active) {
      const int st = r->state.load();
      if (st == 0 || (st == 1 && r->next < r->job.n_first)) return true;
    }
    return false;
  };
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(c->smu);
      if (active.empty() && flights.empty()) c->scv.wait(lk, [&] { return c->stop || !c->queue.empty(); });
      if (c->stop && active.empty() && flights.empty()) return;
      // admission: batch slots and device-memory budget
      while (!c->queue.empty() && (int64_t)active.size() < c->opt.serve_max_batch) {
        auto r = c->queue.front();
        const size_t need = job_bytes(r->job);
        if (!active.empty() && mem_used + need > (size_t)c->opt.serve_mem_budget) break;
        c->queue.pop_front();
        r->admitted = true;
        mem_used += need;
        active.push_back(r);
      }
    }
    if (schedulable()) {
      std::lock_guard<std::recursive_mutex> g(c->mu);  // taken after smu is released (submit nests smu in mu)
      c->serve_max_active = std::max<int64_t>(c->serve_max_active, (int64_t)active.size());
      Flight f;
      bool launched = false;
      {
        std::vector<Job*> all;
        for (auto& r : active) all.push_back(&r->job);
        c->cur_stage = &c->serve_stage[cur];
        try {
          c->serve_stage[cur].reserve(2 * stage_bytes(all));
        } catch (const Error& e) {
          for (auto& r : active)
            if (r->state.load() < 2) {
              fail_request(*r, e);
              r->state = 4;  // failed, to be released below
            }
        }
        c->serve_stage[cur].used = 0;
      }
      if (cudaEventCreate(&f.start) == cudaSuccess) {
        if (cudaEventRecord(f.start, c->stream) != cudaSuccess) {
          cudaEventDestroy(f.start);
          f.start = nullptr;
        }
      } else {
        f.start = nullptr;
      }
      cudaGetLastError();
      // set up newly admitted requests
      for (auto& r : active) {
        if (r->state.load() != 0) continue;
        try {
          stage_setup(c, r->job);
          r->state = 1;
        } catch (const Error& e) {
          fail_request(*r, e);
          r->state = 4;
        }
      }
      // one iteration: requests in admission order take rotations until the
      // iteration's pair-vote budget is spent or one of them completes its
      // first pass (the oldest request finishes first);
      // one launch per (points-per-thread shape, culled mode): key 4 P + mode
      std::map<int, std::vector<PassPart>> parts;
      const int64_t slice = std::max<int64_t>(1, c->opt.serve_tile_rotations);
      double budget = (double)c->opt.serve_iter_pairs;
      try {
        for (auto& r : active) {
          if (r->state.load() != 1 || r->next >= r->job.n_first) continue;
          if (budget <= 0) break;
          const double per_rot = (double)r->job.N * (double)r->job.T->m;
          const int64_t want = std::max<int64_t>(1, (int64_t)(budget / per_rot));
          const int64_t a0 = r->next, b0 = std::min({r->job.n_first, a0 + slice, a0 + want});
          parts[4 * pick_p(c, r->job) + r->job.sparse].push_back({&r->job, false, a0, b0});
          r->next = b0;
          budget -= (double)(b0 - a0) * per_rot;
          // a request that completes its first pass here ends the iteration:
          // its result is then ready when its own work is, and the next
          // request starts in the following iteration (already in flight)
          if (b0 == r->job.n_first) break;
        }
        for (auto& kv : parts) launch_pass(c, kv.second, kv.first / 4);
        std::vector<Job*> fin;
        std::map<int, std::vector<PassPart>> fine;
        for (auto& r : active) {
          if (r->state.load() != 1 || r->next < r->job.n_first) continue;
          stage_candidates(c, r->job, false);
          if (r->job.rtop > 0) {
            stage_refine_grid(c, r->job);
            fine[4 * pick_p(c, r->job) + r->job.sparse].push_back({&r->job, true, 0, r->job.n_fine});
          }
          fin.push_back(&r->job);
        }
        for (auto& kv : fine) {
          launch_pass(c, kv.second, kv.first / 4);
          for (auto& pp : kv.second) stage_candidates(c, *pp.job, true);
        }
        if (!fin.empty()) stage_finalize(c, fin);
        for (auto& r : active) {
          if (r->state.load() != 1 || r->next < r->job.n_first) continue;
          CK(cudaMemcpyAsync(r->host_res, r->job.res, sizeof(dses_result), cudaMemcpyDeviceToHost, c->stream));
          r->state = 3;  // finishing on the device
          f.done.push_back(r);
        }
        CK(cudaEventCreate(&f.ev));
        CK(cudaEventRecord(f.ev, c->stream));
        launched = true;
      } catch (const Error& e) {
        if (f.ev) cudaEventDestroy(f.ev);
        f.ev = nullptr;
        if (f.start) cudaEventDestroy(f.start);
        f.start = nullptr;
        // the stream may hold this iteration's work: let it drain first
        cudaStreamSynchronize(c->stream);
        cudaGetLastError();
        for (auto& r : active)
          if (r->state.load() == 1 || r->state.load() == 3) {
            fail_request(*r, e);
            r->state = 4;
          }
      }
      if (launched) {
        flights.push_back(f);
        cur ^= 1;
      }
      // release requests that failed in this iteration
      for (size_t i = 0; i < active.size();) {
        if (active[i]->state.load() == 4) {
          auto r = active[i];
          release(r);
          for (auto& fl : flights) fl.done.erase(std::remove(fl.done.begin(), fl.done.end(), r), fl.done.end());
          active.erase(active.begin() + (long)i);
        } else {
          ++i;
        }
      }
    }
    // retire: keep at most two iterations in flight; drain when nothing is left to launch
    if (!flights.empty() && (flights.size() >= 2 || !schedulable())) retire_oldest();
  }
}

// ---------------------------------------------------------------------------
// CUDA graphs for repeated batches. A batch whose problems have the same
// shapes, targets, grids and parameters as an earlier call is captured once
// (every upload comes from the graph's own pinned stage, every scratch buffer
// is a stream-ordered allocation inside the graph) and then replayed: the new
// host source clouds are copied into the stage and the graph is launched.

std::string graph_key(dses_ctx* c, const std::vector<Job*>& jobs) {
  if (c->opt.record_timing) return std::string();
  std::string k;
  char buf[512];
  snprintf(buf, sizeof(buf), "o%lld,%lld,%lld,%lld,%lld,%lld,%lld|", (long long)c->opt.hist_mode,
           (long long)c->opt.hist_budget, (long long)c->opt.points_per_thread, (long long)c->opt.fuse_score,
           (long long)c->opt.tile_rotations, (long long)c->opt.vote_sparse, (long long)c->opt.autotune);
  k += buf;
  for (auto* j : jobs) {
    const dses_problem& pb = *j->prob;
    if (pb.grid.kind == DSES_GRID_EXPLICIT) return std::string();  // grid contents not tracked
    const dses_params& P = pb.params;
    // the target by its uid, not its address: a destroyed target's address can
    // come back for a new one while graphs captured on the old one remain
    snprintf(buf, sizeof(buf), "T%llu,%d,%p,%lld,%d,%d,%d,%.17g|", (unsigned long long)j->T->uid, pb.src_is_device,
             pb.src_is_device ? (const void*)pb.src : nullptr, (long long)pb.n_src, pb.grid.kind, pb.grid.hopf_n,
             pb.grid.K, pb.grid.delta_r);
    k += buf;
    for (int a = 0; a < 9; ++a) {
      snprintf(buf, sizeof(buf), "%.17g,", pb.grid.R0[a]);
      k += buf;
    }
    snprintf(buf, sizeof(buf), "|%d,%a,%a,%a,%a,%a,%a,%a,%a,%a,%a,%a,%d,%d,%d,%d,%d,%.17g;", P.metric, P.epsilon,
             P.delta_t, P.tau, P.huber_h, P.p, P.t_center[0], P.t_center[1], P.t_center[2], P.t_half[0],
             P.t_half[1], P.t_half[2], P.q_milli, P.top_k, P.nn_mode, P.refine_top_k, P.refine_K, P.refine_delta_r);
    k += buf;
  }
  return k;
}

void free_graph(dses_ctx::GraphEntry& e) {
  if (e.exec) cudaGraphExecDestroy(e.exec);
  e.exec = nullptr;
  e.stage.release();
  if (e.res) cudaFreeHost(e.res);
  e.res = nullptr;
}

dses_status replay_graph(dses_ctx* c, dses_ctx::GraphEntry& e, std::vector<Job*>& jobs, dses_result* out) {
  for (size_t i = 0; i < jobs.size(); ++i)
    if (!jobs[i]->prob->src_is_device)
      std::memcpy(e.stage.host + e.src_slots[i].first, jobs[i]->prob->src, e.src_slots[i].second);
  CK(cudaGraphLaunch(e.exec, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  dses_status st = DSES_OK;
  for (size_t i = 0; i < jobs.size(); ++i) {
    out[i] = e.res[i];
    if (st == DSES_OK && out[i].status != DSES_OK) st = (dses_status)out[i].status;
  }
  return st;
}

dses_status capture_and_replay(dses_ctx* c, const std::string& key, std::vector<Job*>& jobs, dses_result* out) {
  if (c->graphs.size() >= 8) {  // bounded cache: drop the oldest-keyed entry
    free_graph(c->graphs.begin()->second);
    c->graphs.erase(c->graphs.begin());
  }
  dses_ctx::GraphEntry e;
  e.stage.reserve(stage_bytes(jobs));
  CK(cudaMallocHost((void**)&e.res, sizeof(dses_result) * jobs.size()));
  c->cur_stage = &e.stage;
  e.stage.used = 0;
  cudaStream_t s = c->stream;
  CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
  c->capturing = true;
  cudaGraph_t g = nullptr;
  try {
    run_pipeline(c, jobs);
    for (size_t i = 0; i < jobs.size(); ++i)
      CK(cudaMemcpyAsync(e.res + i, jobs[i]->res, sizeof(dses_result), cudaMemcpyDeviceToHost, s));
    for (auto* j : jobs) j->mem.release();
  } catch (...) {
    c->capturing = false;
    cudaStreamEndCapture(s, &g);
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    free_graph(e);
    throw;
  }
  c->capturing = false;
  CK(cudaStreamEndCapture(s, &g));
  const cudaError_t ie = cudaGraphInstantiate(&e.exec, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) {
    cudaGetLastError();
    free_graph(e);
    throw Error{DSES_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ie)};
  }
  e.src_slots.resize(jobs.size());
  for (size_t i = 0; i < jobs.size(); ++i) e.src_slots[i] = {jobs[i]->src_stage_off, 12 * (size_t)jobs[i]->N};
  auto& slot = c->graphs[key];
  slot = e;
  e.exec = nullptr;
  e.res = nullptr;
  e.stage.host = nullptr;
  return replay_graph(c, slot, jobs, out);
}

// ---------------------------------------------------------------------------
// C ABI plumbing

template <class F>
dses_status guard(dses_ctx* c, F&& f) {
  try {
    f();
    return DSES_OK;
  } catch (const Error& e) {
    if (c) c->err = e.msg;
    return e.code;
  } catch (const std::bad_alloc&) {
    if (c) c->err = "host allocation failed";
    return DSES_ERR_OOM;
  } catch (...) {
    if (c) c->err = "unexpected C++ exception";
    return DSES_ERR_CUDA;
  }
}

// Sum the recorded pass-launch durations (after the stream has drained).
void collect_timing(dses_ctx* c) {
  if (c->pass_events.empty()) return;
  double vote_ms = 0, count_ms = 0;
  for (auto& e : c->pass_events) {
    float a = 0, b = 0;
    if (cudaEventElapsedTime(&a, e.start, e.voted) == cudaSuccess) vote_ms += a;
    if (cudaEventElapsedTime(&b, e.voted, e.counted) == cudaSuccess) count_ms += b;
    cudaEventDestroy(e.start);
    cudaEventDestroy(e.voted);
    cudaEventDestroy(e.counted);
  }
  c->pass_ns = (int64_t)(vote_ms * 1e6);
  c->count_ns = (int64_t)(count_ms * 1e6);
  c->pass_launches = (int64_t)c->pass_events.size();
  c->pass_events.clear();
}

dses_status finish_results(dses_ctx* c, std::vector<Job*>& jobs, dses_result* out) {
  if (c->pinned_cap < jobs.size()) {
    if (c->pinned_res) cudaFreeHost(c->pinned_res);
    c->pinned_res = nullptr;
    c->pinned_cap = 0;
    CK(cudaMallocHost(&c->pinned_res, sizeof(dses_result) * std::max<size_t>(jobs.size(), 64)));
    c->pinned_cap = std::max<size_t>(jobs.size(), 64);
  }
  dses_result* pinned = c->pinned_res;
  for (size_t i = 0; i < jobs.size(); ++i)
    CK(cudaMemcpyAsync(pinned + i, jobs[i]->res, sizeof(dses_result), cudaMemcpyDeviceToHost, c->stream));
  std::vector<unsigned long long> votes(jobs.size(), 0);
  for (size_t i = 0; i < jobs.size(); ++i)
    CK(cudaMemcpyAsync(&votes[i], jobs[i]->best + 1, 8, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->votes_total = 0;
  for (auto v : votes) c->votes_total += (int64_t)v;
  c->vote_sparse_jobs = 0;
  for (auto* j : jobs) c->vote_sparse_jobs += j->sparse ? 1 : 0;
  c->vote_paired_jobs = 0;
  for (auto* j : jobs) c->vote_paired_jobs += j->sparse == 2 ? 1 : 0;
  collect_timing(c);
  dses_status st = DSES_OK;
  for (size_t i = 0; i < jobs.size(); ++i) {
    out[i] = pinned[i];
    if (st == DSES_OK && out[i].status != DSES_OK) st = (dses_status)out[i].status;
  }
  return st;
}

}  // namespace

extern "C" {

dses_status dses_create(int device, void* cuda_stream, dses_ctx** out) {
  if (!out) return DSES_ERR_INVALID_ARG;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return DSES_ERR_INVALID_ARG;
  }
  dses_ctx* c = new (std::nothrow) dses_ctx();
  if (!c) return DSES_ERR_OOM;
  c->device = device;
  dses_status st = guard(c, [&] {
    CK(cudaSetDevice(device));
    CK(cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device));
    if (cuda_stream) {
      c->stream = (cudaStream_t)cuda_stream;
    } else {
      CK(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
      c->own_stream = true;
    }
    cudaMemPool_t pool;
    CK(cudaDeviceGetDefaultMemPool(&pool, device));
    uint64_t thr = UINT64_MAX;
    CK(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
  });
  if (st != DSES_OK) {
    delete c;
    return st;
  }
  *out = c;
  return DSES_OK;
}

static void stop_worker(dses_ctx* c) {
  if (!c->worker_started) return;
  {
    std::lock_guard<std::mutex> lk(c->smu);
    c->stop = true;
  }
  c->scv.notify_all();
  c->worker.join();
  c->worker_started = false;
}

static void free_target(dses_target* T) {
  if (T->Y) cudaFree(T->Y);
  if (T->Ym) cudaFree(T->Ym);
  if (T->gbox) cudaFree(T->gbox);
  if (T->gbox2) cudaFree(T->gbox2);
  if (T->D) cudaFree(T->D);
  if (T->D4) cudaFree(T->D4);
  for (auto& kv : T->cells) {
    cudaFree(kv.second.start);
    cudaFree(kv.second.sorted);
  }
  delete T;
}

dses_status dses_destroy(dses_ctx* c) {
  if (!c) return DSES_ERR_INVALID_ARG;
  stop_worker(c);
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  for (auto* chunk : c->res_chunks) cudaFreeHost(chunk);
  for (auto* T : c->targets) free_target(T);
  for (auto& h : c->hopf) cudaFree(h.second);
  if (c->pinned_res) cudaFreeHost(c->pinned_res);
  for (auto& g : c->graphs) free_graph(g.second);
  c->stage.release();
  c->serve_stage[0].release();
  c->serve_stage[1].release();
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
  return DSES_OK;
}

dses_status dses_create_target(dses_ctx* c, const float* xyz, int64_t m, int32_t ptr_is_device, float grid_cap,
                               int32_t grid_res, dses_target** out) {
  if (!c || !out) return DSES_ERR_INVALID_ARG;
  std::lock_guard<std::recursive_mutex> g(c->mu);
  *out = nullptr;
  return guard(c, [&] {
    if (!xyz || m < 1 || m > (1 << 24)) invalid("target needs 1 <= m <= 2^24 points");
    const int G = grid_res == 0 ? 128 : grid_res;
    if (G < 8 || G > 512) invalid("grid_res must be in [8, 512]");
    if (!(grid_cap > 0) || !std::isfinite(grid_cap)) invalid("grid_cap must be positive and finite");
    set_device(c);
    std::unique_ptr<dses_target> T(new dses_target());
    T->ctx = c;
    T->uid = c->next_target_uid++;
    T->m = (int)m;
    T->host.resize(3 * (size_t)m);
    if (ptr_is_device) {
      CK(cudaMemcpyAsync(T->host.data(), xyz, 12 * (size_t)m, cudaMemcpyDeviceToHost, c->stream));
      CK(cudaStreamSynchronize(c->stream));
    } else {
      std::memcpy(T->host.data(), xyz, 12 * (size_t)m);
    }
    if (!finite3(T->host.data(), m)) invalid("target cloud has a non-finite coordinate");
    for (int a = 0; a < 3; ++a) {
      T->bbmin[a] = T->bbmax[a] = T->host[a];
      for (int64_t j = 1; j < m; ++j) {
        T->bbmin[a] = std::min(T->bbmin[a], T->host[3 * j + a]);
        T->bbmax[a] = std::max(T->bbmax[a], T->host[3 * j + a]);
      }
    }
    float* raw = nullptr;
    CK(cudaMalloc(&T->Y, sizeof(float4) * (size_t)m));
    DevMem tmp;
    tmp.alloc(12 * (size_t)m, c->stream);
    raw = (float*)tmp.p;
    CK(cudaMemcpyAsync(raw, T->host.data(), 12 * (size_t)m, cudaMemcpyHostToDevice, c->stream));
    CK(launch_pack_points(raw, (int)m, T->Y, c->stream));
    tmp.release();
    // truncated distance grid: h = (extent + 2 cap)/(G - 2), origin min - cap - h
    T->G = G;
    T->gcap = grid_cap;
    for (int a = 0; a < 3; ++a) {
      const double h = ((double)T->bbmax[a] - T->bbmin[a] + 2.0 * grid_cap) / (double)(G - 2);
      T->gh[a] = (float)h;
      T->glo[a] = (float)((double)T->bbmin[a] - grid_cap - h);
    }
    build_vote_groups(c, T.get());
    CK(cudaMalloc(&T->D, sizeof(float) * (size_t)G * G * G));
    CK(cudaMalloc(&T->D4, sizeof(float4) * (size_t)G * G * G));
    CK(launch_dist_grid(T->Y, (int)m, G, T->glo, T->gh, grid_cap, T->D, T->D4, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->targets.push_back(T.get());
    *out = T.release();
  });
}

dses_status dses_destroy_target(dses_ctx* c, dses_target* T) {
  if (!c || !T) return DSES_ERR_INVALID_ARG;
  std::lock_guard<std::recursive_mutex> g(c->mu);
  return guard(c, [&] {
    auto it = std::find(c->targets.begin(), c->targets.end(), T);
    if (it == c->targets.end()) invalid("unknown target");
    if (T->inflight.load() > 0) invalid("target is still used by submitted requests");
    set_device(c);
    CK(cudaStreamSynchronize(c->stream));
    // drop the captured graphs (and capture counters) that read this target
    const std::string tok = "T" + std::to_string((unsigned long long)T->uid) + ",";
    for (auto g = c->graphs.begin(); g != c->graphs.end();) {
      if (g->first.find(tok) != std::string::npos) {
        free_graph(g->second);
        g = c->graphs.erase(g);
      } else {
        ++g;
      }
    }
    for (auto g = c->graph_seen.begin(); g != c->graph_seen.end();)
      g = g->first.find(tok) != std::string::npos ? c->graph_seen.erase(g) : std::next(g);
    c->targets.erase(it);
    free_target(T);
  });
}

dses_status dses_register_batch(dses_ctx* c, const dses_problem* problems, int32_t n, dses_result* out) {
  if (!c) return DSES_ERR_INVALID_ARG;
  std::lock_guard<std::recursive_mutex> g(c->mu);
  dses_status st = DSES_OK;
  dses_status gs = guard(c, [&] {
    if (!problems || !out || n < 1) invalid("batch needs problems, out and n >= 1");
    set_device(c);
    std::vector<std::unique_ptr<Job>> owned;
    std::vector<Job*> jobs;
    for (int i = 0; i < n; ++i) {
      owned.emplace_back(new Job());
      resolve(c, &problems[i], *owned.back());
      plan(c, *owned.back());
      jobs.push_back(owned.back().get());
    }
    const std::string key = c->opt.use_graphs ? graph_key(c, jobs) : std::string();
    if (!key.empty() && c->graphs.count(key)) {
      st = replay_graph(c, c->graphs[key], jobs, out);
    } else if (!key.empty() && ++c->graph_seen[key] >= 2) {
      st = capture_and_replay(c, key, jobs, out);
    } else {
      c->cur_stage = &c->stage;
      c->stage.reserve(stage_bytes(jobs));
      c->stage.used = 0;
      run_pipeline(c, jobs);
      st = finish_results(c, jobs, out);
    }
    if (st != DSES_OK) c->err = "a problem found no candidate (no pair voted inside its translation box)";
  });
  return gs != DSES_OK ? gs : st;
}

dses_status dses_register(dses_ctx* c, const dses_problem* problem, dses_result* out) {
  return dses_register_batch(c, problem, 1, out);
}

dses_status dses_debug_per_rotation(dses_ctx* c, const dses_problem* problem, int32_t* k_star, uint32_t* votes,
                                    uint32_t* inliers, float* cost, dses_result* out) {
  if (!c) return DSES_ERR_INVALID_ARG;
  std::lock_guard<std::recursive_mutex> g(c->mu);
  dses_status st = DSES_OK;
  dses_status gs = guard(c, [&] {
    set_device(c);
    Job job;
    resolve(c, problem, job);
    plan(c, job);
    std::vector<Job*> jobs{&job};
    c->cur_stage = &c->stage;
    c->stage.reserve(stage_bytes(jobs));
    c->stage.used = 0;
    run_pipeline(c, jobs);
    const size_t n = (size_t)job.n_total;
    std::vector<int4> kv(n);
    std::vector<uint32_t> M(n);
    std::vector<float> C(n);
    CK(cudaMemcpyAsync(kv.data(), job.kv, 16 * n, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(M.data(), job.M, 4 * n, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(C.data(), job.cost, 4 * n, cudaMemcpyDeviceToHost, c->stream));
    dses_result r;
    st = finish_results(c, jobs, &r);
    for (size_t i = 0; i < n; ++i) {
      if (k_star) {
        k_star[3 * i] = kv[i].x;
        k_star[3 * i + 1] = kv[i].y;
        k_star[3 * i + 2] = kv[i].z;
      }
      if (votes) votes[i] = (uint32_t)kv[i].w;
      if (inliers) inliers[i] = M[i];
      if (cost) cost[i] = C[i];
    }
    if (out) *out = r;
  });
  return gs != DSES_OK ? gs : st;
}

dses_status dses_debug_per_rotation_batch(dses_ctx* c, const dses_problem* problems, int32_t n,
                                          int32_t* const* k_star, uint32_t* const* votes, uint32_t* const* inliers,
                                          float* const* cost, dses_result* out) {
  if (!c) return DSES_ERR_INVALID_ARG;
  std::lock_guard<std::recursive_mutex> g(c->mu);
  dses_status st = DSES_OK;
  dses_status gs = guard(c, [&] {
    if (!problems || !out || n < 1) invalid("batch needs problems, out and n >= 1");
    set_device(c);
    std::vector<std::unique_ptr<Job>> owned;
    std::vector<Job*> jobs;
    for (int i = 0; i < n; ++i) {
      owned.emplace_back(new Job());
      resolve(c, &problems[i], *owned.back());
      plan(c, *owned.back());
      jobs.push_back(owned.back().get());
    }
    c->cur_stage = &c->stage;
    c->stage.reserve(stage_bytes(jobs));
    c->stage.used = 0;
    run_pipeline(c, jobs);  // the batch's persistent launches, as dses_register_batch runs them
    std::vector<std::vector<int4>> kv(jobs.size());
    std::vector<std::vector<uint32_t>> M(jobs.size());
    std::vector<std::vector<float>> C(jobs.size());
    for (size_t b = 0; b < jobs.size(); ++b) {
      const size_t m = (size_t)jobs[b]->n_total;
      kv[b].resize(m);
      M[b].resize(m);
      C[b].resize(m);
      CK(cudaMemcpyAsync(kv[b].data(), jobs[b]->kv, 16 * m, cudaMemcpyDeviceToHost, c->stream));
      CK(cudaMemcpyAsync(M[b].data(), jobs[b]->M, 4 * m, cudaMemcpyDeviceToHost, c->stream));
      CK(cudaMemcpyAsync(C[b].data(), jobs[b]->cost, 4 * m, cudaMemcpyDeviceToHost, c->stream));
    }
    st = finish_results(c, jobs, out);
    for (size_t b = 0; b < jobs.size(); ++b)
      for (size_t i = 0; i < kv[b].size(); ++i) {
        if (k_star && k_star[b]) {
          k_star[b][3 * i] = kv[b][i].x;
          k_star[b][3 * i + 1] = kv[b][i].y;
          k_star[b][3 * i + 2] = kv[b][i].z;
        }
        if (votes && votes[b]) votes[b][i] = (uint32_t)kv[b][i].w;
        if (inliers && inliers[b]) inliers[b][i] = M[b][i];
        if (cost && cost[b]) cost[b][i] = C[b][i];
      }
  });
  return gs != DSES_OK ? gs : st;
}

dses_status dses_submit(dses_ctx* c, const dses_problem* problem, uint64_t* ticket) {
  if (!c || !problem || !ticket) return DSES_ERR_INVALID_ARG;
  std::lock_guard<std::recursive_mutex> g(c->mu);
  return guard(c, [&] {
    auto r = std::make_shared<Request>();
    r->prob = *problem;
    if (problem->src_is_device) invalid("dses_submit takes a host source cloud");
    if (!problem->src || problem->n_src < 1 || problem->n_src > (1 << 24)) invalid("bad source cloud");
    r->src.assign(problem->src, problem->src + 3 * problem->n_src);
    r->prob.src = r->src.data();
    if (problem->grid.kind == DSES_GRID_EXPLICIT && problem->grid.explicit_R && problem->grid.n_explicit > 0) {
      r->explicit_R.assign(problem->grid.explicit_R, problem->grid.explicit_R + 9 * problem->grid.n_explicit);
      r->prob.grid.explicit_R = r->explicit_R.data();
    }
    resolve(c, &r->prob, r->job);
    plan(c, r->job);
    set_device(c);
    {
      std::lock_guard<std::mutex> lk(c->smu);
      if ((int64_t)c->queue.size() >= c->opt.serve_queue_cap)
        throw Error{DSES_ERR_QUEUE_FULL, "serving queue is full"};
      if (c->res_free.empty()) {
        constexpr int kChunk = 256;
        dses_result* chunk = nullptr;
        CK(cudaMallocHost((void**)&chunk, sizeof(dses_result) * kChunk));
        c->res_chunks.push_back(chunk);
        for (int i = kChunk - 1; i >= 0; --i) c->res_free.push_back(chunk + i);
      }
      r->host_res = c->res_free.back();
      c->res_free.pop_back();
      *ticket = c->next_ticket++;
      c->tickets[*ticket] = r;
      r->job.T->inflight++;
      c->queue.push_back(r);
      if (!c->worker_started) {
        c->stop = false;
        c->worker = std::thread(worker_loop, c);
        c->worker_started = true;
      }
    }
    c->scv.notify_all();
  });
}

dses_status dses_poll(dses_ctx* c, uint64_t ticket, dses_result* out) {
  if (!c || !out) return DSES_ERR_INVALID_ARG;
  std::shared_ptr<Request> r;
  {
    std::lock_guard<std::mutex> lk(c->smu);
    auto it = c->tickets.find(ticket);
    if (it == c->tickets.end()) return DSES_ERR_UNKNOWN_TICKET;
    r = it->second;
    if (r->state.load() != 2) return DSES_NOT_READY;
    c->tickets.erase(it);
    if (r->host_res) c->res_free.push_back(r->host_res);  // its result is already in r->result
    r->host_res = nullptr;
  }
  *out = r->result;
  if (r->status != DSES_OK) {
    std::lock_guard<std::recursive_mutex> g(c->mu);
    c->err = r->err.empty() ? "registration found no candidate" : r->err;
  }
  return r->status;
}

// Rotation count of a HOPF or EULER_BOX grid and, when out_R is set, its FP32
// rotations copied to host memory (the values every pass over the grid uses).
static int64_t build_grid_host(dses_ctx* c, const dses_rotation_grid* grid, float* out_R, int64_t capacity) {
  int64_t n = 0;
  if (grid->kind == DSES_GRID_HOPF) {
    if (grid->hopf_n < 1 || grid->hopf_n > 48) invalid("hopf_n must be in [1, 48]");
    n = 72LL * grid->hopf_n * grid->hopf_n * grid->hopf_n;
  } else if (grid->kind == DSES_GRID_EULER_BOX) {
    if (grid->K < 0 || grid->K > 100 || !(grid->delta_r > 0)) invalid("bad Euler box");
    n = (int64_t)(2 * grid->K + 1) * (2 * grid->K + 1) * (2 * grid->K + 1);
  } else {
    invalid("only HOPF and EULER_BOX grids are built on the device");
  }
  if (!out_R) return n;
  if (n > capacity) invalid("capacity is smaller than the grid");
  if (grid->kind == DSES_GRID_HOPF) {
    const float* p = hopf_grid(c, grid->hopf_n);
    CK(cudaMemcpyAsync(out_R, p, 36 * (size_t)n, cudaMemcpyDeviceToHost, c->stream));
  } else {
    DevMem m;
    m.alloc(align256(36 * (size_t)n) + 256, c->stream);
    double* R0 = (double*)((char*)m.p + align256(36 * (size_t)n));
    CK(cudaMemcpyAsync(R0, grid->R0, 72, cudaMemcpyHostToDevice, c->stream));
    CK(launch_euler_box_single(R0, grid->K, grid->delta_r, (float*)m.p, c->stream));
    CK(cudaMemcpyAsync(out_R, m.p, 36 * (size_t)n, cudaMemcpyDeviceToHost, c->stream));
    m.release();
  }
  CK(cudaStreamSynchronize(c->stream));
  return n;
}

dses_status dses_rotation_grid_build(dses_ctx* c, const dses_rotation_grid* grid, float* out_R, int64_t capacity,
                                     int64_t* count) {
  if (!c || !grid || !count) return DSES_ERR_INVALID_ARG;
  std::lock_guard<std::recursive_mutex> g(c->mu);
  return guard(c, [&] {
    set_device(c);
    *count = build_grid_host(c, grid, nullptr, 0);
    if (out_R) build_grid_host(c, grid, out_R, capacity);
  });
}

dses_status dses_shard_range(int64_t n_rot, int32_t rank, int32_t world, int64_t* begin, int64_t* end) {
  if (!begin || !end || n_rot < 0 || world < 1 || rank < 0 || rank >= world) return DSES_ERR_INVALID_ARG;
  *begin = n_rot * rank / world;
  *end = n_rot * (rank + 1) / world;
  return DSES_OK;
}

dses_status dses_register_shard(dses_ctx* c, const dses_problem* problem, int32_t rank, int32_t world,
                                dses_result* out) {
  if (!c || !problem || !out) return DSES_ERR_INVALID_ARG;
  std::lock_guard<std::recursive_mutex> g(c->mu);
  dses_status st = DSES_OK;
  const dses_status gs = guard(c, [&] {
    set_device(c);
    if (world < 1 || rank < 0 || rank >= world) invalid("shard rank must be in [0, world)");
    const dses_params& P = problem->params;
    if (P.q_milli != 0 || P.top_k != 0 || P.refine_top_k != 0)
      invalid("a shard without an exchange scores every rotation of its range: q_milli, top_k and refine_top_k "
              "must be 0 (dses_register_sharded exchanges what they need)");
    st = run_sharded(c, problem, rank, world, nullptr, out);
  });
  return gs != DSES_OK ? gs : st;
}

dses_status dses_register_sharded(dses_ctx* c, const dses_problem* problem, int32_t rank, int32_t world,
                                  dses_allgather_fn allgather, void* user, dses_result* out) {
  if (!c || !problem || !out || !allgather) return DSES_ERR_INVALID_ARG;
  std::lock_guard<std::recursive_mutex> g(c->mu);
  dses_status st = DSES_OK;
  const dses_status gs = guard(c, [&] {
    set_device(c);
    if (world < 1 || rank < 0 || rank >= world) invalid("shard rank must be in [0, world)");
    Exchange X;
    X.fn = allgather;
    X.user = user;
    X.world = world;
    st = run_sharded(c, problem, rank, world, &X, out);
  });
  return gs != DSES_OK ? gs : st;
}

dses_status dses_combine_results(const dses_result* parts, int32_t n, dses_result* out) {
  if (!parts || !out || n < 1) return DSES_ERR_INVALID_ARG;
  int best = -1;
  bool voted = false;
  for (int i = 0; i < n; ++i) {
    const dses_result& r = parts[i];
    if (r.status != DSES_OK && r.status != DSES_ERR_NO_CANDIDATE) return DSES_ERR_INVALID_ARG;
    voted |= r.status == DSES_OK;
    if (r.rot_index < 0) continue;  // a shard without any candidate
    uint32_t cb, bb = 0;
    std::memcpy(&cb, &r.cost, 4);
    if (best >= 0) std::memcpy(&bb, &parts[best].cost, 4);
    // the kernels' argmin order: cost bits (cost >= 0), then the rotation index
    if (best < 0 || cb < bb || (cb == bb && r.rot_index < parts[best].rot_index)) best = i;
  }
  if (best < 0) {
    std::memset(out, 0, sizeof(*out));
    out->rot_index = -1;
    out->cost = std::numeric_limits<float>::quiet_NaN();
    out->status = DSES_ERR_NO_CANDIDATE;
    return DSES_ERR_NO_CANDIDATE;
  }
  *out = parts[best];
  out->status = voted ? DSES_OK : DSES_ERR_NO_CANDIDATE;
  return (dses_status)out->status;
}

dses_status dses_target_distance_grid(dses_ctx* c, const dses_target* T, float* D, float lo[3], float h[3],
                                      int32_t* res, float* cap) {
  if (!c || !T) return DSES_ERR_INVALID_ARG;
  std::lock_guard<std::recursive_mutex> g(c->mu);
  return guard(c, [&] {
    if (T->ctx != c) invalid("target belongs to another context");
    if (res) *res = T->G;
    if (cap) *cap = T->gcap;
    for (int a = 0; a < 3; ++a) {
      if (lo) lo[a] = T->glo[a];
      if (h) h[a] = T->gh[a];
    }
    if (D) {
      set_device(c);
      CK(cudaMemcpyAsync(D, T->D, sizeof(float) * (size_t)T->G * T->G * T->G, cudaMemcpyDeviceToHost, c->stream));
      CK(cudaStreamSynchronize(c->stream));
    }
  });
}

dses_status dses_refine_translation(dses_ctx* c, const dses_target* Tc, const float* src, int64_t n_src,
                                    int32_t src_is_device, const float R[9], const float t[3], float epsilon,
                                    int32_t iterations, float t_out[3], uint32_t* n_inliers) {
  if (!c || !Tc) return DSES_ERR_INVALID_ARG;
  std::lock_guard<std::recursive_mutex> g(c->mu);
  return guard(c, [&] {
    dses_target* T = const_cast<dses_target*>(Tc);
    if (T->ctx != c) invalid("target belongs to another context");
    if (!src || n_src < 1 || n_src > (1 << 24)) invalid("n_src must be in [1, 2^24]");
    if (!R || !t || !t_out) invalid("R, t and t_out are required");
    if (!finite3(R, 3) || !finite3(t, 1)) invalid("R and t must be finite");
    if (!(epsilon > 0) || !std::isfinite(epsilon)) invalid("epsilon must be positive and finite");
    if (iterations < 1 || iterations > 64) invalid("iterations must be in [1, 64]");
    if (!src_is_device && !finite3(src, n_src)) invalid("source cloud has a non-finite coordinate");
    set_device(c);
    CellList* cl = cell_list(c, T, epsilon);
    DevMem scratch, xs;
    scratch.alloc(64, c->stream);  // t (3 doubles), acc (4 doubles), count
    double* td = (double*)scratch.p;
    double* acc = td + 3;
    uint32_t* nd = (uint32_t*)(td + 7);
    double th[8] = {t[0], t[1], t[2], 0.0, 0.0, 0.0, 0.0, 0.0};
    CK(cudaMemcpyAsync(td, th, sizeof(th), cudaMemcpyHostToDevice, c->stream));
    const float* X = src;
    if (!src_is_device) {
      xs.alloc(12 * (size_t)n_src, c->stream);
      CK(cudaMemcpyAsync(xs.p, src, 12 * (size_t)n_src, cudaMemcpyHostToDevice, c->stream));
      X = (const float*)xs.p;
    }
    RefineDesc d;
    d.X = X;
    d.N = (int)n_src;
    d.Y = cl->sorted;
    d.cell_start = cl->start;
    for (int a = 0; a < 3; ++a) {
      d.cell_lo[a] = cl->lo[a];
      d.cell_dim[a] = cl->dim[a];
    }
    d.cell_inv = cl->inv;
    d.eps2 = epsilon * epsilon;
    for (int k = 0; k < 9; ++k) d.R[k] = R[k];
    d.t = td;
    d.acc = acc;
    for (int it = 0; it < iterations; ++it) CK(launch_refine_step(d, nd, c->stream));
    double tr[3];
    uint32_t n = 0;
    CK(cudaMemcpyAsync(tr, td, sizeof(tr), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(&n, nd, sizeof(n), cudaMemcpyDeviceToHost, c->stream));
    xs.release();
    scratch.release();
    CK(cudaStreamSynchronize(c->stream));
    for (int a = 0; a < 3; ++a) t_out[a] = (float)tr[a];
    if (n_inliers) *n_inliers = n;
  });
}

dses_status dses_exhaustive_search(dses_ctx* c, const dses_problem* problem, float* cost_out, int64_t cost_capacity,
                                   dses_result* out) {
  if (!c || !problem || !out) return DSES_ERR_INVALID_ARG;
  std::lock_guard<std::recursive_mutex> g(c->mu);
  return guard(c, [&] {
    // exact nearest neighbours; the candidate filter and the second pass do not apply
    dses_problem q = *problem;
    q.params.nn_mode = DSES_NN_BRUTE;
    q.params.q_milli = 0;
    q.params.top_k = 0;
    q.params.refine_top_k = 0;
    Job j;
    resolve(c, &q, j);
    if (j.T->m > kExhaustiveMaxTargets) invalid("exhaustive search stages the target in shared memory: m <= 12288");
    const int64_t nt = (int64_t)j.E[0] * j.E[1] * j.E[2];
    const int64_t total = j.n_first * nt;
    if (total > (1LL << 28)) invalid("exhaustive search is limited to 2^28 (rotation, translation) pairs");
    if (cost_out && cost_capacity < total) invalid("cost_capacity is smaller than rotations x translations");
    set_device(c);
    cudaStream_t s = c->stream;
    const dses_rotation_grid& gr = q.grid;
    DevMem rmem, xmem, omem;
    const float* rot = nullptr;
    if (gr.kind == DSES_GRID_HOPF) {
      rot = hopf_grid(c, gr.hopf_n);
    } else if (gr.kind == DSES_GRID_EULER_BOX) {
      rmem.alloc(align256(36 * (size_t)j.n_first) + 256, s);
      double* R0 = (double*)((char*)rmem.p + align256(36 * (size_t)j.n_first));
      CK(cudaMemcpyAsync(R0, gr.R0, 72, cudaMemcpyHostToDevice, s));
      CK(launch_euler_box_single(R0, gr.K, gr.delta_r, (float*)rmem.p, s));
      rot = (const float*)rmem.p;
    } else {
      if (!finite3(gr.explicit_R, 3 * gr.n_explicit)) invalid("explicit rotations have a non-finite entry");
      rmem.alloc(36 * (size_t)j.n_first, s);
      CK(cudaMemcpyAsync(rmem.p, gr.explicit_R, 36 * (size_t)j.n_first, cudaMemcpyHostToDevice, s));
      rot = (const float*)rmem.p;
    }
    const float* X = q.src;
    if (!q.src_is_device) {
      xmem.alloc(12 * (size_t)j.N, s);
      CK(cudaMemcpyAsync(xmem.p, q.src, 12 * (size_t)j.N, cudaMemcpyHostToDevice, s));
      X = (const float*)xmem.p;
    }
    omem.alloc(align256(4 * (size_t)total) * 2 + 256, s);
    float* cost = (float*)omem.p;
    uint32_t* count = (uint32_t*)((char*)omem.p + align256(4 * (size_t)total));
    unsigned long long* best = (unsigned long long*)((char*)count + align256(4 * (size_t)total));
    CK(launch_fill_u64(best, ~0ull, 1, s));
    ExhaustiveDesc d;
    d.X = X;
    d.N = j.N;
    d.Y = j.T->Y;
    d.M = j.T->m;
    d.rot = rot;
    d.n_rot = (int)j.n_first;
    for (int a = 0; a < 3; ++a) {
      d.lo[a] = j.lo[a];
      d.E[a] = j.E[a];
    }
    d.n_t = (int)nt;
    d.delta = j.delta;
    d.metric = j.metric;
    d.eps = j.eps;
    d.tau = j.tau;
    d.huber_h = j.hh;
    d.p_exp = j.pexp;
    d.cost = cost;
    d.count = count;
    d.best = best;
    CK(launch_exhaustive(d, s));
    unsigned long long key = 0;
    CK(cudaMemcpyAsync(&key, best, 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const int64_t idx = (int64_t)(key & 0xffffffffull);
    const int64_t r = idx / nt, ti = idx % nt;
    float Rh[9], ch = 0.f;
    uint32_t nh = 0;
    CK(cudaMemcpyAsync(Rh, rot + 9 * r, 36, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&ch, cost + idx, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&nh, count + idx, 4, cudaMemcpyDeviceToHost, s));
    if (cost_out) CK(cudaMemcpyAsync(cost_out, cost, 4 * (size_t)total, cudaMemcpyDeviceToHost, s));
    rmem.release();
    xmem.release();
    omem.release();
    CK(cudaStreamSynchronize(s));
    dses_result res;
    std::memset(&res, 0, sizeof(res));
    for (int k = 0; k < 9; ++k) res.R[k] = Rh[k];
    const int64_t k3[3] = {ti / ((int64_t)j.E[1] * j.E[2]), (ti / j.E[2]) % j.E[1], ti % j.E[2]};
    for (int a = 0; a < 3; ++a) res.t[a] = (float)(j.lo[a] + k3[a]) * j.delta;
    res.rot_index = r;
    res.inliers = nh;
    res.votes = 0;
    res.cost = ch;
    res.status = DSES_OK;
    *out = res;
  });
}

static int64_t* option_slot(dses_ctx* c, const char* key) {
  if (!key) return nullptr;
  const std::string k(key);
  Options& o = c->opt;
  if (k == "hist_mode") return &o.hist_mode;
  if (k == "hist_budget_bytes") return &o.hist_budget;
  if (k == "points_per_thread") return &o.points_per_thread;
  if (k == "fuse_score") return &o.fuse_score;
  if (k == "tile_rotations") return &o.tile_rotations;
  if (k == "autotune") return &o.autotune;
  if (k == "use_graphs") return &o.use_graphs;
  if (k == "serve_max_batch") return &o.serve_max_batch;
  if (k == "serve_queue_cap") return &o.serve_queue_cap;
  if (k == "serve_mem_budget") return &o.serve_mem_budget;
  if (k == "serve_tile_rotations") return &o.serve_tile_rotations;
  if (k == "serve_iter_pairs") return &o.serve_iter_pairs;
  if (k == "record_timing") return &o.record_timing;
  if (k == "vote_sparse") return &o.vote_sparse;
  if (k == "fail_next_allocs") return &o.fail_next_allocs;
  if (k == "target_order") return &o.target_order;
  if (k == "hist_strides") return &o.hist_strides;
  if (k == "serve_max_active") return &c->serve_max_active;
  if (k == "serve_busy_ns") return &c->serve_busy_ns;
  if (k == "serve_iterations") return &c->serve_iterations;
  if (k == "last_pass_ns") return &c->pass_ns;
  if (k == "last_pass_launches") return &c->pass_launches;
  if (k == "last_count_ns") return &c->count_ns;
  if (k == "last_votes_total") return &c->votes_total;
  if (k == "last_vote_sparse") return &c->vote_sparse_jobs;
  if (k == "last_vote_paired") return &c->vote_paired_jobs;
  if (k == "last_p_mask") return &c->last_p_mask;
  if (k == "last_tile_max") return &c->last_tile_max;
  if (k == "graphs_cached") {
    c->graph_count = (int64_t)c->graphs.size();
    return &c->graph_count;
  }
  if (k == "kernel_launches") {
    c->launch_snapshot = kernel_launch_count();
    return &c->launch_snapshot;
  }
  return nullptr;
}

dses_status dses_set_option(dses_ctx* c, const char* key, int64_t value) {
  if (!c) return DSES_ERR_INVALID_ARG;
  std::lock_guard<std::recursive_mutex> g(c->mu);
  return guard(c, [&] {
    int64_t* slot = option_slot(c, key);
    if (!slot) invalid(std::string("unknown option ") + (key ? key : "(null)"));
    const std::string k(key);
    bool ok = true;
    if (k == "hist_mode") ok = value >= 0 && value <= 3;
    else if (k == "vote_sparse") ok = value >= 0 && value <= 3;
    else if (k == "hist_budget_bytes") ok = value >= 1024 && value <= kHistBudget;
    else if (k == "points_per_thread") ok = value == 0 || value == 1 || value == 2 || value == 4 || value == 8;
    else if (k == "fuse_score" || k == "autotune" || k == "use_graphs" || k == "record_timing")
      ok = value == 0 || value == 1;
    else if (k == "last_pass_ns" || k == "last_pass_launches" || k == "kernel_launches" || k == "last_count_ns" ||
             k == "last_votes_total" || k == "last_vote_sparse" || k == "last_vote_paired" ||
             k == "last_p_mask" || k == "last_tile_max" ||
             k == "graphs_cached")
      ok = false;  // read-only
    else if (k == "tile_rotations") ok = value >= 0 && value <= 4096;
    else if (k == "fail_next_allocs") ok = value >= 0;
    else if (k == "target_order" || k == "hist_strides") ok = value == 0 || value == 1;
    else if (k == "serve_max_active" || k == "serve_busy_ns" || k == "serve_iterations") ok = value == 0;  // reset only
    else ok = value >= 1;
    if (!ok) invalid("option value out of range for " + k);
    *slot = value;
  });
}

dses_status dses_get_option(dses_ctx* c, const char* key, int64_t* value) {
  if (!c || !value) return DSES_ERR_INVALID_ARG;
  std::lock_guard<std::recursive_mutex> g(c->mu);
  return guard(c, [&] {
    int64_t* slot = option_slot(c, key);
    if (!slot) invalid(std::string("unknown option ") + (key ? key : "(null)"));
    *value = *slot;
  });
}

const char* dses_last_error(dses_ctx* c) { return c ? c->err.c_str() : "null context"; }

const char* dses_status_string(dses_status s) {
  switch (s) {
    case DSES_OK: return "DSES_OK";
    case DSES_NOT_READY: return "DSES_NOT_READY";
    case DSES_ERR_INVALID_ARG: return "DSES_ERR_INVALID_ARG";
    case DSES_ERR_OOM: return "DSES_ERR_OOM";
    case DSES_ERR_CUDA: return "DSES_ERR_CUDA";
    case DSES_ERR_QUEUE_FULL: return "DSES_ERR_QUEUE_FULL";
    case DSES_ERR_TIMEOUT: return "DSES_ERR_TIMEOUT";
    case DSES_ERR_NO_CANDIDATE: return "DSES_ERR_NO_CANDIDATE";
    case DSES_ERR_UNKNOWN_TICKET: return "DSES_ERR_UNKNOWN_TICKET";
    case DSES_ERR_EXCHANGE: return "DSES_ERR_EXCHANGE";
  }
  return "unknown status";
}

}  // extern "C"
