// Auxiliary kernels of the DSES library: rotation grids, target
// preprocessing (distance grid, cell list), candidate selection, candidate
// scoring (grid lookup or exact brute-force nearest neighbour), the argmin
// reduction and the result finaliser.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "dses.h"
#include "kernels.cuh"

#include <atomic>

namespace dses {

std::atomic<long long> g_launches{0};
long long kernel_launch_count() { return g_launches.load(); }

namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;

// ---------------------------------------------------------------------------
// rotation grids

__device__ void quat_to_matrix(double w, double x, double y, double z, double* R) {
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

// HEALPix RING pixel p at N_side = n -> (theta, phi), closed form per pixel
// (north cap, equatorial belt, south cap; Gorski et al. 2005).
__device__ void healpix_pix2ang(int n, long long p, double* theta, double* phi) {
  const long long N = n;
  const long long npix = 12 * N * N, ncap = 2 * N * (N - 1);
  double z;
  if (p < ncap) {
    long long i = (long long)(0.5 * (1.0 + sqrt(1.0 + 2.0 * (double)p)));
    while (2 * i * (i + 1) <= p) ++i;
    while (i > 1 && 2 * i * (i - 1) > p) --i;
    const long long j = p + 1 - 2 * i * (i - 1);
    z = 1.0 - (double)(i * i) / (3.0 * (double)(N * N));
    *phi = ((double)j - 0.5) * kPi / (2.0 * (double)i);
  } else if (p < npix - ncap) {
    const long long q = p - ncap;
    const long long i = q / (4 * N) + N;
    const long long j = q % (4 * N) + 1;
    const double shift = ((i + N) & 1) ? 1.0 : 0.5;
    z = (double)(2 * N - i) * 2.0 / (3.0 * (double)N);
    *phi = ((double)j - shift) * kPi / (2.0 * (double)N);
  } else {
    const long long q = npix - p;
    long long i = (long long)(0.5 * (1.0 + sqrt(2.0 * (double)q - 1.0)));
    while (2 * i * (i + 1) < q) ++i;
    while (i > 1 && 2 * (i - 1) * i >= q) --i;
    const long long j = 4 * i + 1 - (q - 2 * i * (i - 1));
    z = -1.0 + (double)(i * i) / (3.0 * (double)(N * N));
    *phi = ((double)j - 0.5) * kPi / (2.0 * (double)i);
  }
  *theta = acos(z);
}

__device__ void hopf_matrix(int n, long long r, double* R) {
  const long long per = 6LL * n;
  double th, ph;
  healpix_pix2ang(n, r / per, &th, &ph);
  const double psi = 2.0 * kPi * ((double)(r % per) + 0.5) / (double)per;
  double st, ct, sp, cp, sa, ca;
  sincos(0.5 * th, &st, &ct);
  sincos(0.5 * psi, &sp, &cp);
  sincos(ph + 0.5 * psi, &sa, &ca);
  quat_to_matrix(ct * cp, ct * sp, st * ca, st * sa, R);
}

__global__ void hopf_grid_kernel(int n, long long total, float* out) {
  const long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (r >= total) return;
  double R[9];
  hopf_matrix(n, r, R);
#pragma unroll
  for (int k = 0; k < 9; ++k) out[9 * r + k] = (float)R[k];
}

__device__ void mul3(const double* A, const double* B, double* C) {
  double T[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) T[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
  for (int k = 0; k < 9; ++k) C[k] = T[k];
}

// R = Rc Rz(a) Ry(b) Rx(c) for local index ((a w) + b) w + c, angles (i - K) delta_r.
__device__ void euler_box_matrix(const double* Rc, int K, double dr, int local, double* out) {
  const int w = 2 * K + 1;
  const int a = local / (w * w), b = (local / w) % w, c = local % w;
  double sa, ca, sb, cb, sc, cc;
  sincos((a - K) * dr, &sa, &ca);
  sincos((b - K) * dr, &sb, &cb);
  sincos((c - K) * dr, &sc, &cc);
  const double Rz[9] = {ca, -sa, 0, sa, ca, 0, 0, 0, 1};
  const double Ry[9] = {cb, 0, sb, 0, 1, 0, -sb, 0, cb};
  const double Rx[9] = {1, 0, 0, 0, cc, -sc, 0, sc, cc};
  double T[9];
  mul3(Rc, Rz, T);
  mul3(T, Ry, T);
  mul3(T, Rx, out);
}

__device__ __forceinline__ uint32_t key_centre(const unsigned long long* keys, int c) {
  // padding keys (all ones) repeat the previous valid centre
  int cc = c;
  while (cc > 0 && keys[cc] == ~0ull) --cc;
  const unsigned long long k = keys[cc];
  return k == ~0ull ? 0u : (uint32_t)(k & 0xffffffffull);
}

// centre source: an FP64 matrix (centre64), FP32 matrices (centres, one per
// box), Hopf indices from keys (hopf_n > 0), or FP32 rotations picked by key
__global__ void euler_boxes_kernel(const float* centres, int hopf_n, const unsigned long long* keys,
                                   const float* keyed_rot, const double* centre64, int count, int K, double dr,
                                   float* out) {
  const int w = 2 * K + 1, B = w * w * w;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)count * B) return;
  const int c = (int)(t / B), local = (int)(t % B);
  double Rc[9];
  if (centre64) {
    for (int k = 0; k < 9; ++k) Rc[k] = centre64[k];
  } else if (centres) {
    for (int k = 0; k < 9; ++k) Rc[k] = (double)centres[9 * c + k];
  } else if (hopf_n > 0) {
    hopf_matrix(hopf_n, (long long)key_centre(keys, c), Rc);
  } else {
    const uint32_t r = key_centre(keys, c);
    for (int k = 0; k < 9; ++k) Rc[k] = (double)keyed_rot[9 * (size_t)r + k];
  }
  double R[9];
  euler_box_matrix(Rc, K, dr, local, R);
  for (int k = 0; k < 9; ++k) out[9 * t + k] = (float)R[k];
}

// ---------------------------------------------------------------------------
// target preprocessing

__global__ void pack_points_kernel(const float* xyz, int m, float4* out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < m) out[j] = make_float4(xyz[3 * j], xyz[3 * j + 1], xyz[3 * j + 2], 0.f);
}

// D[v] = min(cap, min_j ||centre(v) - y_j||): brute force with target tiles in shared memory.
__global__ void __launch_bounds__(256) dist_grid_kernel(const float4* __restrict__ Y, int m, int G, float lox,
                                                        float loy, float loz, float hx, float hy, float hz,
                                                        float cap, float* __restrict__ D) {
  __shared__ float4 tile[1024];
  const long long total = (long long)G * G * G;
  const long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long vv = v < total ? v : total - 1;
  const int a = (int)(vv / ((long long)G * G)), b = (int)((vv / G) % G), c = (int)(vv % G);
  const float px = lox + ((float)a + 0.5f) * hx, py = loy + ((float)b + 0.5f) * hy, pz = loz + ((float)c + 0.5f) * hz;
  float best = INFINITY;
  for (int t0 = 0; t0 < m; t0 += 1024) {
    const int n = min(1024, m - t0);
    __syncthreads();
    for (int k = threadIdx.x; k < n; k += blockDim.x) tile[k] = Y[t0 + k];
    __syncthreads();
    for (int k = 0; k < n; ++k) {
      const float4 q = tile[k];
      const float dx = q.x - px, dy = q.y - py, dz = q.z - pz;
      best = fminf(best, fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
    }
  }
  if (v < total) D[v] = fminf(cap, sqrtf(best));
}

__global__ void pack_corners_kernel(const float* __restrict__ D, int G, float4* __restrict__ D4) {
  const long long total = (long long)G * G * G;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < total;
       v += (long long)gridDim.x * blockDim.x) {
    const int a = (int)(v / ((long long)G * G)), b = (int)((v / G) % G), c = (int)(v % G);
    const int b1 = min(b + 1, G - 1), c1 = min(c + 1, G - 1);
    const float* row0 = D + ((size_t)a * G + b) * G;
    const float* row1 = D + ((size_t)a * G + b1) * G;
    D4[v] = make_float4(row0[c], row0[c1], row1[c], row1[c1]);
  }
}

__device__ __forceinline__ int cell_of(float p, float lo, float inv, int dim) {
  const float f = floorf((p - lo) * inv);
  return (int)fminf(fmaxf(f, 0.f), (float)(dim - 1));
}

__global__ void cell_count_kernel(const float4* Y, int m, float lx, float ly, float lz, float inv, int dx, int dy,
                                  int dz, int* counts, int* cell_of_pt) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  const float4 p = Y[j];
  const int c = (cell_of(p.z, lz, inv, dz) * dy + cell_of(p.y, ly, inv, dy)) * dx + cell_of(p.x, lx, inv, dx);
  cell_of_pt[j] = c;
  atomicAdd(counts + c, 1);
}

// exclusive prefix of counts[0..n) into start[0..n], one block of 1024 threads
__global__ void __launch_bounds__(1024) exclusive_scan_kernel(const int* counts, int n, int* start) {
  __shared__ int part[1024];
  const int t = threadIdx.x;
  const int per = (n + 1023) / 1024;
  const int b = min(n, t * per), e = min(n, b + per);
  int s = 0;
  for (int i = b; i < e; ++i) s += counts[i];
  part[t] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {  // Hillis-Steele inclusive scan
    const int v = t >= o ? part[t - o] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int run = t > 0 ? part[t - 1] : 0;
  for (int i = b; i < e; ++i) {
    start[i] = run;
    run += counts[i];
  }
  if (t == 1023) start[n] = part[1023];
}

__global__ void cell_scatter_kernel(const float4* Y, int m, const int* cell_of_pt, int* cursor, float4* sorted) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  const int pos = atomicAdd(cursor + cell_of_pt[j], 1);
  sorted[pos] = Y[j];
}

__global__ void copy_int_kernel(const int* a, int n, int* b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = a[i];
}

// ---------------------------------------------------------------------------
// candidate selection

__global__ void select_q_kernel(const uint32_t* Mout, uint32_t first, int n, const uint32_t* acc, int q_milli,
                                uint32_t* cand, uint32_t* n_cand) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const unsigned long long Mstar = acc[0];
  if (1000ull * Mout[first + r] >= (unsigned long long)q_milli * Mstar) cand[atomicAdd(n_cand, 1u)] = first + r;
}

__global__ void keys_from_M_kernel(const uint32_t* Mout, uint32_t first, int n, uint32_t out_base,
                                   unsigned long long* keys) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n)
    keys[r] = ((unsigned long long)(0xffffffffu - Mout[first + r]) << 32) |
              (unsigned long long)(out_base + first + r);
}

__global__ void keys_from_cost_kernel(const float* cost, const uint32_t* cand, const uint32_t* n_cand, int n_max,
                                      uint32_t out_base, unsigned long long* keys) {
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t n = n_cand ? *n_cand : (uint32_t)n_max;
  if (c >= n) return;
  const uint32_t o = cand ? cand[c] : c;
  keys[c] = ((unsigned long long)__float_as_uint(cost[o]) << 32) | (unsigned long long)(out_base + o);
}

constexpr int kSortN = 4096;

// Each block sorts kSortN keys (bitonic, shared memory) and keeps its k smallest.
__global__ void __launch_bounds__(1024) block_k_smallest_kernel(const unsigned long long* keys, int n_max,
                                                                const uint32_t* n_dev, int k,
                                                                unsigned long long* out) {
  __shared__ unsigned long long s[kSortN];
  const int n = n_dev ? (int)min((uint32_t)n_max, *n_dev) : n_max;
  const long long base = (long long)blockIdx.x * kSortN;
  for (int i = threadIdx.x; i < kSortN; i += blockDim.x) {
    const long long g = base + i;
    s[i] = g < n ? keys[g] : ~0ull;
  }
  __syncthreads();
  for (int size = 2; size <= kSortN; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < kSortN / 2; i += blockDim.x) {
        const int lo = 2 * i - (i & (stride - 1));
        const int hi = lo + stride;
        const bool up = ((lo & size) == 0);
        const unsigned long long a = s[lo], b = s[hi];
        if ((a > b) == up) { s[lo] = b; s[hi] = a; }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < k; i += blockDim.x) out[(long long)blockIdx.x * k + i] = s[i];
}

__global__ void cand_from_keys_kernel(const unsigned long long* keys, int k, uint32_t out_base, uint32_t* cand,
                                      uint32_t* n_cand) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= k) return;
  const unsigned long long key = keys[c];
  if (key == ~0ull) return;
  cand[atomicAdd(n_cand, 1u)] = (uint32_t)(key & 0xffffffffull) - out_base;
}

// ---------------------------------------------------------------------------
// candidate scoring

__device__ __forceinline__ float grid_lookup_s(const ScoreDesc& d, float qx, float qy, float qz) {
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
  const float4* b = d.D4 + ((size_t)ix * d.G + iy) * d.G + iz;
  const float4 p = __ldg(b), q = __ldg(b + (size_t)d.G * d.G);  // x = ix and ix + 1
  const float c00 = p.x + fz * (p.y - p.x);
  const float c01 = p.z + fz * (p.w - p.z);
  const float c10 = q.x + fz * (q.y - q.x);
  const float c11 = q.z + fz * (q.w - q.z);
  const float c0 = c00 + fy * (c01 - c00);
  const float c1 = c10 + fy * (c11 - c10);
  return c0 + fx * (c1 - c0);
}

// one warp per candidate: cost_r = sum_i rho(D~(R x_i + t*))
__global__ void score_grid_kernel(ScoreDesc d, const uint32_t* cand, const uint32_t* n_cand) {
  const uint32_t n = *n_cand;
  const int lane = threadIdx.x & 31;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < n; c += warps) {
    const uint32_t o = cand[c];
    const uint32_t r = o + d.out_base - d.rot_base;
    const float* R = d.rot + 9 * (size_t)r;
    const int4 kv = d.kv[o];
    const float tx = (float)kv.x * d.delta, ty = (float)kv.y * d.delta, tz = (float)kv.z * d.delta;
    float s = 0.f;
    for (int i = lane; i < d.N; i += 32) {
      const float x = d.X[3 * i], y = d.X[3 * i + 1], z = d.X[3 * i + 2];
      const float qx = fmaf(R[0], x, fmaf(R[1], y, R[2] * z)) + tx;
      const float qy = fmaf(R[3], x, fmaf(R[4], y, R[5] * z)) + ty;
      const float qz = fmaf(R[6], x, fmaf(R[7], y, R[8] * z)) + tz;
      s += robust_rho(d.metric, grid_lookup_s(d, qx, qy, qz), d.eps, d.tau, d.huber_h, d.p_exp);
    }
#pragma unroll
    for (int k = 16; k > 0; k >>= 1) s += __shfl_xor_sync(0xffffffffu, s, k);
    if (lane == 0) d.cost[o] = s;
  }
}

// one block per candidate: exact nearest neighbour by brute force, targets
// staged through shared memory, up to 4 source points per thread.
constexpr int kBruteThreads = 256;
constexpr int kBruteTile = 2048;

__global__ void __launch_bounds__(kBruteThreads) score_brute_kernel(ScoreDesc d, const uint32_t* cand,
                                                                    const uint32_t* n_cand) {
  __shared__ float4 tile[kBruteTile];
  __shared__ float red[kBruteThreads / 32];
  const uint32_t n = *n_cand;
  for (uint32_t c = blockIdx.x; c < n; c += gridDim.x) {
    const uint32_t o = cand[c];
    const uint32_t r = o + d.out_base - d.rot_base;
    const float* R = d.rot + 9 * (size_t)r;
    const int4 kv = d.kv[o];
    const float tx = (float)kv.x * d.delta, ty = (float)kv.y * d.delta, tz = (float)kv.z * d.delta;
    float s = 0.f;
    for (int g0 = 0; g0 < d.N; g0 += 4 * kBruteThreads) {
      float qx[4], qy[4], qz[4], best[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = g0 + u * kBruteThreads + threadIdx.x;
        best[u] = INFINITY;
        if (i < d.N) {
          const float x = d.X[3 * i], y = d.X[3 * i + 1], z = d.X[3 * i + 2];
          qx[u] = fmaf(R[0], x, fmaf(R[1], y, R[2] * z)) + tx;
          qy[u] = fmaf(R[3], x, fmaf(R[4], y, R[5] * z)) + ty;
          qz[u] = fmaf(R[6], x, fmaf(R[7], y, R[8] * z)) + tz;
        } else {
          qx[u] = qy[u] = qz[u] = 0.f;
        }
      }
      for (int t0 = 0; t0 < d.M; t0 += kBruteTile) {
        const int nt = min(kBruteTile, d.M - t0);
        __syncthreads();
        for (int k = threadIdx.x; k < nt; k += kBruteThreads) tile[k] = d.Y[t0 + k];
        __syncthreads();
        for (int k = 0; k < nt; ++k) {
          const float4 q = tile[k];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float dx = q.x - qx[u], dy = q.y - qy[u], dz = q.z - qz[u];
            best[u] = fminf(best[u], fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = g0 + u * kBruteThreads + threadIdx.x;
        if (i < d.N) s += robust_rho(d.metric, sqrtf(best[u]), d.eps, d.tau, d.huber_h, d.p_exp);
      }
    }
#pragma unroll
    for (int k = 16; k > 0; k >>= 1) s += __shfl_xor_sync(0xffffffffu, s, k);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      float t = 0.f;
      for (int w = 0; w < kBruteThreads / 32; ++w) t += red[w];
      d.cost[o] = t;
    }
    __syncthreads();
  }
}

// cost of INLIER-metric candidates: N - M (written so the per-rotation dump carries it)
__global__ void inlier_cost_kernel(const uint32_t* Mout, int N, const uint32_t* cand, const uint32_t* n_cand,
                                   float* cost) {
  const uint32_t n = *n_cand;
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x)
    cost[cand[c]] = (float)(N - (int)Mout[cand[c]]);
}

__global__ void argmin_kernel(const float* cost, const uint32_t* cand, const uint32_t* n_cand, uint32_t out_base,
                              unsigned long long* best) {
  const uint32_t n = *n_cand;
  unsigned long long k = ~0ull;
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
    const uint32_t o = cand[c];
    const unsigned long long key =
        ((unsigned long long)__float_as_uint(cost[o]) << 32) | (unsigned long long)(out_base + o);
    k = key < k ? key : k;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, k, o);
    k = w < k ? w : k;
  }
  __shared__ unsigned long long red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = k;
  __syncthreads();
  if (threadIdx.x < 32) {
    k = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : ~0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long w = __shfl_xor_sync(0xffffffffu, k, o);
      k = w < k ? w : k;
    }
    if (threadIdx.x == 0 && k != ~0ull) atomicMin(best, k);
  }
}

__global__ void finalize_kernel(const FinalDesc* fd, int count) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count) return;
  const FinalDesc d = fd[p];
  dses_result* res = reinterpret_cast<dses_result*>(d.result);
  const unsigned long long key = *d.best;
  if (key == ~0ull) {
    for (int k = 0; k < 9; ++k) res->R[k] = 0.f;
    res->t[0] = res->t[1] = res->t[2] = 0.f;
    res->rot_index = -1;
    res->inliers = 0;
    res->votes = 0;
    res->cost = __int_as_float(0x7fc00000);
    res->status = DSES_ERR_NO_CANDIDATE;
    return;
  }
  const uint32_t g = (uint32_t)(key & 0xffffffffull);
  const uint32_t o = g - d.out_base;
  const int4 kv = d.kv[o];
  const float* R = g < d.n_first ? d.rot + 9 * (size_t)g : d.rot_fine + 9 * (size_t)(g - d.n_first);
  for (int k = 0; k < 9; ++k) res->R[k] = R[k];
  res->t[0] = (float)kv.x * d.delta;
  res->t[1] = (float)kv.y * d.delta;
  res->t[2] = (float)kv.z * d.delta;
  res->rot_index = g;
  res->inliers = d.Mout[o];
  res->votes = (uint32_t)kv.w;
  res->cost = __uint_as_float((uint32_t)(key >> 32));
  res->status = (d.acc[1] | d.acc[3]) == 0 ? DSES_ERR_NO_CANDIDATE : DSES_OK;
}

__global__ void fill_u32_kernel(uint32_t* p, uint32_t v, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) p[i] = v;
}
__global__ void fill_f32_kernel(float* p, float v, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) p[i] = v;
}
__global__ void fill_u64_kernel(unsigned long long* p, unsigned long long v, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) p[i] = v;
}

inline int blocks_for(long long n, int t) { return (int)std::max<long long>(1, (n + t - 1) / t); }

}  // namespace

cudaError_t launch_hopf_grid(int n, float* out, cudaStream_t s) {
  const long long total = 72LL * n * n * n;
  g_launches.fetch_add(1, std::memory_order_relaxed);
  hopf_grid_kernel<<<blocks_for(total, 256), 256, 0, s>>>(n, total, out);
  return cudaGetLastError();
}

static long long box_total(int count, int K) { return (long long)count * (2 * K + 1) * (2 * K + 1) * (2 * K + 1); }

cudaError_t launch_euler_boxes(const float* centres, int count, int K, double dr, float* out, cudaStream_t s) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  euler_boxes_kernel<<<blocks_for(box_total(count, K), 128), 128, 0, s>>>(centres, 0, nullptr, nullptr, nullptr,
                                                                          count, K, dr, out);
  return cudaGetLastError();
}

cudaError_t launch_euler_boxes_hopf(int n, const unsigned long long* keys, int count, int K, double dr, float* out,
                                    cudaStream_t s) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  euler_boxes_kernel<<<blocks_for(box_total(count, K), 128), 128, 0, s>>>(nullptr, n, keys, nullptr, nullptr, count,
                                                                          K, dr, out);
  return cudaGetLastError();
}

cudaError_t launch_euler_boxes_keyed(const float* rot, const unsigned long long* keys, int count, int K, double dr,
                                     float* out, cudaStream_t s) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  euler_boxes_kernel<<<blocks_for(box_total(count, K), 128), 128, 0, s>>>(nullptr, 0, keys, rot, nullptr, count, K,
                                                                          dr, out);
  return cudaGetLastError();
}

cudaError_t launch_euler_box_single(const double* R0_dev, int K, double dr, float* out, cudaStream_t s) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  euler_boxes_kernel<<<blocks_for(box_total(1, K), 128), 128, 0, s>>>(nullptr, 0, nullptr, nullptr, R0_dev, 1, K,
                                                                      dr, out);
  return cudaGetLastError();
}

cudaError_t launch_pack_points(const float* xyz, int m, float4* out, cudaStream_t s) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  pack_points_kernel<<<blocks_for(m, 256), 256, 0, s>>>(xyz, m, out);
  return cudaGetLastError();
}

cudaError_t launch_dist_grid(const float4* Y, int m, int G, const float* lo, const float* h, float cap, float* D,
                             float4* D4, cudaStream_t s) {
  const long long total = (long long)G * G * G;
  g_launches.fetch_add(2, std::memory_order_relaxed);
  dist_grid_kernel<<<blocks_for(total, 256), 256, 0, s>>>(Y, m, G, lo[0], lo[1], lo[2], h[0], h[1], h[2], cap, D);
  pack_corners_kernel<<<(int)std::min<long long>(blocks_for(total, 256), 148 * 16), 256, 0, s>>>(D, G, D4);
  return cudaGetLastError();
}

cudaError_t launch_cell_list(const float4* Y, int m, const float* cell_lo, float cell_inv, const int* dim,
                             int* counts, int* cell_start, int* scratch, float4* sorted, cudaStream_t s) {
  const int ncells = dim[0] * dim[1] * dim[2];
  cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(int) * (size_t)ncells, s);
  if (e != cudaSuccess) return e;
  int* cursor = scratch;
  int* cell_of_pt = scratch + ncells;
  g_launches.fetch_add(1, std::memory_order_relaxed);
  cell_count_kernel<<<blocks_for(m, 256), 256, 0, s>>>(Y, m, cell_lo[0], cell_lo[1], cell_lo[2], cell_inv, dim[0],
                                                        dim[1], dim[2], counts, cell_of_pt);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  exclusive_scan_kernel<<<1, 1024, 0, s>>>(counts, ncells, cell_start);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  copy_int_kernel<<<blocks_for(ncells, 256), 256, 0, s>>>(cell_start, ncells, cursor);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  cell_scatter_kernel<<<blocks_for(m, 256), 256, 0, s>>>(Y, m, cell_of_pt, cursor, sorted);
  return cudaGetLastError();
}

cudaError_t launch_select_q(const uint32_t* Mout, uint32_t first, int n, const uint32_t* acc, int q_milli,
                            uint32_t* cand, uint32_t* n_cand, cudaStream_t s) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  select_q_kernel<<<blocks_for(n, 256), 256, 0, s>>>(Mout, first, n, acc, q_milli, cand, n_cand);
  return cudaGetLastError();
}

cudaError_t launch_keys_from_M(const uint32_t* Mout, uint32_t first, int n, uint32_t out_base,
                               unsigned long long* keys, cudaStream_t s) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  keys_from_M_kernel<<<blocks_for(n, 256), 256, 0, s>>>(Mout, first, n, out_base, keys);
  return cudaGetLastError();
}

cudaError_t launch_keys_from_cost(const float* cost, const uint32_t* cand, const uint32_t* n_cand, int n_max,
                                  uint32_t out_base, unsigned long long* keys, cudaStream_t s) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  keys_from_cost_kernel<<<blocks_for(n_max, 256), 256, 0, s>>>(cost, cand, n_cand, n_max, out_base, keys);
  return cudaGetLastError();
}

size_t k_smallest_scratch(int n_max, int k) { return 2 * (size_t)((n_max + kSortN - 1) / kSortN) * (size_t)k + 1; }

cudaError_t launch_k_smallest(const unsigned long long* keys, int n_max, const uint32_t* n_dev, int k,
                              unsigned long long* scratch, unsigned long long* out, cudaStream_t s) {
  if (k < 1 || k > 1024) return cudaErrorInvalidValue;
  const unsigned long long* src = keys;
  int n_cur = n_max;
  const uint32_t* nd = n_dev;
  unsigned long long* bufs[2] = {scratch, scratch + (size_t)((n_max + kSortN - 1) / kSortN) * k};
  int which = 0;
  while (n_cur > kSortN) {
    const int blocks = (n_cur + kSortN - 1) / kSortN;
    g_launches.fetch_add(1, std::memory_order_relaxed);
    block_k_smallest_kernel<<<blocks, 1024, 0, s>>>(src, n_cur, nd, k, bufs[which]);
    src = bufs[which];
    n_cur = blocks * k;
    nd = nullptr;
    which ^= 1;
  }
  g_launches.fetch_add(1, std::memory_order_relaxed);
  block_k_smallest_kernel<<<1, 1024, 0, s>>>(src, n_cur, nd, k, out);
  return cudaGetLastError();
}

cudaError_t launch_cand_from_keys(const unsigned long long* keys, int k, uint32_t out_base, uint32_t* cand,
                                  uint32_t* n_cand, cudaStream_t s) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  cand_from_keys_kernel<<<blocks_for(k, 256), 256, 0, s>>>(keys, k, out_base, cand, n_cand);
  return cudaGetLastError();
}

cudaError_t launch_score_grid(const ScoreDesc& d, const uint32_t* cand, const uint32_t* n_cand, int n_max,
                              cudaStream_t s) {
  const int blocks = std::min(blocks_for((long long)n_max * 32, 256), 148 * 16);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  score_grid_kernel<<<blocks, 256, 0, s>>>(d, cand, n_cand);
  return cudaGetLastError();
}

cudaError_t launch_score_brute(const ScoreDesc& d, const uint32_t* cand, const uint32_t* n_cand, int n_max,
                               cudaStream_t s) {
  const int blocks = std::min(std::max(n_max, 1), 148 * 8);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  score_brute_kernel<<<blocks, kBruteThreads, 0, s>>>(d, cand, n_cand);
  return cudaGetLastError();
}

cudaError_t launch_argmin(float* cost, const uint32_t* Mout, int N, int metric, const uint32_t* cand,
                          const uint32_t* n_cand, int n_max, uint32_t out_base, unsigned long long* best,
                          cudaStream_t s) {
  const int blocks = std::min(blocks_for(n_max, 256), 148 * 4);
  if (metric == 0) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    inlier_cost_kernel<<<blocks, 256, 0, s>>>(Mout, N, cand, n_cand, cost);
  }
  g_launches.fetch_add(1, std::memory_order_relaxed);
  argmin_kernel<<<blocks, 256, 0, s>>>(cost, cand, n_cand, out_base, best);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const FinalDesc* d_dev, int count, cudaStream_t s) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  finalize_kernel<<<blocks_for(count, 64), 64, 0, s>>>(d_dev, count);
  return cudaGetLastError();
}

cudaError_t launch_fill_u32(uint32_t* p, uint32_t v, size_t n, cudaStream_t s) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  fill_u32_kernel<<<std::min(blocks_for((long long)n, 256), 4096), 256, 0, s>>>(p, v, n);
  return cudaGetLastError();
}

cudaError_t launch_fill_f32(float* p, float v, size_t n, cudaStream_t s) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  fill_f32_kernel<<<std::min(blocks_for((long long)n, 256), 4096), 256, 0, s>>>(p, v, n);
  return cudaGetLastError();
}

cudaError_t launch_fill_u64(unsigned long long* p, unsigned long long v, size_t n, cudaStream_t s) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  fill_u64_kernel<<<std::min(blocks_for((long long)n, 256), 4096), 256, 0, s>>>(p, v, n);
  return cudaGetLastError();
}

}  // namespace dses
