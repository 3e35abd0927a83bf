// Rotation pass: the hot loop of Direct Semi-Exhaustive Search (Algorithm 2).
//
// vote_kernel -- one persistent CTA per SM (32 warps). For every rotation R of
// a work item it
//   1. rotates the source cloud and stages per-point lattice offsets in shared
//      memory;
//   2. votes every pair (i, j): the lattice index k = ROUND((y_j - R x_i)/delta)
//      relative to the box corner; pairs inside the lattice box increment a
//      shared-memory histogram (Lemma 1, Eq. 5: the translation mode of the
//      rotated pairwise differences, discretised as in Section IV-B) -- 16-bit
//      packed or 32-bit counters, or a 32-bit copy per lane for small boxes,
//      in x-slabs when the box does not fit, the layout padded to odd extents;
//      pairs outside the box add to a per-lane sink word instead, so the
//      atomic needs no branch; boxes small against the target cull (source,
//      32-point target group) pairs first;
//   3. scans and clears the histogram for the mode (skipping padding bins):
//      V = max count, k* = the lexicographically smallest bin holding V;
//      publishes (k*, V).
// Work items are (problem, rotation tile) pairs taken from a global counter, so
// one persistent launch serves one problem or a batch of uneven problems.
//
// count_kernel -- one warp per rotation: the inlier count M of Eq. 3 at
// t* = k* delta through the target cell list (exact Euclidean test against
// epsilon) and, when every rotation is a candidate, the robust cost from the
// target's truncated distance grid; folds M* and the argmin key into
// per-problem accumulators.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>

#include "kernels.cuh"
#include "optin.h"

namespace dses {

extern std::atomic<long long> g_launches;

namespace {

// Adding 1.5 * 2^23 to |v| < 2^22 leaves an integer rounding of v in the low
// mantissa bits; the float bit pattern of (1.5 * 2^23 + n) is kMagicBits + n.
constexpr float kMagic = 12582912.0f;
constexpr unsigned kMagicBits = 0x4B400000u;

__device__ __forceinline__ unsigned floor_bits(float v) {
  return (unsigned)(__float_as_int(__fadd_rd(v, kMagic)) - (int)kMagicBits);
}

// Trilinear value of the distance grid at q (interpolation between voxel
// centres, clamped at the outermost centres; the cap outside the grid box),
// together with two decisions from bounds on the exact nearest-target distance
// d(q): the stored values are min(d, cap) at voxel centres and d is
// 1-Lipschitz, so every corner c_k used gives D_k - |q - c_k| <= d(q), and, if
// D_k < cap, d(q) <= D_k + |q - c_k|. *far: some corner proves d(q) >= e_far;
// *near: some corner proves d(q) < e_near. Both tests compare squares
// (D_k - e_far >= |q - c_k| iff D_k >= e_far and (D_k - e_far)^2 >= |q - c_k|^2),
// so no square root is taken.
__device__ __forceinline__ float grid_lookup_decide(const PassDesc& d, float qx, float qy, float qz, float e_far,
                                                    float e_near, bool* far, bool* near) {
  const float G = (float)d.G;
  const float ux = (qx - d.glo[0]) * d.ginv_h[0];
  const float uy = (qy - d.glo[1]) * d.ginv_h[1];
  const float uz = (qz - d.glo[2]) * d.ginv_h[2];
  if (!(ux >= 0.f && ux <= G && uy >= 0.f && uy <= G && uz >= 0.f && uz <= G)) {
    // outside the grid box every target lies at least cap + h away
    *far = d.gcap >= e_far;
    *near = false;
    return d.gcap;
  }
  const float gx = fminf(fmaxf(ux - 0.5f, 0.f), G - 1.f);
  const float gy = fminf(fmaxf(uy - 0.5f, 0.f), G - 1.f);
  const float gz = fminf(fmaxf(uz - 0.5f, 0.f), G - 1.f);
  const int ix = min((int)gx, d.G - 2), iy = min((int)gy, d.G - 2), iz = min((int)gz, d.G - 2);
  const float fx = gx - (float)ix, fy = gy - (float)iy, fz = gz - (float)iz;
  // the 8 corners as two 16-byte loads of the corner-block grid
  const float4* b = d.D4 + ((size_t)ix * d.G + iy) * d.G + iz;
  const float4 p = __ldg(b), q = __ldg(b + (size_t)d.G * d.G);
  const float v[8] = {p.x, p.y, p.z, p.w, q.x, q.y, q.z, q.w};
  // q - corner per axis, in world units (corner i at lo + (i + 1/2) h)
  const float h0 = 1.f / d.ginv_h[0], h1 = 1.f / d.ginv_h[1], h2 = 1.f / d.ginv_h[2];
  const float dx0 = (ux - 0.5f - (float)ix) * h0, dy0 = (uy - 0.5f - (float)iy) * h1, dz0 = (uz - 0.5f - (float)iz) * h2;
  bool f = false, n = false;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float ex = (k & 4) ? dx0 - h0 : dx0, ey = (k & 2) ? dy0 - h1 : dy0, ez = (k & 1) ? dz0 - h2 : dz0;
    const float r2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
    const float a = v[k] - e_far, c = e_near - v[k];
    f |= a >= 0.f && a * a >= r2;
    n |= v[k] < d.gcap && c > 0.f && c * c > r2;
  }
  *far = f;
  *near = n;
  const float c00 = v[0] + fz * (v[1] - v[0]);
  const float c01 = v[2] + fz * (v[3] - v[2]);
  const float c10 = v[4] + fz * (v[5] - v[4]);
  const float c11 = v[6] + fz * (v[7] - v[6]);
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

__device__ __forceinline__ unsigned warp_sum_u32(unsigned v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

// Two 16-bit counters per word: their lane-wise maximum, and acc plus both.
__device__ __forceinline__ uint32_t max_u16x2(uint32_t a, uint32_t b) {
  uint32_t d;
  asm("max.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}
__device__ __forceinline__ uint32_t add_halves(uint32_t v, uint32_t acc) {
  uint32_t d;  // acc + lo16(v) * 1 + hi16(v) * 1
  asm("dp2a.lo.u32.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(v), "r"(0x0101u), "r"(acc));
  return d;
}
// Maximum over the block (one value per warp in red[32]; every thread gets it).
__device__ __forceinline__ unsigned block_max_u32(unsigned v, unsigned* red, int lane, int warp) {
  v = __reduce_max_sync(0xffffffffu, v);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  return __reduce_max_sync(0xffffffffu, red[lane]);
}

// Shared-memory histogram increment of a pair whose box-relative lattice
// coordinates are w (inside the centred box iff |w_a| < h_a on all three axes),
// made unconditional: a pair outside the box adds to `sink` (a word outside
// the histogram) instead, so no branch wraps the atomic.
template <bool CUBE = false>
__device__ __forceinline__ void red_or_sink(uint32_t addr, uint32_t inc, uint32_t sink, float wx, float wy,
                                            float wz, float hx, float hy, float hz) {
  if (CUBE)  // one half-width: max(|w_x|, |w_y|, |w_z|) < h
    asm volatile(
        "{\n\t.reg .pred p;\n\t.reg .f32 ax, ay, az;\n\t.reg .b32 a;\n\t"
        "abs.f32 ax, %3;\n\tabs.f32 ay, %4;\n\tabs.f32 az, %5;\n\t"
        "max.f32 ax, ax, ay, az;\n\t"
        "setp.lt.f32 p, ax, %6;\n\t"
        "selp.b32 a, %0, %2, p;\n\t"
        "red.shared.add.u32 [a], %1;\n\t}" ::"r"(addr),
        "r"(inc), "r"(sink), "f"(wx), "f"(wy), "f"(wz), "f"(hx));
  else
    asm volatile(
        "{\n\t.reg .pred p;\n\t.reg .f32 ax, ay, az;\n\t.reg .b32 a;\n\t"
        "abs.f32 ax, %3;\n\tabs.f32 ay, %4;\n\tabs.f32 az, %5;\n\t"
        "setp.lt.f32 p, ax, %6;\n\t"
        "setp.lt.and.f32 p, ay, %7, p;\n\t"
        "setp.lt.and.f32 p, az, %8, p;\n\t"
        "selp.b32 a, %0, %2, p;\n\t"
        "red.shared.add.u32 [a], %1;\n\t}" ::"r"(addr),
        "r"(inc), "r"(sink), "f"(wx), "f"(wy), "f"(wz), "f"(hx), "f"(hy), "f"(hz));
}

// Next vote item of this CTA (dynamic balance across warps).
__device__ __forceinline__ int next_item(int* counter, int lane) {
  int it = 0;
  if (lane == 0) it = atomicAdd(counter, 1);
  return __shfl_sync(0xffffffffu, it, 0);
}

__device__ __forceinline__ void load_targets(const float4* __restrict__ Y, int M, int base, int lane, int P,
                                             float (*ty)[3]) {
  for (int p = 0; p < P; ++p) {
    const int j = base + p * 32 + lane;
    if (j < M) {
      const float4 q = __ldg(Y + j);
      ty[p][0] = q.x; ty[p][1] = q.y; ty[p][2] = q.z;
    } else {  // padding lane: lands far outside every box
      ty[p][0] = 1e30f; ty[p][1] = 1e30f; ty[p][2] = 1e30f;
    }
  }
}

// Centred fast path (odd slab extents on all axes). The staged offset makes
// w_a = y_a/delta + c_a the box-relative lattice coordinate minus S_a/2, so
// the box test is |w_a| < S_a/2 and, with h'_a = (S_a - 1)/2 an integer,
// w_a + (1.5 * 2^23 + h'_a) rounded to nearest holds k_a in its low bits (a
// tie means y_j - R x_i lies on a voxel face). The bin's shared address is
// then three multiply-adds of those bit patterns.
template <int P, bool U16>
__device__ __forceinline__ void vote_centred(const PassDesc& d, const float4* __restrict__ srcc, int nsrc,
                                             unsigned SX, uint32_t hist_base, int* item_ctr, int lane,
                                             uint32_t sink) {
  const int n_tchunks = d.n_tchunks, n_sgroups = d.n_sgroups;
  const int n_items = n_tchunks * n_sgroups;
  const int spg = (nsrc + n_sgroups - 1) / n_sgroups;
  const unsigned Ey = (unsigned)d.E[1], Ez = (unsigned)d.E[2];
  const uint32_t Sx = d.hs[0], Sy = d.hs[1];  // bins per x-plane and per y-row of the layout
  const float inv = d.inv_delta;
  const float hx = 0.5f * (float)SX, hy = 0.5f * (float)Ey, hz = 0.5f * (float)Ez;
  const float mx = kMagic + (float)((SX - 1) / 2), my = kMagic + (float)((Ey - 1) / 2),
              mz = kMagic + (float)((Ez - 1) / 2);
  // address = base + unit * (kx Sx + ky Sy + kz), the kMagicBits offsets folded in
  const uint32_t bias = kMagicBits * (Sx + Sy + 1u);
  // 32-bit counters: word stride `unit` bytes (4, or 128 with a copy per lane)
  const uint32_t unit = d.hist_lanes ? 128u : 4u;
  const uint32_t SxU = Sx * unit, SyU = Sy * unit;
  const uint32_t abase32 = hist_base + (d.hist_lanes ? 4u * (uint32_t)lane : 0u) - unit * bias;
  const uint32_t abase16 = hist_base - 2u * bias;
  const uint32_t sinkl = sink + 4u * (uint32_t)lane;
  for (int it = next_item(item_ctr, lane); it < n_items; it = next_item(item_ctr, lane)) {
    const int tc = it % n_tchunks, sg = it / n_tchunks;
    float ty[P][3];
    load_targets(d.Yv, d.M, tc * P * 32, lane, P, ty);
    const int i0 = sg * spg, i1 = min(i0 + spg, nsrc);
#pragma unroll 4
    for (int i = i0; i < i1; ++i) {
      const float4 c = srcc[i];
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const float wx = __fmaf_rn(ty[p][0], inv, c.x);
        const float wy = __fmaf_rn(ty[p][1], inv, c.y);
        const float wz = __fmaf_rn(ty[p][2], inv, c.z);
        const uint32_t bx = __float_as_uint(__fadd_rn(wx, mx));
        const uint32_t by = __float_as_uint(__fadd_rn(wy, my));
        const uint32_t bz = __float_as_uint(__fadd_rn(wz, mz));
        if (U16) {
          const uint32_t b = bx * Sx + (by * Sy + bz);  // bin + bias (bias even)
          const uint32_t addr = abase16 + ((b >> 1) << 2);
          const uint32_t inc = 1u + (b & 1u) * 0xffffu;
          red_or_sink(addr, inc, sinkl, wx, wy, wz, hx, hy, hz);
        } else {
          const uint32_t addr = abase32 + bx * SxU + (by * SyU + bz * unit);
          red_or_sink(addr, 1u, sinkl, wx, wy, wz, hx, hy, hz);
        }
      }
    }
  }
}

// The three steps shared by every form: w = y / delta + c, the magic-number
// rounding of w and the lattice index t of both pairs, with the x axis on
// packed FP32 pairs (fma.rn.f32x2 / add.rn.f32x2) and the y and z axes either
// packed too (DSES_VOTE2_HEAD_P: fewest instructions), or z (DSES_VOTE2_HEAD_Z)
// or y and z (DSES_VOTE2_HEAD_S) as scalar FP32 on each half: the packed
// operations issue to the FMA-heavy pipe only, scalar ones to either FMA pipe.
// Measured: the culled vote's list loop fastest with HEAD_Z (1.4% ahead of
// HEAD_S, 5% ahead of HEAD_P), its direct form with HEAD_S (2% ahead of
// HEAD_Z), the dense 16-bit vote with HEAD_P (HEAD_S 6% slower). Every form
// rounds each value once, identically. Box
// test: |w_a| < h_a on every axis, either per axis (three chained compares) or,
// when the padded box is a cube, as max(|w_x|, |w_y|, |w_z|) < h (one
// three-input max and one compare).
#define DSES_VOTE2_DECL                                                                          \
  "{\n\t.reg .b64 wx, wy, wz, fx, fy, fz;\n\t"                                                   \
  ".reg .b32 bx0, bx1, by0, by1, bz0, bz1, t0, t1, a0, a1, i0, i1, u0, u1, v0, v1, s0, s1;\n\t"  \
  ".reg .f32 x0, x1, y0, y1, z0, z1;\n\t.reg .pred p0, p1;\n\t"
#define DSES_VOTE2_HEAD_P                                                                        \
  DSES_VOTE2_DECL                                                                                \
  "fma.rn.f32x2 wx, %0, %3, %4;\n\tfma.rn.f32x2 wy, %1, %3, %5;\n\tfma.rn.f32x2 wz, %2, %3, %6;\n\t" \
  "add.rn.f32x2 fx, wx, %7;\n\tadd.rn.f32x2 fy, wy, %8;\n\tadd.rn.f32x2 fz, wz, %9;\n\t"         \
  "mov.b64 {bx0, bx1}, fx;\n\tmov.b64 {by0, by1}, fy;\n\tmov.b64 {bz0, bz1}, fz;\n\t"
#define DSES_VOTE2_HEAD_S                                                                        \
  DSES_VOTE2_DECL                                                                                \
  ".reg .f32 j0, j1, qy0, qy1, cy0, cy1, my0, my1, wy0, wy1, gy0, gy1;\n\t"                      \
  ".reg .f32 qz0, qz1, cz0, cz1, mz0, mz1, wz0, wz1, gz0, gz1;\n\t"                              \
  "fma.rn.f32x2 wx, %0, %3, %4;\n\tadd.rn.f32x2 fx, wx, %7;\n\t"                                 \
  "mov.b64 {j0, j1}, %3;\n\t"                                                                    \
  "mov.b64 {qy0, qy1}, %1;\n\tmov.b64 {cy0, cy1}, %5;\n\tmov.b64 {my0, my1}, %8;\n\t"            \
  "fma.rn.f32 wy0, qy0, j0, cy0;\n\tfma.rn.f32 wy1, qy1, j1, cy1;\n\t"                           \
  "add.rn.f32 gy0, wy0, my0;\n\tadd.rn.f32 gy1, wy1, my1;\n\t"                                   \
  "mov.b64 {qz0, qz1}, %2;\n\tmov.b64 {cz0, cz1}, %6;\n\tmov.b64 {mz0, mz1}, %9;\n\t"            \
  "fma.rn.f32 wz0, qz0, j0, cz0;\n\tfma.rn.f32 wz1, qz1, j1, cz1;\n\t"                           \
  "add.rn.f32 gz0, wz0, mz0;\n\tadd.rn.f32 gz1, wz1, mz1;\n\t"                                   \
  "mov.b64 wy, {wy0, wy1};\n\tmov.b64 wz, {wz0, wz1};\n\t"                                       \
  "mov.b64 {bx0, bx1}, fx;\n\tmov.b32 by0, gy0;\n\tmov.b32 by1, gy1;\n\t"                        \
  "mov.b32 bz0, gz0;\n\tmov.b32 bz1, gz1;\n\t"
#define DSES_VOTE2_HEAD_Z                                                                        \
  DSES_VOTE2_DECL                                                                                \
  ".reg .f32 j0, j1, qz0, qz1, cz0, cz1, mz0, mz1, wz0, wz1, gz0, gz1;\n\t"                      \
  "fma.rn.f32x2 wx, %0, %3, %4;\n\tfma.rn.f32x2 wy, %1, %3, %5;\n\t"                             \
  "add.rn.f32x2 fx, wx, %7;\n\tadd.rn.f32x2 fy, wy, %8;\n\t"                                     \
  "mov.b64 {j0, j1}, %3;\n\t"                                                                    \
  "mov.b64 {qz0, qz1}, %2;\n\tmov.b64 {cz0, cz1}, %6;\n\tmov.b64 {mz0, mz1}, %9;\n\t"            \
  "fma.rn.f32 wz0, qz0, j0, cz0;\n\tfma.rn.f32 wz1, qz1, j1, cz1;\n\t"                           \
  "add.rn.f32 gz0, wz0, mz0;\n\tadd.rn.f32 gz1, wz1, mz1;\n\t"                                   \
  "mov.b64 wz, {wz0, wz1};\n\t"                                                                  \
  "mov.b64 {bx0, bx1}, fx;\n\tmov.b64 {by0, by1}, fy;\n\t"                                       \
  "mov.b32 bz0, gz0;\n\tmov.b32 bz1, gz1;\n\t"
// 16-bit counters: word t >> 1 (address = base + 4 word), half t & 1: the
// increment 1 << 16 (t & 1) is a funnel shift by (t << 4) mod 32; the
// multiplies of the bin index are the only work on the FMA-heavy pipe
#define DSES_VOTE2_ADDR16                                                                     \
  "mad.lo.u32 t0, by0, %11, bz0;\n\tmad.lo.u32 t0, bx0, %10, t0;\n\t"                        \
  "mad.lo.u32 t1, by1, %11, bz1;\n\tmad.lo.u32 t1, bx1, %10, t1;\n\t"                        \
  "shr.u32 a0, t0, 1;\n\tshr.u32 a1, t1, 1;\n\t"                                             \
  "shl.b32 a0, a0, 2;\n\tshl.b32 a1, a1, 2;\n\tadd.u32 a0, a0, %12;\n\tadd.u32 a1, a1, %12;\n\t" \
  "shl.b32 i0, t0, 4;\n\tshl.b32 i1, t1, 4;\n\t"                                             \
  "shf.l.wrap.b32 i0, 0, 1, i0;\n\tshf.l.wrap.b32 i1, 0, 1, i1;\n\t"
// 32-bit counters: base + 4 kz + %11 ky + %10 kx (strides %10 / %11 in bytes)
#define DSES_VOTE2_ADDR32                                                                      \
  "shl.b32 t0, bz0, 2;\n\tadd.u32 t0, t0, %12;\n\tmad.lo.u32 t0, by0, %11, t0;\n\tmad.lo.u32 a0, bx0, %10, t0;\n\t" \
  "shl.b32 t1, bz1, 2;\n\tadd.u32 t1, t1, %12;\n\tmad.lo.u32 t1, by1, %11, t1;\n\tmad.lo.u32 a1, bx1, %10, t1;\n\t"
#define DSES_VOTE2_ABS                                                                      \
  "mov.b64 {u0, u1}, wx;\n\tmov.b64 {v0, v1}, wy;\n\tmov.b64 {s0, s1}, wz;\n\t"             \
  "mov.b32 x0, u0;\n\tmov.b32 x1, u1;\n\tmov.b32 y0, v0;\n\tmov.b32 y1, v1;\n\t"           \
  "mov.b32 z0, s0;\n\tmov.b32 z1, s1;\n\t"                                                  \
  "abs.f32 x0, x0;\n\tabs.f32 x1, x1;\n\tabs.f32 y0, y0;\n\tabs.f32 y1, y1;\n\t"           \
  "abs.f32 z0, z0;\n\tabs.f32 z1, z1;\n\t"
#define DSES_VOTE2_TEST_AXES                                                                          \
  "setp.lt.f32 p0, x0, %13;\n\tsetp.lt.and.f32 p0, y0, %14, p0;\n\tsetp.lt.and.f32 p0, z0, %15, p0;\n\t" \
  "setp.lt.f32 p1, x1, %13;\n\tsetp.lt.and.f32 p1, y1, %14, p1;\n\tsetp.lt.and.f32 p1, z1, %15, p1;\n\t"
#define DSES_VOTE2_TEST_CUBE                                                 \
  "max.f32 x0, x0, y0, z0;\n\tmax.f32 x1, x1, y1, z1;\n\t"                   \
  "setp.lt.f32 p0, x0, %13;\n\tsetp.lt.f32 p1, x1, %13;\n\t"
// a pair outside the box adds to the lane's sink word %16
#define DSES_VOTE2_RED16                                                     \
  "selp.b32 a0, a0, %16, p0;\n\tselp.b32 a1, a1, %16, p1;\n\t"               \
  "red.shared.add.u32 [a0], i0;\n\tred.shared.add.u32 [a1], i1;\n\t}"
#define DSES_VOTE2_RED32                                                     \
  "selp.b32 a0, a0, %16, p0;\n\tselp.b32 a1, a1, %16, p1;\n\t"               \
  "red.shared.add.u32 [a0], 1;\n\tred.shared.add.u32 [a1], 1;\n\t}"

// Two (source, target) pairs as packed FP32 pairs: lattice index, box test and
// one unconditional shared add per pair (shared 16- or 32-bit counters; the
// lane-private layout takes the scalar path). FORM: 0 every axis packed
// (DSES_VOTE2_HEAD_P), 1 z scalar (DSES_VOTE2_HEAD_Z), 2 y and z scalar
// (DSES_VOTE2_HEAD_S).
template <bool U16, bool CUBE, int FORM>
__device__ __forceinline__ void vote_two_pairs(uint64_t yx, uint64_t yy, uint64_t yz, uint64_t inv2, uint64_t cx2,
                                               uint64_t cy2, uint64_t cz2, uint64_t mx2, uint64_t my2, uint64_t mz2,
                                               uint32_t Sx, uint32_t Sy, uint32_t abase, float hx, float hy,
                                               float hz, uint32_t adummy) {
  const uint32_t sy = U16 ? Sx : Sx * 4u, sz = U16 ? Sy : Sy * 4u;
#define DSES_VOTE2_ARGS                                                                                         \
  ::"l"(yx), "l"(yy), "l"(yz), "l"(inv2), "l"(cx2), "l"(cy2), "l"(cz2), "l"(mx2), "l"(my2), "l"(mz2), "r"(sy), \
      "r"(sz), "r"(abase), "f"(hx), "f"(hy), "f"(hz), "r"(adummy)
#define DSES_VOTE2_FORMS(HEAD)                                                                                   \
  if (U16 && CUBE)                                                                                               \
    asm volatile(HEAD DSES_VOTE2_ADDR16 DSES_VOTE2_ABS DSES_VOTE2_TEST_CUBE DSES_VOTE2_RED16 DSES_VOTE2_ARGS);   \
  else if (U16)                                                                                                  \
    asm volatile(HEAD DSES_VOTE2_ADDR16 DSES_VOTE2_ABS DSES_VOTE2_TEST_AXES DSES_VOTE2_RED16 DSES_VOTE2_ARGS);   \
  else if (CUBE)                                                                                                 \
    asm volatile(HEAD DSES_VOTE2_ADDR32 DSES_VOTE2_ABS DSES_VOTE2_TEST_CUBE DSES_VOTE2_RED32 DSES_VOTE2_ARGS);   \
  else                                                                                                           \
    asm volatile(HEAD DSES_VOTE2_ADDR32 DSES_VOTE2_ABS DSES_VOTE2_TEST_AXES DSES_VOTE2_RED32 DSES_VOTE2_ARGS);
  if (FORM == 2) {
    DSES_VOTE2_FORMS(DSES_VOTE2_HEAD_S)
  } else if (FORM == 1) {
    DSES_VOTE2_FORMS(DSES_VOTE2_HEAD_Z)
  } else {
    DSES_VOTE2_FORMS(DSES_VOTE2_HEAD_P)
  }
#undef DSES_VOTE2_FORMS
#undef DSES_VOTE2_ARGS
}

__device__ __forceinline__ uint64_t pack2(float lo, float hi) {
  return ((uint64_t)__float_as_uint(hi) << 32) | (uint64_t)__float_as_uint(lo);
}

// Sources [i0, i1) against a lane's Q target pairs (dense packed path). The
// staged layout of source i: float4 [2i] holds (c_x, c_x, c_y, c_y), float4
// [2i + 1] holds (c_z, c_z, 0, 0).
template <int Q, bool U16, bool CUBE>
__device__ __forceinline__ void vote_sources_x2(const float4* __restrict__ srcd, int i0, int i1, const uint64_t* yx,
                                                const uint64_t* yy, const uint64_t* yz, uint64_t inv2, uint64_t mx2,
                                                uint64_t my2, uint64_t mz2, uint32_t Sx, uint32_t Sy, uint32_t abase,
                                                float hx, float hy, float hz, uint32_t adummy) {
#pragma unroll 4
  for (int i = i0; i < i1; ++i) {
    const float4 ca = srcd[2 * i];
    const float2 cb = *reinterpret_cast<const float2*>(srcd + 2 * i + 1);
    const uint64_t cx2 = pack2(ca.x, ca.y), cy2 = pack2(ca.z, ca.w), cz2 = pack2(cb.x, cb.y);
#pragma unroll
    for (int q = 0; q < Q; ++q)
      vote_two_pairs<U16, CUBE, U16 ? 0 : 2>(yx[q], yy[q], yz[q], inv2, cx2, cy2, cz2, mx2, my2, mz2, Sx, Sy, abase,
                                             hx, hy, hz, adummy);
  }
}

// Dense centred path on packed FP32 pairs (fma.rn.f32x2 / add.rn.f32x2): a
// lane's targets are held two by two per axis and each source offset is staged
// duplicated, so one packed op computes the lattice coordinate (or its
// rounding) of one source against two targets. Same per-pair arithmetic and
// box test as vote_centred; the histogram increment is unconditional, with the
// address selected by the box test (a pair outside the box adds to a per-lane
// sink word that is never read), which keeps the loop free of branches around
// the atomic. A cubic box takes the three-input-max test (DENSE_INST: only in
// the dense kernel instances; the culled instances, which reach this path for
// problems that are not culled, keep one form: their culled loops measured 1%
// slower with both forms in the kernel).
template <int P, bool U16, bool DENSE_INST>
__device__ __forceinline__ void vote_centred_x2(const PassDesc& d, const float4* __restrict__ srcd, int nsrc,
                                                unsigned SX, uint32_t hist_base, int* item_ctr, int lane,
                                                uint32_t sink) {
  static_assert(P % 2 == 0, "targets are packed two by two");
  const int n_tchunks = d.n_tchunks, n_sgroups = d.n_sgroups;
  const int n_items = n_tchunks * n_sgroups;
  const int spg = (nsrc + n_sgroups - 1) / n_sgroups;
  const unsigned Ey = (unsigned)d.E[1], Ez = (unsigned)d.E[2];
  const uint32_t Sx = d.hs[0], Sy = d.hs[1];  // bins per x-plane and per y-row of the layout
  const float inv = d.inv_delta;
  const float hx = 0.5f * (float)SX, hy = 0.5f * (float)Ey, hz = 0.5f * (float)Ez;
  const bool cube = SX == Ey && Ey == Ez;  // one half-width for the three axes
  const float mx = kMagic + (float)((SX - 1) / 2), my = kMagic + (float)((Ey - 1) / 2),
              mz = kMagic + (float)((Ez - 1) / 2);
  const uint64_t inv2 = pack2(inv, inv), mx2 = pack2(mx, mx), my2 = pack2(my, my), mz2 = pack2(mz, mz);
  const uint32_t bias = kMagicBits * (Sx + Sy + 1u);
  // shared counters (the lane-private layout takes the scalar path)
  const uint32_t abase = U16 ? hist_base - 2u * bias : hist_base - 4u * bias;
  // a pair outside the box adds to this lane's sink word outside the
  // histogram instead (no branch, and the increment needs no select)
  const uint32_t adummy = sink + 4u * (uint32_t)lane;
  for (int it = next_item(item_ctr, lane); it < n_items; it = next_item(item_ctr, lane)) {
    const int tc = it % n_tchunks, sg = it / n_tchunks;
    float ty[P][3];
    load_targets(d.Yv, d.M, tc * P * 32, lane, P, ty);
    uint64_t yx[P / 2], yy[P / 2], yz[P / 2];
#pragma unroll
    for (int q = 0; q < P / 2; ++q) {
      yx[q] = pack2(ty[2 * q][0], ty[2 * q + 1][0]);
      yy[q] = pack2(ty[2 * q][1], ty[2 * q + 1][1]);
      yz[q] = pack2(ty[2 * q][2], ty[2 * q + 1][2]);
    }
    const int i0 = sg * spg, i1 = min(i0 + spg, nsrc);
    if (DENSE_INST && cube)
      vote_sources_x2<P / 2, U16, true>(srcd, i0, i1, yx, yy, yz, inv2, mx2, my2, mz2, Sx, Sy, abase, hx, hy, hz,
                                       adummy);
    else
      vote_sources_x2<P / 2, U16, false>(srcd, i0, i1, yx, yy, yz, inv2, mx2, my2, mz2, Sx, Sy, abase, hx, hy, hz,
                                        adummy);
  }
}

// Keep windows of an item's G target groups (groups tc G .. tc G + G - 1 of
// d.gbox): a staged source offset c keeps group g iff t[2a] <= c_a <= t[2a+1]
// on every axis (8 floats per group at thr + 8 g; a missing group keeps
// nothing). Lanes 0 .. G - 1 write one group each.
template <int G>
__device__ __forceinline__ void item_windows(const PassDesc& d, int tc, int lane, float* thr, float hx, float hy,
                                             float hz, float inv) {
  if (lane < G) {
    const int g = tc * G + lane;
    float* t = thr + 8 * lane;
    if (g < d.n_groups) {
      const float4 lo = __ldg(d.gbox + 2 * g), hi = __ldg(d.gbox + 2 * g + 1);
      const float m = d.cull_margin;
      t[0] = -hx - m - hi.x * inv; t[1] = hx + m - lo.x * inv;
      t[2] = -hy - m - hi.y * inv; t[3] = hy + m - lo.y * inv;
      t[4] = -hz - m - hi.z * inv; t[5] = hz + m - lo.z * inv;
    } else {
      t[0] = t[2] = t[4] = INFINITY;
      t[1] = t[3] = t[5] = -INFINITY;
    }
  }
}

// Can a block of 32 staged sources keep one of an item's G groups? b holds
// the block's offset bounds (lo_x, hi_x, lo_y, hi_y, lo_z, hi_z), thr the
// groups' windows (8 floats each, same order). A block whose bounds miss every
// window on some axis holds no source that keeps a group (the per-source test
// compares the same values), so it is skipped whole.
template <int G>
__device__ __forceinline__ bool block_keeps(const float* __restrict__ b, const float* __restrict__ thr) {
  const float4 b0 = *reinterpret_cast<const float4*>(b);
  const float2 b1 = *reinterpret_cast<const float2*>(b + 4);
  bool any = false;
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const float4 u0 = *reinterpret_cast<const float4*>(thr + 8 * g);
    const float2 u1 = *reinterpret_cast<const float2*>(thr + 8 * g + 4);
    any |= (b0.y >= u0.x) & (b0.x <= u0.y) & (b0.w >= u0.z) & (b0.z <= u0.w) & (b1.y >= u1.x) & (b1.x <= u1.y);
  }
  return any;
}

// Sparse centred path, for translation boxes small against the target: the
// P x 32 targets of an item are P groups of 32 consecutive points (in the
// vote's target order) with known bounding boxes. For each block of 32
// sources the lanes test (source, group) pairs against the source's
// translation window, widened by a margin of d.cull_margin lattice units (far
// above the FP32 roundings of w, the staged offsets and the thresholds, so no
// pair that could vote is dropped); only surviving (source, group) pairs are
// voted, one group at a time over the set bits of its ballot.

template <int P, bool U16, bool CUBE>
__device__ __forceinline__ void vote_centred_sparse(const PassDesc& d, const float4* __restrict__ srcc, int nsrc,
                                                    unsigned SX, uint32_t hist_base, int* item_ctr, int lane,
                                                    float* __restrict__ thr, uint32_t sink,
                                                    const float* __restrict__ blkp) {
  const int n_tchunks = d.n_tchunks, n_sgroups = d.n_sgroups;
  const int n_items = n_tchunks * n_sgroups;
  const int spg = (nsrc + n_sgroups - 1) / n_sgroups;
  const unsigned Ey = (unsigned)d.E[1], Ez = (unsigned)d.E[2];
  const uint32_t Sx = d.hs[0], Sy = d.hs[1];  // bins per x-plane and per y-row of the layout
  const float inv = d.inv_delta;
  const float hx = 0.5f * (float)SX, hy = 0.5f * (float)Ey, hz = 0.5f * (float)Ez;
  const float mx = kMagic + (float)((SX - 1) / 2), my = kMagic + (float)((Ey - 1) / 2),
              mz = kMagic + (float)((Ez - 1) / 2);
  const uint32_t bias = kMagicBits * (Sx + Sy + 1u);
  const uint32_t unit = d.hist_lanes ? 128u : 4u;
  const uint32_t SxU = Sx * unit, SyU = Sy * unit;
  const uint32_t abase32 = hist_base + (d.hist_lanes ? 4u * (uint32_t)lane : 0u) - unit * bias;
  const uint32_t abase16 = hist_base - 2u * bias;
  const uint32_t sinkl = sink + 4u * (uint32_t)lane;
  for (int it = next_item(item_ctr, lane); it < n_items; it = next_item(item_ctr, lane)) {
    const int tc = it % n_tchunks, sg = it / n_tchunks;
    float ty[P][3];
    load_targets(d.Yv, d.M, tc * P * 32, lane, P, ty);
    item_windows<P>(d, tc, lane, thr, hx, hy, hz, inv);
    __syncwarp();
    const int i0 = sg * spg, i1 = min(i0 + spg, nsrc);
    // the aligned blocks of 32 staged sources that meet [i0, i1), 32 at a
    // time: a lane tests one block's bounds, and only blocks that can keep a
    // group are walked
    for (int bb = i0 >> 5; bb < ((i1 + 31) >> 5); bb += 32) {
      const int myb = bb + lane;
      bool rel = myb < ((i1 + 31) >> 5);
      if (blkp && rel) rel = block_keeps<P>(blkp + 8 * myb, thr);
      uint32_t bmask = __ballot_sync(0xffffffffu, rel);
      while (bmask) {
        const int s0 = (bb + __ffs(bmask) - 1) << 5;
        bmask &= bmask - 1;
        const int mine = s0 + lane;  // the aligned block may start before i0
        const bool valid = mine >= i0 && mine < i1;
        const float4 cm = srcc[valid ? mine : i0];
        uint32_t kmask[P];
#pragma unroll
        for (int p = 0; p < P; ++p) {
          const float4 ta = *reinterpret_cast<const float4*>(thr + 8 * p);
          const float2 tb = *reinterpret_cast<const float2*>(thr + 8 * p + 4);
          const bool keep = valid & (cm.x >= ta.x) & (cm.x <= ta.y) & (cm.y >= ta.z) & (cm.y <= ta.w) &
                            (cm.z >= tb.x) & (cm.z <= tb.y);
          kmask[p] = __ballot_sync(0xffffffffu, keep);
        }
#pragma unroll
        for (int p = 0; p < P; ++p) {
          uint32_t m = kmask[p];
          while (m) {
            const int j = __ffs(m) - 1;
            m &= m - 1;
            const float4 c = srcc[s0 + j];
            const float wx = __fmaf_rn(ty[p][0], inv, c.x);
            const float wy = __fmaf_rn(ty[p][1], inv, c.y);
            const float wz = __fmaf_rn(ty[p][2], inv, c.z);
            const uint32_t bx = __float_as_uint(__fadd_rn(wx, mx));
            const uint32_t by = __float_as_uint(__fadd_rn(wy, my));
            const uint32_t bz = __float_as_uint(__fadd_rn(wz, mz));
            if (U16) {
              const uint32_t b = bx * Sx + (by * Sy + bz);
              red_or_sink<CUBE>(abase16 + ((b >> 1) << 2), 1u + (b & 1u) * 0xffffu, sinkl, wx, wy, wz, hx, hy, hz);
            } else {
              red_or_sink<CUBE>(abase32 + bx * SxU + (by * SyU + bz * unit), 1u, sinkl, wx, wy, wz, hx, hy, hz);
            }
          }
        }
      }
    }
    __syncwarp();
  }
}

// One kept source against a lane's target pair of each of G groups: its
// staged pairs (c_x, c_x), (c_y, c_y), (c_z, c_z) read from the tile layout at
// shared address a (a + 64, a + 128).
template <int G, bool U16, bool CUBE, int FORM>
__device__ __forceinline__ void vote_staged(uint32_t a, const uint64_t* yx, const uint64_t* yy, const uint64_t* yz,
                                            uint64_t inv2, uint64_t mx2, uint64_t my2, uint64_t mz2, uint32_t Sx,
                                            uint32_t Sy, uint32_t abase, float hx, float hy, float hz,
                                            uint32_t adummy) {
  uint64_t cx2, cy2, cz2;
  asm("ld.shared.b64 %0, [%3];\n\tld.shared.b64 %1, [%3+64];\n\tld.shared.b64 %2, [%3+128];"
      : "=l"(cx2), "=l"(cy2), "=l"(cz2)
      : "r"(a));
#pragma unroll
  for (int g = 0; g < G; ++g)
    vote_two_pairs<U16, CUBE, FORM>(yx[g], yy[g], yz[g], inv2, cx2, cy2, cz2, mx2, my2, mz2, Sx, Sy, abase, hx, hy,
                                    hz, adummy);
}

// The n kept sources of a list against the lane's target pairs of G groups,
// four per iteration (the list is 16-byte aligned; z coordinates in scalar
// FP32, DSES_VOTE2_HEAD_Z).
template <int G, bool U16, bool CUBE>
__device__ __forceinline__ void vote_list(const uint32_t* __restrict__ lst, int n, const uint64_t* yx,
                                          const uint64_t* yy, const uint64_t* yz, uint64_t inv2, uint64_t mx2,
                                          uint64_t my2, uint64_t mz2, uint32_t Sx, uint32_t Sy, uint32_t abase,
                                          float hx, float hy, float hz, uint32_t adummy) {
  int k = 0;
#pragma unroll 1
  for (; k + 4 <= n; k += 4) {
    const uint4 a = *reinterpret_cast<const uint4*>(lst + k);
    vote_staged<G, U16, CUBE, 1>(a.x, yx, yy, yz, inv2, mx2, my2, mz2, Sx, Sy, abase, hx, hy, hz, adummy);
    vote_staged<G, U16, CUBE, 1>(a.y, yx, yy, yz, inv2, mx2, my2, mz2, Sx, Sy, abase, hx, hy, hz, adummy);
    vote_staged<G, U16, CUBE, 1>(a.z, yx, yy, yz, inv2, mx2, my2, mz2, Sx, Sy, abase, hx, hy, hz, adummy);
    vote_staged<G, U16, CUBE, 1>(a.w, yx, yy, yz, inv2, mx2, my2, mz2, Sx, Sy, abase, hx, hy, hz, adummy);
  }
#pragma unroll 1
  for (; k < n; ++k)
    vote_staged<G, U16, CUBE, 1>(lst[k], yx, yy, yz, inv2, mx2, my2, mz2, Sx, Sy, abase, hx, hy, hz, adummy);
}

// Shared address of staged source i's offsets in the tile layout.
__device__ __forceinline__ uint32_t tile_entry(uint32_t tbase, int i) {
  return tbase + (uint32_t)((i / kTileSources) * kTileBytes + 8 * (i % kTileSources));
}

// Appends the lanes whose flag is set to a warp's list (each at its rank in
// the ballot); n is the list's length, the same in every lane.
__device__ __forceinline__ void list_push(uint32_t* __restrict__ lst, int& n, bool flag, uint32_t entry,
                                          uint32_t lanes_below) {
  const uint32_t m = __ballot_sync(0xffffffffu, flag);
  if (flag) lst[n + __popc(m & lanes_below)] = entry;
  n += __popc(m);
}

// Paired culled path, for windows that span many target groups (large
// targets: the robot-like problem): groups of 64 consecutive targets
// (d.gbox / d.n_groups hold the 64-point boxes in this mode), a lane holding
// two of each of its item's P / 2 groups (points 64 g + lane and 64 g + 32 +
// lane) as a packed FP32 pair; each kept source votes a group's 64 targets in
// one packed step. Against the 32-point path this halves the iterations per
// kept target but keeps more (source, group) pairs, so it pays only when the
// window is large against a group. Sources are staged in tiles of 8 (their
// duplicated offsets, one 8-byte pair per axis: the keep tests of 32
// consecutive sources read two words per bank, a vote step three uniform
// 8-byte loads). The kept sources of each 32-source block gather in the warp's
// lists: a source kept by both of an item's groups is read once and votes
// both; the lists are voted once one holds kPairedListFlush entries, and at
// the end of the item (DIRECT, for items of a few sources: each block's kept
// sources are voted at once, without the lists). A cubic padded box takes the
// three-input-max box test (CUBE, an instantiation of its own: with the
// choice made per step the loop ran 11% slower).
template <int P, bool U16, bool CUBE, bool DIRECT>
__device__ __forceinline__ void vote_centred_paired(const PassDesc& d, const float* __restrict__ srct, int nsrc,
                                                    unsigned SX, uint32_t hist_base, int* item_ctr, int lane,
                                                    float* __restrict__ thr, uint32_t sink,
                                                    const float* __restrict__ blkp, uint32_t* __restrict__ lst) {
  static_assert(P == 2 || P == 4, "two targets of each of P / 2 groups per lane");
  constexpr int Q = P / 2;            // 64-point groups per item
  constexpr int NL = Q == 2 ? 3 : 1;  // lists: first group only, second only, both
  const int n_tchunks = d.n_tchunks, n_sgroups = d.n_sgroups;
  const int n_items = n_tchunks * n_sgroups;
  const int spg = (nsrc + n_sgroups - 1) / n_sgroups;
  const unsigned Ey = (unsigned)d.E[1], Ez = (unsigned)d.E[2];
  const uint32_t Sx = d.hs[0], Sy = d.hs[1];  // bins per x-plane and per y-row of the layout
  const float inv = d.inv_delta;
  // a cubic box has one half-width and one rounding constant (fewer live registers)
  const float hx = 0.5f * (float)SX, hy = CUBE ? hx : 0.5f * (float)Ey, hz = CUBE ? hx : 0.5f * (float)Ez;
  const float mx = kMagic + (float)((SX - 1) / 2), my = CUBE ? mx : kMagic + (float)((Ey - 1) / 2),
              mz = CUBE ? mx : kMagic + (float)((Ez - 1) / 2);
  const uint64_t inv2 = pack2(inv, inv), mx2 = pack2(mx, mx), my2 = CUBE ? mx2 : pack2(my, my),
                 mz2 = CUBE ? mx2 : pack2(mz, mz);
  const uint32_t bias = kMagicBits * (Sx + Sy + 1u);
  // shared counters (the planner keeps the lane-private layout off this path)
  const uint32_t abase = U16 ? hist_base - 2u * bias : hist_base - 4u * bias;
  const uint32_t adummy = sink + 4u * (uint32_t)lane;
  const uint32_t lt = (1u << lane) - 1u;
  const uint32_t tbase = (uint32_t)__cvta_generic_to_shared(srct);

  for (int it = next_item(item_ctr, lane); it < n_items; it = next_item(item_ctr, lane)) {
    const int tc = it % n_tchunks, sg = it / n_tchunks;
    item_windows<Q>(d, tc, lane, thr, hx, hy, hz, inv);
    __syncwarp();
    // the lane's target pairs, one per group; padding lanes never vote
    uint64_t yx[Q], yy[Q], yz[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int j0 = (tc * Q + q) * 64 + lane, j1 = j0 + 32;
      const float4 a = j0 < d.M ? __ldg(d.Yv + j0) : make_float4(1e30f, 1e30f, 1e30f, 0.f);
      const float4 b = j1 < d.M ? __ldg(d.Yv + j1) : make_float4(1e30f, 1e30f, 1e30f, 0.f);
      yx[q] = pack2(a.x, b.x);
      yy[q] = pack2(a.y, b.y);
      yz[q] = pack2(a.z, b.z);
    }
    const int i0 = sg * spg, i1 = min(i0 + spg, nsrc);
    int cnt[NL];
#pragma unroll
    for (int l = 0; l < NL; ++l) cnt[l] = 0;
    // the aligned blocks of 32 staged sources that meet [i0, i1), 32 at a
    // time: a lane tests one block's bounds, and only blocks that can keep a
    // group are walked
    for (int bb = i0 >> 5; bb < ((i1 + 31) >> 5); bb += 32) {
      const int myb = bb + lane;
      bool rel = myb < ((i1 + 31) >> 5);
      if (blkp && rel) rel = block_keeps<Q>(blkp + 8 * myb, thr);
      uint32_t bmask = __ballot_sync(0xffffffffu, rel);
      while (bmask) {
        const int s0 = (bb + __ffs(bmask) - 1) << 5;
        bmask &= bmask - 1;
        const int mine = s0 + lane;  // the aligned block may start before i0
        const bool valid = mine >= i0 && mine < i1;
        const int ms = valid ? mine : i0;
        const int o = (ms / kTileSources) * (kTileBytes / 4) + 2 * (ms % kTileSources);
        const float cx = srct[o], cy = srct[o + 16], cz = srct[o + 32];
        bool keep[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const float4 ta = *reinterpret_cast<const float4*>(thr + 8 * q);
          const float2 tb = *reinterpret_cast<const float2*>(thr + 8 * q + 4);
          // bitwise (no short-circuit branches): one predicate chain per group
          keep[q] = valid & (cx >= ta.x) & (cx <= ta.y) & (cy >= ta.z) & (cy <= ta.w) & (cz >= tb.x) & (cz <= tb.y);
        }
        if constexpr (DIRECT) {
          // few sources per item: vote this block's kept sources at once
          const uint32_t k0 = __ballot_sync(0xffffffffu, keep[0]);
          const uint32_t k1 = Q == 2 ? __ballot_sync(0xffffffffu, keep[Q - 1]) : 0u;
          uint32_t mb = k0 & k1, m0 = k0 & ~k1, m1 = k1 & ~k0;
          while (mb) {
            const int jj = s0 + __ffs(mb) - 1;
            mb &= mb - 1;
            vote_staged<Q, U16, CUBE, 2>(tile_entry(tbase, jj), yx, yy, yz, inv2, mx2, my2, mz2, Sx, Sy, abase, hx, hy,
                                      hz, adummy);
          }
          while (m0) {
            const int jj = s0 + __ffs(m0) - 1;
            m0 &= m0 - 1;
            vote_staged<1, U16, CUBE, 2>(tile_entry(tbase, jj), yx, yy, yz, inv2, mx2, my2, mz2, Sx, Sy, abase, hx, hy,
                                      hz, adummy);
          }
          while (m1) {
            const int jj = s0 + __ffs(m1) - 1;
            m1 &= m1 - 1;
            vote_staged<1, U16, CUBE, 2>(tile_entry(tbase, jj), yx + Q - 1, yy + Q - 1, yz + Q - 1, inv2, mx2, my2, mz2,
                                      Sx, Sy, abase, hx, hy, hz, adummy);
          }
        } else {
          const uint32_t entry = tbase + 4u * (uint32_t)o;
          if constexpr (Q == 2) {
            list_push(lst, cnt[0], keep[0] && !keep[1], entry, lt);
            list_push(lst + kPairedListCap, cnt[1], keep[1] && !keep[0], entry, lt);
            list_push(lst + 2 * kPairedListCap, cnt[2], keep[0] && keep[1], entry, lt);
          } else {
            list_push(lst, cnt[0], keep[0], entry, lt);
          }
          __syncwarp();
          // a list holds at most kPairedListFlush - 1 + 32 entries before its vote
          bool full = cnt[0] >= kPairedListFlush;
          if constexpr (Q == 2) full |= (cnt[1] >= kPairedListFlush) | (cnt[2] >= kPairedListFlush);
          if (full) {
            if (cnt[0] >= kPairedListFlush) {
              vote_list<1, U16, CUBE>(lst, cnt[0], yx, yy, yz, inv2, mx2, my2, mz2, Sx, Sy, abase, hx, hy, hz, adummy);
              cnt[0] = 0;
              __syncwarp();  // read before the next block rewrites the list
            }
            if constexpr (Q == 2) {
              if (cnt[1] >= kPairedListFlush) {
                vote_list<1, U16, CUBE>(lst + kPairedListCap, cnt[1], yx + 1, yy + 1, yz + 1, inv2, mx2, my2, mz2, Sx, Sy,
                                        abase, hx, hy, hz, adummy);
                cnt[1] = 0;
                __syncwarp();
              }
              if (cnt[2] >= kPairedListFlush) {
                vote_list<2, U16, CUBE>(lst + 2 * kPairedListCap, cnt[2], yx, yy, yz, inv2, mx2, my2, mz2, Sx, Sy, abase,
                                        hx, hy, hz, adummy);
                cnt[2] = 0;
                __syncwarp();
              }
            }
          }
        }
      }
    }
    if (cnt[0])
      vote_list<1, U16, CUBE>(lst, cnt[0], yx, yy, yz, inv2, mx2, my2, mz2, Sx, Sy, abase, hx, hy, hz, adummy);
    if constexpr (Q == 2) {
      if (cnt[1])
        vote_list<1, U16, CUBE>(lst + kPairedListCap, cnt[1], yx + 1, yy + 1, yz + 1, inv2, mx2, my2, mz2, Sx, Sy,
                                abase, hx, hy, hz, adummy);
      if (cnt[2])
        vote_list<2, U16, CUBE>(lst + 2 * kPairedListCap, cnt[2], yx, yy, yz, inv2, mx2, my2, mz2, Sx, Sy, abase, hx,
                                hy, hz, adummy);
    }
    __syncwarp();
  }
}

// Generic path (any extents): k_a = floor(w_a) by a round-down add, box test on
// the integer indices. The engine pads every layout to odd extents (centred
// paths); this serves dses_vote_static boxes with an even extent.
template <int P, bool U16>
__device__ __forceinline__ void vote_generic(const PassDesc& d, const float4* __restrict__ srcc, int nsrc,
                                             unsigned SX, uint32_t* __restrict__ hist, int* item_ctr, int lane) {
  const int n_tchunks = d.n_tchunks, n_sgroups = d.n_sgroups;
  const int n_items = n_tchunks * n_sgroups;
  const int spg = (nsrc + n_sgroups - 1) / n_sgroups;
  const unsigned Ey = (unsigned)d.E[1], Ez = (unsigned)d.E[2];
  const float inv = d.inv_delta;
  const unsigned bstride = d.hist_lanes ? 32u : 1u, boff = d.hist_lanes ? (unsigned)lane : 0u;
  for (int it = next_item(item_ctr, lane); it < n_items; it = next_item(item_ctr, lane)) {
    const int tc = it % n_tchunks, sg = it / n_tchunks;
    float ty[P][3];
    load_targets(d.Yv, d.M, tc * P * 32, lane, P, ty);
    const int i0 = sg * spg, i1 = min(i0 + spg, nsrc);
    for (int i = i0; i < i1; ++i) {
      const float4 c = srcc[i];
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const unsigned bx = floor_bits(fmaf(ty[p][0], inv, c.x));
        const unsigned by = floor_bits(fmaf(ty[p][1], inv, c.y));
        const unsigned bz = floor_bits(fmaf(ty[p][2], inv, c.z));
        if (bx < SX && by < Ey && bz < Ez) {
          const unsigned bin = bx * d.hs[0] + by * d.hs[1] + bz;
          if (U16)
            atomicAdd(&hist[bin >> 1], 1u << ((bin & 1u) << 4));
          else
            atomicAdd(&hist[bin * bstride + boff], 1u);
        }
      }
    }
  }
}

// SPARSE: 0 dense; 1 this instance also carries the culled path, 2 the paired
// culled path (for problems with d.sparse set to that mode); the dense
// instance leaves them out so it keeps its registers.
template <int P, int SPARSE, bool PADDED>
__global__ void __launch_bounds__(kPassThreads, 1) vote_kernel(PassLaunch L) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ PassDesc sd;
  __shared__ unsigned long long red64[32];
  __shared__ unsigned red32[32];
  __shared__ int s_item, s_prob, s_vote_item;
  __shared__ uint32_t s_sink[32];  // increments of out-of-box pairs (never read)
  __shared__ __align__(16) float s_thr[SPARSE ? 32 : 1][8 * 8];

  uint32_t* hist = reinterpret_cast<uint32_t*>(smem);
  const uint32_t hist_base = (uint32_t)__cvta_generic_to_shared(hist);
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
    const int tr = d.tile_rot > 0 ? d.tile_rot : L.tile_rot;
    const int r0 = (item - L.tile_prefix[p]) * tr;
    const int r1 = min(r0 + tr, d.n_rot);

    for (int r = r0; r < r1; ++r) {
      float R[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) R[k] = __ldg(d.rot + 9 * (size_t)r + k);
      const unsigned Ey = (unsigned)d.E[1], Ez = (unsigned)d.E[2];
      unsigned long long best = 0ull;  // (count << 32) | ~global_bin, max wins
      unsigned long long vtotal = 0ull;  // this warp's share of the rotation's votes

      for (int s = 0; s < d.n_slabs; ++s) {
        const int x0 = s * d.slab_x;
        const unsigned SX = (unsigned)min(d.slab_x, d.E[0] - x0);
        const bool centred = (SX & 1u) && (Ey & 1u) && (Ez & 1u);
        // staged offsets: centred path c = -(lo + off) - (S - 1)/2 - u/delta,
        // generic path c = 1/2 - (lo + off) - u/delta
        float off0, off1, off2;
        if (centred) {
          off0 = -(float)(d.lo[0] + x0) - (float)((SX - 1) / 2);
          off1 = -(float)d.lo[1] - (float)((Ey - 1) / 2);
          off2 = -(float)d.lo[2] - (float)((Ez - 1) / 2);
        } else {
          off0 = 0.5f - (float)(d.lo[0] + x0);
          off1 = 0.5f - (float)d.lo[1];
          off2 = 0.5f - (float)d.lo[2];
        }
        // the packed path stages 32 bytes per source; the sources are split
        // into equal chunks that fit the staging region
        const bool packed = P >= 2 && centred && !(SPARSE == 1 && d.sparse) && !d.hist_lanes;
        // (the paired culled instances stage tiles of 8 sources)
        const int chunk = max(1, d.chunk[packed ? (SPARSE == 2 ? 2 : 1) : 0]);  // >= 1 whatever the descriptor holds
        for (int c0 = 0; c0 < d.N; c0 += chunk) {
          const int c1 = min(c0 + chunk, d.N);
          __syncthreads();  // previous chunk's readers are done
          if (tid == 0) s_vote_item = 0;
          for (int i = c0 + tid; i < c1; i += kPassThreads) {
            const size_t si = (SPARSE && d.Xperm) ? (size_t)__ldg(d.Xperm + i) : (size_t)i;
            const float x = __ldg(d.X + 3 * si), y = __ldg(d.X + 3 * si + 1), z = __ldg(d.X + 3 * si + 2);
            const float ux = fmaf(R[0], x, fmaf(R[1], y, R[2] * z));
            const float uy = fmaf(R[3], x, fmaf(R[4], y, R[5] * z));
            const float uz = fmaf(R[6], x, fmaf(R[7], y, R[8] * z));
            const float cx = fmaf(-ux, d.inv_delta, off0), cy = fmaf(-uy, d.inv_delta, off1),
                        cz = fmaf(-uz, d.inv_delta, off2);
            if (SPARSE == 2) {
              float* t = reinterpret_cast<float*>(srcc) + ((i - c0) / kTileSources) * (kTileBytes / 4) +
                         2 * ((i - c0) % kTileSources);
              *reinterpret_cast<float2*>(t) = make_float2(cx, cx);
              *reinterpret_cast<float2*>(t + 16) = make_float2(cy, cy);
              *reinterpret_cast<float2*>(t + 32) = make_float2(cz, cz);
            } else if (packed) {
              srcc[2 * (i - c0)] = make_float4(cx, cx, cy, cy);
              srcc[2 * (i - c0) + 1] = make_float4(cz, cz, 0.f, 0.f);
            } else {
              srcc[i - c0] = make_float4(cx, cy, cz, 0.f);
            }
          }
          __syncthreads();
          // culled launches: the bounds of every block of 32 staged offsets,
          // so a block whose bounds miss an item's groups is skipped whole
          const float* blkp = nullptr;
          if (SPARSE && d.sparse && L.blk_bytes) {
            float* blk = reinterpret_cast<float*>(smem + L.hist_bytes + L.src_bytes);
            const int n = c1 - c0, nb = (n + 31) >> 5;
            for (int b = warp; b < nb; b += kPassThreads / 32) {
              const int i = b * 32 + lane;
              float lx = INFINITY, ly = INFINITY, lz = INFINITY, hx = -INFINITY, hy = -INFINITY, hz = -INFINITY;
              if (i < n) {
                if (SPARSE == 2) {
                  const float* t = reinterpret_cast<const float*>(srcc) + (i / kTileSources) * (kTileBytes / 4) +
                                   2 * (i % kTileSources);
                  lx = hx = t[0];
                  ly = hy = t[16];
                  lz = hz = t[32];
                } else if (packed) {
                  const float4 a = srcc[2 * i];
                  lx = hx = a.x;
                  ly = hy = a.z;
                  lz = hz = srcc[2 * i + 1].x;
                } else {
                  const float4 a = srcc[i];
                  lx = hx = a.x;
                  ly = hy = a.y;
                  lz = hz = a.z;
                }
              }
#pragma unroll
              for (int o = 16; o > 0; o >>= 1) {
                lx = fminf(lx, __shfl_xor_sync(0xffffffffu, lx, o));
                ly = fminf(ly, __shfl_xor_sync(0xffffffffu, ly, o));
                lz = fminf(lz, __shfl_xor_sync(0xffffffffu, lz, o));
                hx = fmaxf(hx, __shfl_xor_sync(0xffffffffu, hx, o));
                hy = fmaxf(hy, __shfl_xor_sync(0xffffffffu, hy, o));
                hz = fmaxf(hz, __shfl_xor_sync(0xffffffffu, hz, o));
              }
              if (lane == 0) {
                *reinterpret_cast<float4*>(blk + 8 * b) = make_float4(lx, hx, ly, hy);
                *reinterpret_cast<float2*>(blk + 8 * b + 4) = make_float2(lz, hz);
              }
            }
            __syncthreads();
            blkp = blk;
          }
          if (SPARSE == 2) {  // launches of this instance hold paired culled problems only (odd layouts)
            constexpr int PS = P >= 4 ? 4 : 2;  // paired instances are built for 2 and 4
            float* thr = s_thr[SPARSE ? warp : 0];
            const uint32_t sink = (uint32_t)__cvta_generic_to_shared(s_sink);
            const bool cube = SX == (unsigned)d.E[1] && d.E[1] == d.E[2];
            uint32_t* lst = reinterpret_cast<uint32_t*>(smem + L.hist_bytes + L.src_bytes + L.blk_bytes) +
                            warp * 3 * kPairedListCap;
            const float* srct = reinterpret_cast<const float*>(srcc);
            // items of a few sources each (below the 256 where block bounds
            // pay) vote each block's kept sources directly: gathering them in
            // lists and voting at the end of the item costs more than it saves
            // there (ModelNet-shaped +-0.2 box: 31%)
            const bool direct = (c1 - c0 + d.n_sgroups - 1) / d.n_sgroups < 256;
#define DSES_PAIRED(U, C, D)                                                                                   \
  vote_centred_paired<PS, U, C, D>(d, srct, c1 - c0, SX, hist_base, &s_vote_item, lane, thr, sink, blkp, lst)
            if (d.hist_u16 && cube)
              direct ? DSES_PAIRED(true, true, true) : DSES_PAIRED(true, true, false);
            else if (d.hist_u16)
              direct ? DSES_PAIRED(true, false, true) : DSES_PAIRED(true, false, false);
            else if (cube)
              direct ? DSES_PAIRED(false, true, true) : DSES_PAIRED(false, true, false);
            else
              direct ? DSES_PAIRED(false, false, true) : DSES_PAIRED(false, false, false);
#undef DSES_PAIRED
          } else if (SPARSE == 1) {  // ... and of this one 32-point culled problems only
            const bool cube = SX == (unsigned)d.E[1] && d.E[1] == d.E[2];
            float* thr = s_thr[SPARSE ? warp : 0];
            const uint32_t sink = (uint32_t)__cvta_generic_to_shared(s_sink);
            if (d.hist_u16 && cube)
              vote_centred_sparse<P, true, true>(d, srcc, c1 - c0, SX, hist_base, &s_vote_item, lane, thr, sink,
                                                     blkp);
            else if (d.hist_u16)
              vote_centred_sparse<P, true, false>(d, srcc, c1 - c0, SX, hist_base, &s_vote_item, lane, thr, sink,
                                                     blkp);
            else if (cube)
              vote_centred_sparse<P, false, true>(d, srcc, c1 - c0, SX, hist_base, &s_vote_item, lane, thr, sink,
                                                     blkp);
            else
              vote_centred_sparse<P, false, false>(d, srcc, c1 - c0, SX, hist_base, &s_vote_item, lane, thr, sink,
                                                     blkp);
          } else if (centred) {
            constexpr int PP = P >= 2 ? P : 2;  // the P = 1 instance never takes the packed path
            if (packed) {
              if (d.hist_u16)
                vote_centred_x2<PP, true, SPARSE == 0>(d, srcc, c1 - c0, SX, hist_base, &s_vote_item, lane,
                                              (uint32_t)__cvta_generic_to_shared(s_sink));
              else
                vote_centred_x2<PP, false, SPARSE == 0>(d, srcc, c1 - c0, SX, hist_base, &s_vote_item, lane,
                                               (uint32_t)__cvta_generic_to_shared(s_sink));
            } else if (d.hist_u16) {
              vote_centred<P, true>(d, srcc, c1 - c0, SX, hist_base, &s_vote_item, lane,
                                    (uint32_t)__cvta_generic_to_shared(s_sink));
            } else {
              vote_centred<P, false>(d, srcc, c1 - c0, SX, hist_base, &s_vote_item, lane,
                                     (uint32_t)__cvta_generic_to_shared(s_sink));
            }
          } else {
            if (d.hist_u16)
              vote_generic<P, true>(d, srcc, c1 - c0, SX, hist, &s_vote_item, lane);
            else
              vote_generic<P, false>(d, srcc, c1 - c0, SX, hist, &s_vote_item, lane);
          }
        }
        __syncthreads();
        // mode of this slab: scan and clear; each thread walks increasing bins
        const unsigned nbins = SX * d.hs[0];  // the slab's bins, stride padding included (never voted)
        unsigned bc = 0, bb = 0, vsum = 0;
        // (only PADDED instances carry the padded scan: the others keep the
        // hot loop's code generation of a kernel without it)
        const bool padded = PADDED && (d.Ev[0] != d.E[0] || d.Ev[1] != d.E[1] || d.Ev[2] != d.E[2]);
        if (padded) {
          // layout padded to odd extents: read the lattice box's bins only, a
          // warp per (x, y) row of the slab (each thread's bins increase),
          // then clear the whole slab
          const unsigned Eyv = (unsigned)d.Ev[1], Ezv = (unsigned)d.Ev[2];
          const unsigned rows = (unsigned)max(0, min((int)SX, d.Ev[0] - x0)) * Eyv;
          for (unsigned row = warp; row < rows; row += kPassThreads / 32) {
            const unsigned x = row / Eyv;
            const unsigned base = x * d.hs[0] + (row - x * Eyv) * d.hs[1];
            if (d.hist_lanes) {
              for (unsigned z = 0; z < Ezv; ++z) {
                const unsigned c = warp_sum_u32(hist[(base + z) * 32u + lane]);
                if (lane == 0) {
                  vsum += c;
                  if (c > bc) { bc = c; bb = base + z; }
                }
              }
            } else {
              for (unsigned z = lane; z < Ezv; z += 32) {
                const unsigned b = base + z;
                const unsigned c = d.hist_u16 ? (hist[b >> 1] >> ((b & 1u) << 4)) & 0xffffu : hist[b];
                vsum += c;
                if (c > bc) { bc = c; bb = b; }
              }
            }
          }
          __syncthreads();
          const unsigned words = d.hist_lanes ? nbins * 32u : (d.hist_u16 ? (nbins + 1) >> 1 : nbins);
          for (unsigned w = tid; w < words; w += kPassThreads) hist[w] = 0u;
        } else if (d.hist_lanes) {
          // a warp per bin: its 32 lane copies, summed across the warp (lane 0
          // keeps the warp's first maximum, increasing bins)
          for (unsigned b = warp; b < nbins; b += kPassThreads / 32) {
            const uint32_t v = hist[b * 32u + lane];
            hist[b * 32u + lane] = 0u;
            const unsigned c = warp_sum_u32(v);
            if (lane == 0) {
              vsum += c;
              if (c > bc) { bc = c; bb = b; }
            }
          }
        } else if (SPARSE != 0 && d.hist_u16) {
          // culled instances: one walk, each thread keeping its first maximum
          // (the two-walk form below measured 1% slower in their loops)
          const unsigned q4 = (((nbins + 1) >> 1) + 3) >> 2;
          uint4* h4 = reinterpret_cast<uint4*>(hist);
          for (unsigned w4 = tid; w4 < q4; w4 += kPassThreads) {
            const uint4 v4 = h4[w4];
            h4[w4] = make_uint4(0u, 0u, 0u, 0u);
            const uint32_t vv[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const unsigned a = vv[k] & 0xffffu, b = vv[k] >> 16;
              vsum += a + b;
              if (a > bc) { bc = a; bb = 8 * w4 + 2 * k; }
              if (b > bc) { bc = b; bb = 8 * w4 + 2 * k + 1; }
            }
          }
        } else if (SPARSE != 0) {
          const unsigned q4 = (nbins + 3) >> 2;
          uint4* h4 = reinterpret_cast<uint4*>(hist);
          for (unsigned w4 = tid; w4 < q4; w4 += kPassThreads) {
            const uint4 v4 = h4[w4];
            h4[w4] = make_uint4(0u, 0u, 0u, 0u);
            const uint32_t vv[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              vsum += vv[k];
              if (vv[k] > bc) { bc = vv[k]; bb = 4 * w4 + k; }
            }
          }
        } else if (d.hist_u16) {
          // 16-byte reads: the histogram's bytes are a multiple of 16 and the
          // words past this slab's bins are zero (never voted, or cleared).
          // First walk: the thread's packed maximum and vote sum; then the
          // block maximum M; second walk: clear, and the thread's first bin
          // holding M (only threads whose maximum is M read again)
          const unsigned q4 = (((nbins + 1) >> 1) + 3) >> 2;
          uint4* h4 = reinterpret_cast<uint4*>(hist);
          uint32_t m2 = 0u;
          for (unsigned w4 = tid; w4 < q4; w4 += kPassThreads) {
            const uint4 v4 = h4[w4];
            m2 = max_u16x2(m2, max_u16x2(max_u16x2(v4.x, v4.y), max_u16x2(v4.z, v4.w)));
            vsum = add_halves(v4.w, add_halves(v4.z, add_halves(v4.y, add_halves(v4.x, vsum))));
          }
          const unsigned tmax = max(m2 & 0xffffu, m2 >> 16);
          const unsigned M = block_max_u32(tmax, red32, lane, warp);
          bool look = tmax == M;
          for (unsigned w4 = tid; w4 < q4; w4 += kPassThreads) {
            if (look) {
              const uint4 v4 = h4[w4];
              const uint32_t vv[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
              for (int k = 3; k >= 0; --k) {  // the last assignment is the first bin
                if ((vv[k] >> 16) == M) { bb = 8 * w4 + 2 * k + 1; look = false; }
                if ((vv[k] & 0xffffu) == M) { bb = 8 * w4 + 2 * k; look = false; }
              }
            }
            h4[w4] = make_uint4(0u, 0u, 0u, 0u);
          }
          const bool found = tmax == M && !look;  // else: bin 0 at count 0
          bc = found ? M : 0u;
          bb = found ? bb : 0u;
        } else {
          const unsigned q4 = (nbins + 3) >> 2;
          uint4* h4 = reinterpret_cast<uint4*>(hist);
          unsigned tmax = 0u;
          for (unsigned w4 = tid; w4 < q4; w4 += kPassThreads) {
            const uint4 v4 = h4[w4];
            tmax = max(tmax, max(max(v4.x, v4.y), max(v4.z, v4.w)));
            vsum += v4.x + v4.y + v4.z + v4.w;
          }
          const unsigned M = block_max_u32(tmax, red32, lane, warp);
          bool look = tmax == M;
          for (unsigned w4 = tid; w4 < q4; w4 += kPassThreads) {
            if (look) {
              const uint4 v4 = h4[w4];
              const uint32_t vv[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
              for (int k = 3; k >= 0; --k)
                if (vv[k] == M) { bb = 4 * w4 + k; look = false; }
            }
            h4[w4] = make_uint4(0u, 0u, 0u, 0u);
          }
          const bool found = tmax == M && !look;
          bc = found ? M : 0u;
          bb = found ? bb : 0u;
        }
        vtotal += warp_sum_u32(vsum);
        const unsigned gbin = (unsigned)x0 * d.hs[0] + bb;
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
      }
      if (lane == 0 && d.votes_total && vtotal) atomicAdd(d.votes_total, vtotal);
      if (tid == 0) {
        const unsigned V = (unsigned)(best >> 32);
        const unsigned gbin = 0xffffffffu - (unsigned)(best & 0xffffffffull);
        const int kx = d.lo[0] + (int)(gbin / d.hs[0]);
        const int ky = d.lo[1] + (int)((gbin % d.hs[0]) / d.hs[1]);
        const int kz = d.lo[2] + (int)(gbin % d.hs[0] % d.hs[1]);
        d.kv[d.rot_base + (uint32_t)r - d.out_base] = make_int4(kx, ky, kz, (int)V);
        atomicMax(d.acc + 1, V);
      }
    }
  }
}

// One warp per rotation: inlier count (Eq. 3) at t* and, on the fused path,
// the robust cost from the distance grid and the argmin key.
constexpr int kCountPts = 2;  // source points per lane and iteration of count_kernel
constexpr int kCountThreads = 256;
// Per warp: queries the distance-grid bounds leave undecided, searched 32 at a
// time (one per lane) instead of by the few lanes that hold them. Up to 31
// wait between iterations and an iteration adds up to 32 kCountPts.
constexpr int kCountQueue = 32 + 32 * kCountPts;

__global__ void __launch_bounds__(kCountThreads) count_kernel(PassLaunch L) {
  __shared__ float4 s_queue[kCountThreads / 32][kCountQueue];
  const int lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  float4* queue = s_queue[threadIdx.x >> 5];
  const int warps = (gridDim.x * blockDim.x) >> 5;
  const int total = L.rot_prefix[L.n_probs];
  for (int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < total; g += warps) {
    int lo = 0, hi = L.n_probs - 1;  // last p with rot_prefix[p] <= g
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (__ldg(L.rot_prefix + mid) <= g) lo = mid; else hi = mid - 1;
    }
    const PassDesc& d = L.probs[lo];
    const int r = g - __ldg(L.rot_prefix + lo);
    const uint32_t gidx = d.rot_base + (uint32_t)r, o = gidx - d.out_base;
    float R[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) R[k] = __ldg(d.rot + 9 * (size_t)r + k);
    const int4 kv = d.kv[o];
    const float tx = (float)kv.x * d.delta, ty = (float)kv.y * d.delta, tz = (float)kv.z * d.delta;
    const bool grid_cost = d.fuse_score && d.metric != 0;
    int cnt = 0;
    float csum = 0.f;
    // kCountPts source points per lane and iteration: all their distance-grid
    // loads are in flight together (the kernel waits on L2 latency)
    const float e_far = d.eps + d.grid_err, e_near = d.eps - d.grid_err;
    int nq = 0;  // queued undecided queries (the same in every lane)
    for (int i0 = 0; i0 < d.N; i0 += 32 * kCountPts) {  // the same trip count in every lane
      const int i = i0 + lane;
      float qx[kCountPts], qy[kCountPts], qz[kCountPts], dg[kCountPts];
      bool valid[kCountPts], far[kCountPts], near[kCountPts];
#pragma unroll
      for (int k = 0; k < kCountPts; ++k) {
        valid[k] = i + 32 * k < d.N;
        const size_t ik = (size_t)(valid[k] ? i + 32 * k : i0);
        const float x = __ldg(d.X + 3 * ik), y = __ldg(d.X + 3 * ik + 1), z = __ldg(d.X + 3 * ik + 2);
        qx[k] = fmaf(R[0], x, fmaf(R[1], y, R[2] * z)) + tx;
        qy[k] = fmaf(R[3], x, fmaf(R[4], y, R[5] * z)) + ty;
        qz[k] = fmaf(R[6], x, fmaf(R[7], y, R[8] * z)) + tz;
      }
      // bounds on the exact nearest-target distance from the grid's corners
      // decide most queries; those within grid_err of epsilon take the exact
      // cell-list search
#pragma unroll
      for (int k = 0; k < kCountPts; ++k)
        dg[k] = grid_lookup_decide(d, qx[k], qy[k], qz[k], e_far, e_near, &far[k], &near[k]);
#pragma unroll
      for (int k = 0; k < kCountPts; ++k) {
        cnt += (valid[k] && !far[k] && near[k]) ? 1 : 0;
        const bool undecided = valid[k] && !far[k] && !near[k];
        const uint32_t m = __ballot_sync(0xffffffffu, undecided);
        if (undecided) queue[nq + __popc(m & lt)] = make_float4(qx[k], qy[k], qz[k], 0.f);
        nq += __popc(m);
        if (valid[k] && grid_cost) csum += robust_rho(d.metric, dg[k], d.eps, d.tau, d.huber_h, d.p_exp);
      }
      __syncwarp();
      while (nq >= 32) {  // the exact cell search, every lane on a queued query
        nq -= 32;
        const float4 q = queue[nq + lane];
        cnt += has_inlier(d, q.x, q.y, q.z) ? 1 : 0;
      }
      __syncwarp();  // queue reads done before the next pushes
    }
    if (lane < nq) {
      const float4 q = queue[lane];
      cnt += has_inlier(d, q.x, q.y, q.z) ? 1 : 0;
    }
    __syncwarp();  // before the next rotation's pushes
#pragma unroll
    for (int k = 16; k > 0; k >>= 1) {
      cnt += __shfl_xor_sync(0xffffffffu, cnt, k);
      csum += __shfl_xor_sync(0xffffffffu, csum, k);
    }
    if (lane == 0) {
      d.Mout[o] = (uint32_t)cnt;
      atomicMax(d.acc + 0, (uint32_t)cnt);
      if (d.fuse_score) {
        const float cost = d.metric == 0 ? (float)(d.N - cnt) : csum;
        d.cost[o] = cost;
        atomicMin(d.best, ((unsigned long long)__float_as_uint(cost) << 32) | (unsigned long long)gidx);
      }
    }
  }
}

template <int P, int SPARSE, bool PADDED>
cudaError_t launch_vote_p(const PassLaunch& L, int grid_ctas, cudaStream_t s) {
  const int smem = pass_smem_bytes(L.hist_bytes, L.src_bytes) + L.blk_bytes + L.list_bytes;
  // the opt-in is per device: a process may launch this instance on several GPUs
  static OptIn optin;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (optin.needed(dev, smem)) {
    e = cudaFuncSetAttribute(vote_kernel<P, SPARSE, PADDED>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    optin.done(dev, smem);
  }
  g_launches.fetch_add(1, std::memory_order_relaxed);
  vote_kernel<P, SPARSE, PADDED><<<grid_ctas, kPassThreads, smem, s>>>(L);
  return cudaGetLastError();
}

template <bool PADDED>
cudaError_t launch_vote_padded(const PassLaunch& L, int points_per_thread, int sparse, int grid_ctas,
                               cudaStream_t s) {
  if (sparse == 2) {
    switch (points_per_thread) {
      case 2: return launch_vote_p<2, 2, PADDED>(L, grid_ctas, s);
      case 4: return launch_vote_p<4, 2, PADDED>(L, grid_ctas, s);
      default: return cudaErrorInvalidValue;
    }
  }
  if (sparse == 1) {
    switch (points_per_thread) {
      case 1: return launch_vote_p<1, 1, PADDED>(L, grid_ctas, s);
      case 2: return launch_vote_p<2, 1, PADDED>(L, grid_ctas, s);
      case 4: return launch_vote_p<4, 1, PADDED>(L, grid_ctas, s);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (points_per_thread) {
    case 1: return launch_vote_p<1, 0, PADDED>(L, grid_ctas, s);
    case 2: return launch_vote_p<2, 0, PADDED>(L, grid_ctas, s);
    case 4: return launch_vote_p<4, 0, PADDED>(L, grid_ctas, s);
    case 8: return launch_vote_p<8, 0, PADDED>(L, grid_ctas, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

int pass_smem_bytes(int hist_bytes, int src_bytes) { return hist_bytes + src_bytes; }


cudaError_t launch_vote(const PassLaunch& L, int points_per_thread, int sparse, int grid_ctas, cudaStream_t s) {
  return L.padded ? launch_vote_padded<true>(L, points_per_thread, sparse, grid_ctas, s)
                  : launch_vote_padded<false>(L, points_per_thread, sparse, grid_ctas, s);
}

cudaError_t launch_count(const PassLaunch& L, int total_rot, cudaStream_t s) {
  const int blocks = (int)std::min<long long>(((long long)total_rot * 32 + 255) / 256, 148LL * 16);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  count_kernel<<<blocks > 0 ? blocks : 1, kCountThreads, 0, s>>>(L);
  return cudaGetLastError();
}

}  // namespace dses
