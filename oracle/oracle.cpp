// DSES oracle: a plain, slow, FP64, single-threaded CPU restatement of the
// Direct Semi-Exhaustive Search of "A Direct Semi-Exhaustive Search Method for
// Robust, Partial-to-Full Point Cloud Registration" (arXiv 2502.00115).
//
// TEST INFRASTRUCTURE ONLY. Nothing in the product path links, loads or calls
// this file; only the tests, the smoke check and the benchmark's CPU-baseline
// leg do. It shares no code, header, table or constant with the CUDA library.
//
// Every function states the passage it follows. Where the paper is silent or
// garbled the reading taken is stated next to the code:
//   * rotation grid: the dense SO(3) grid is a Hopf-fibration grid (HEALPix RING
//     pixel centres x 6n circle points); the local grid is the Euler box of
//     Algorithm 2's three rotation loops, R = R0 Rz(theta) Ry(phi) Rx(xi);
//   * ROUND(., delta_t) is k = floor(t / delta_t + 1/2) per axis on a lattice
//     anchored at the origin; the translation search range is the set of
//     lattice points k*delta_t inside [c - s, c + s];
//   * the MODE's tie-break is the smallest key in lexicographic (kx, ky, kz);
//   * M is the per-point inlier count of Eq. 3 at t* (Euclidean, strict
//     "< epsilon"); V is the peak frequency of the vote;
//   * the error sums over source points the distance to the nearest target
//     point (Eq. 1), passed through the chosen robust function rho;
//   * the q filter keeps rotations with 1000 M >= q_milli M*.
//
// Parity bookkeeping (not part of the method): a point pair is a "boundary
// pair" if one coordinate of (y_j - R x_i)/delta_t + 1/2 lies within
// band/delta_t of an integer, i.e. within `band` of a voxel face; a source
// point is a "boundary point" if its nearest-target distance lies within `band`
// of epsilon. These are the only places where FP32 and FP64 may decide
// differently.
//
// Parity status per function (what pins it, see tests/test_oracle_pins.py):
//   healpix / hopf grid        pinned: HEALPix base layout (N_side = 1), ring
//                              structure, fiber structure of the Hopf map;
//                              the phase of the fiber samples (the half step
//                              in psi_k = 2 pi (k + 1/2) / 6n) is a reading
//                              no external fact fixes: parity unpinned for
//                              that phase alone
//   euler box grid             pinned: closed form for single-axis boxes
//   lattice box                pinned: closed form
//   vote (mode)                pinned: brute force over every lattice cell
//                              using voxel membership; theorem special case
//   vote consistency check     pinned: planted perturbations
//   nn distance / inliers      pinned: scipy cKDTree
//   exact cost                 pinned: cKDTree distances
//   distance grid + lookup     pinned: cKDTree at centres, scipy
//                              RegularGridInterpolator between them
//   translation refinement     pinned: exact recovery on a noiseless subset,
//                              the least-squares optimality of the mean
//                              (scipy least squares), equivariance
//   exhaustive (Algorithm 1)   pinned: independent numpy brute force on tiny
//                              inputs, the theorem special case (zero error at
//                              the planted pose)
//   register (Algorithm 2)     pinned: theorem special case, exhaustive
//                              search (Algorithm 1) on tiny inputs
// tests/test_oracle_mutations.py plants plausible mistakes in copies of this
// file and checks that the pins catch every one.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <thread>
#include <vector>

namespace {

const double kPi = 3.14159265358979323846264338327950288;

struct V3 {
  double x, y, z;
};

inline V3 rot(const double* R, const double* p) {
  return {R[0] * p[0] + R[1] * p[1] + R[2] * p[2],
          R[3] * p[0] + R[4] * p[1] + R[5] * p[2],
          R[6] * p[0] + R[7] * p[1] + R[8] * p[2]};
}

void matmul3(const double* A, const double* B, double* C) {
  double T[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * k + j];
      T[3 * i + j] = s;
    }
  std::memcpy(C, T, sizeof(T));
}

void quat_to_matrix(double w, double x, double y, double z, double* R) {
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

}  // namespace

extern "C" {

// ---------------------------------------------------------------------------
// Problem parameters (the oracle's own layout).
struct orc_params {
  int metric;          // 0 inlier, 1 truncated L1, 2 truncated L2, 3 Huber, 4 L_p
  double epsilon;      // inlier threshold of Eq. 3
  double delta_t;      // translation discretisation of Algorithm 2
  double tau;          // truncation of the robust functions
  double huber_h;      // Huber knee
  double p;            // exponent of the L_p metric
  double t_center[3];  // translation search range: centre ...
  double t_half[3];    // ... and half-width per axis
  int q_milli;         // q of Algorithm 2 in thousandths (0 keeps every rotation)
  int top_k;           // >0: keep the top_k rotations by (M desc, index asc) instead
  int nn_mode;         // 0: distance-grid lookup, 1: exact brute-force nearest neighbour
  int grid_res;        // distance grid voxels per axis
  double grid_cap;     // distance grid truncation (>= tau)
  double band;         // boundary band for the parity bookkeeping
  int refine_top_k;    // >0: local Euler-box pass around this many best rotations
  int refine_K;        // Euler box half-size (2K+1 samples per angle)
  double refine_delta_r;  // Euler box angular step (radians)
};

struct orc_result {
  int status;          // 0 ok, -6 no candidate (no pair voted inside the box)
  int64_t rot_index;
  double R[9];
  double t[3];
  int64_t votes;       // V at the best rotation
  int64_t inliers;     // M at the best rotation
  double cost;
};

// ---------------------------------------------------------------------------
// Rotation grids (Algorithm 2's loop over orientations).

int64_t orc_hopf_count(int n) { return 72LL * n * n * n; }

// HEALPix RING-scheme pixel centres for N_side = n (Gorski et al. 2005): rings
// i = 1..4n-1 from north to south, pixels in increasing phi within a ring.
void orc_healpix_centres(int n, double* theta, double* phi) {
  int64_t idx = 0;
  const double nn = (double)n;
  for (int i = 1; i <= 4 * n - 1; ++i) {
    if (i < n) {  // north polar cap
      const double z = 1.0 - (double)i * i / (3.0 * nn * nn);
      for (int j = 1; j <= 4 * i; ++j) {
        theta[idx] = std::acos(z);
        phi[idx] = kPi / (2.0 * i) * (j - 0.5);
        ++idx;
      }
    } else if (i <= 3 * n) {  // equatorial belt
      const double z = 4.0 / 3.0 - 2.0 * i / (3.0 * nn);
      // rings with (i - n) even are shifted by half a pixel; phi starts at 0
      // on the others, as in the reference HEALPix library's pixel order
      const int s = (i - n + 1) % 2;
      for (int j = 1; j <= 4 * n; ++j) {
        theta[idx] = std::acos(z);
        phi[idx] = kPi / (2.0 * nn) * (j - 1 + s / 2.0);
        ++idx;
      }
    } else {  // south polar cap, mirror of the north cap
      const int ip = 4 * n - i;
      const double z = -(1.0 - (double)ip * ip / (3.0 * nn * nn));
      for (int j = 1; j <= 4 * ip; ++j) {
        theta[idx] = std::acos(z);
        phi[idx] = kPi / (2.0 * ip) * (j - 0.5);
        ++idx;
      }
    }
  }
}

// Dense SO(3) grid: Hopf coordinates (theta, phi) from the HEALPix centres and
// psi_k = 2 pi (k + 1/2) / (6n); unit quaternion
//   (cos(t/2) cos(p/2), cos(t/2) sin(p/2), sin(t/2) cos(f + p/2), sin(t/2) sin(f + p/2))
// with (t, f, p) = (theta, phi, psi); index r = pixel * 6n + k.
void orc_hopf_rotation(int n, int64_t r, double* R) {
  const int64_t npix = 12LL * n * n;
  const int64_t per = 6LL * n;
  const int64_t pix = r / per;
  const int64_t k = r % per;
  std::vector<double> th(npix), ph(npix);
  orc_healpix_centres(n, th.data(), ph.data());
  const double psi = 2.0 * kPi * (k + 0.5) / (double)per;
  const double t = th[pix], f = ph[pix];
  quat_to_matrix(std::cos(t / 2) * std::cos(psi / 2), std::cos(t / 2) * std::sin(psi / 2),
                 std::sin(t / 2) * std::cos(f + psi / 2), std::sin(t / 2) * std::sin(f + psi / 2), R);
}

void orc_hopf_grid(int n, double* R) {
  const int64_t npix = 12LL * n * n;
  const int64_t per = 6LL * n;
  std::vector<double> th(npix), ph(npix);
  orc_healpix_centres(n, th.data(), ph.data());
  for (int64_t pix = 0; pix < npix; ++pix)
    for (int64_t k = 0; k < per; ++k) {
      const double psi = 2.0 * kPi * (k + 0.5) / (double)per;
      const double t = th[pix], f = ph[pix];
      quat_to_matrix(std::cos(t / 2) * std::cos(psi / 2), std::cos(t / 2) * std::sin(psi / 2),
                     std::sin(t / 2) * std::cos(f + psi / 2), std::sin(t / 2) * std::sin(f + psi / 2),
                     R + 9 * (pix * per + k));
    }
}

// Euler box of Algorithm 2's three nested loops: theta, phi, xi each run over
// -K delta_r .. +K delta_r; R = R0 Rz(theta) Ry(phi) Rx(xi); theta outermost.
void orc_euler_box(const double* R0, int K, double dr, double* out) {
  const int w = 2 * K + 1;
  int64_t idx = 0;
  for (int a = 0; a < w; ++a)
    for (int b = 0; b < w; ++b)
      for (int c = 0; c < w; ++c) {
        const double th = (a - K) * dr, ph = (b - K) * dr, xi = (c - K) * dr;
        const double Rz[9] = {std::cos(th), -std::sin(th), 0, std::sin(th), std::cos(th), 0, 0, 0, 1};
        const double Ry[9] = {std::cos(ph), 0, std::sin(ph), 0, 1, 0, -std::sin(ph), 0, std::cos(ph)};
        const double Rx[9] = {1, 0, 0, 0, std::cos(xi), -std::sin(xi), 0, std::sin(xi), std::cos(xi)};
        double T[9];
        matmul3(R0, Rz, T);
        matmul3(T, Ry, T);
        matmul3(T, Rx, out + 9 * idx);
        ++idx;
      }
}

// ---------------------------------------------------------------------------
// Translation lattice (the discretisation delta_t of Algorithm 2).

// Lattice points k (k * delta inside [c - s, c + s]) per axis.
void orc_lattice_box(const double* c, const double* s, double delta, int* lo, int* hi) {
  for (int a = 0; a < 3; ++a) {
    lo[a] = (int)std::ceil((c[a] - s[a]) / delta);
    hi[a] = (int)std::floor((c[a] + s[a]) / delta);
  }
}

// ---------------------------------------------------------------------------
// Vote: t* = MODE{ROUND(y_j - R x_i, delta_t)} (Lemma 1, Eq. 5, discretised as
// in Section IV-B; Algorithm 2 line computing t*).

static inline void pair_coord(const double* X, const double* Y, int64_t i, int64_t j, const double* R,
                              double delta, double v[3]) {
  const V3 u = rot(R, X + 3 * i);
  v[0] = (Y[3 * j + 0] - u.x) / delta + 0.5;
  v[1] = (Y[3 * j + 1] - u.y) / delta + 0.5;
  v[2] = (Y[3 * j + 2] - u.z) / delta + 0.5;
}

static inline bool near_face(double v, double bandv) { return std::fabs(v - std::nearbyint(v)) <= bandv; }

void orc_vote(const double* X, int64_t N, const double* Y, int64_t M, const double* R, double delta,
              const int* lo, const int* hi, double band, int* kstar, int64_t* V, int64_t* n_boundary) {
  const int64_t Ey = hi[1] - lo[1] + 1, Ez = hi[2] - lo[2] + 1;
  const double bandv = band / delta;
  std::vector<int64_t> keys;
  keys.reserve((size_t)(N * M));
  int64_t nb = 0;
  for (int64_t i = 0; i < N; ++i)
    for (int64_t j = 0; j < M; ++j) {
      double v[3];
      pair_coord(X, Y, i, j, R, delta, v);
      if (near_face(v[0], bandv) || near_face(v[1], bandv) || near_face(v[2], bandv)) ++nb;
      const int64_t k0 = (int64_t)std::floor(v[0]), k1 = (int64_t)std::floor(v[1]),
                    k2 = (int64_t)std::floor(v[2]);
      if (k0 < lo[0] || k0 > hi[0] || k1 < lo[1] || k1 > hi[1] || k2 < lo[2] || k2 > hi[2]) continue;
      keys.push_back(((k0 - lo[0]) * Ey + (k1 - lo[1])) * Ez + (k2 - lo[2]));
    }
  std::sort(keys.begin(), keys.end());
  int64_t best_key = 0, best_len = 0;
  for (size_t a = 0; a < keys.size();) {
    size_t b = a;
    while (b < keys.size() && keys[b] == keys[a]) ++b;
    if ((int64_t)(b - a) > best_len) {  // strict: ties keep the smaller key
      best_len = (int64_t)(b - a);
      best_key = keys[a];
    }
    a = b;
  }
  kstar[0] = lo[0] + (int)(best_key / (Ey * Ez));
  kstar[1] = lo[1] + (int)((best_key / Ez) % Ey);
  kstar[2] = lo[2] + (int)(best_key % Ez);
  *V = best_len;
  if (n_boundary) *n_boundary = nb;
}

// Is a claimed (k, V) for one rotation what the vote yields when every
// boundary pair may land in any voxel within `band` of its FP64 position?
// Returns 2 if the claim equals the FP64 mode, 1 if it is consistent only
// through boundary pairs, 0 if inconsistent.
int orc_vote_consistent(const double* X, int64_t N, const double* Y, int64_t M, const double* R,
                        double delta, const int* lo, const int* hi, double band, const int* kc,
                        int64_t Vc) {
  int kx[3];
  int64_t V0 = 0;
  orc_vote(X, N, Y, M, R, delta, lo, hi, band, kx, &V0, nullptr);
  if (kx[0] == kc[0] && kx[1] == kc[1] && kx[2] == kc[2] && V0 == Vc) return 2;
  const int64_t Ex = hi[0] - lo[0] + 1, Ey = hi[1] - lo[1] + 1, Ez = hi[2] - lo[2] + 1;
  const double bandv = band / delta;
  std::vector<int64_t> certain, possible;
  for (int64_t i = 0; i < N; ++i)
    for (int64_t j = 0; j < M; ++j) {
      double v[3];
      pair_coord(X, Y, i, j, R, delta, v);
      int64_t opts[3][3];
      int nopt[3];
      bool boundary = false;
      for (int a = 0; a < 3; ++a) {
        const int64_t k = (int64_t)std::floor(v[a]);
        nopt[a] = 0;
        opts[a][nopt[a]++] = k;
        if (v[a] - (double)k <= bandv) { opts[a][nopt[a]++] = k - 1; boundary = true; }
        if ((double)(k + 1) - v[a] <= bandv) { opts[a][nopt[a]++] = k + 1; boundary = true; }
      }
      for (int p = 0; p < nopt[0]; ++p)
        for (int q = 0; q < nopt[1]; ++q)
          for (int r = 0; r < nopt[2]; ++r) {
            const int64_t a0 = opts[0][p], a1 = opts[1][q], a2 = opts[2][r];
            if (a0 < lo[0] || a0 > hi[0] || a1 < lo[1] || a1 > hi[1] || a2 < lo[2] || a2 > hi[2]) continue;
            const int64_t key = ((a0 - lo[0]) * Ey + (a1 - lo[1])) * Ez + (a2 - lo[2]);
            possible.push_back(key);
            if (!boundary) certain.push_back(key);
          }
    }
  if (kc[0] < lo[0] || kc[0] > hi[0] || kc[1] < lo[1] || kc[1] > hi[1] || kc[2] < lo[2] || kc[2] > hi[2])
    return 0;
  (void)Ex;
  const int64_t kkey = ((int64_t)(kc[0] - lo[0]) * Ey + (kc[1] - lo[1])) * Ez + (kc[2] - lo[2]);
  std::sort(certain.begin(), certain.end());
  std::sort(possible.begin(), possible.end());
  const int64_t cert_k = std::upper_bound(certain.begin(), certain.end(), kkey) -
                         std::lower_bound(certain.begin(), certain.end(), kkey);
  const int64_t poss_k = std::upper_bound(possible.begin(), possible.end(), kkey) -
                         std::lower_bound(possible.begin(), possible.end(), kkey);
  if (Vc == 0) return (certain.empty() && kkey == 0) ? 1 : 0;
  if (Vc < cert_k || Vc > poss_k) return 0;
  for (size_t a = 0; a < certain.size();) {
    size_t b = a;
    while (b < certain.size() && certain[b] == certain[a]) ++b;
    const int64_t cnt = (int64_t)(b - a);
    if (cnt > Vc) return 0;
    if (certain[a] < kkey && cnt >= Vc) return 0;
    a = b;
  }
  return 1;
}

// ---------------------------------------------------------------------------
// Nearest-neighbour distances and the inlier count of Eq. 3 at a fixed pose.

void orc_nn_dist(const double* X, int64_t N, const double* Y, int64_t M, const double* R, const double* t,
                 double* d) {
  for (int64_t i = 0; i < N; ++i) {
    const V3 u = rot(R, X + 3 * i);
    const double qx = u.x + t[0], qy = u.y + t[1], qz = u.z + t[2];
    double best = std::numeric_limits<double>::infinity();
    for (int64_t j = 0; j < M; ++j) {
      const double dx = Y[3 * j] - qx, dy = Y[3 * j + 1] - qy, dz = Y[3 * j + 2] - qz;
      const double s = dx * dx + dy * dy + dz * dz;
      if (s < best) best = s;
    }
    d[i] = std::sqrt(best);
  }
}

// M = #{i : min_j ||y_j - R x_i - t|| < epsilon}: the number of source points
// whose saturated L0 term of Eq. 3 is zero at tolerance epsilon.
void orc_inliers(const double* X, int64_t N, const double* Y, int64_t M, const double* R, const double* t,
                 double eps, double band, int64_t* count, int64_t* n_boundary) {
  std::vector<double> d((size_t)N);
  orc_nn_dist(X, N, Y, M, R, t, d.data());
  int64_t c = 0, nb = 0;
  for (int64_t i = 0; i < N; ++i) {
    if (d[i] < eps) ++c;
    if (std::fabs(d[i] - eps) <= band) ++nb;
  }
  *count = c;
  if (n_boundary) *n_boundary = nb;
}

// ---------------------------------------------------------------------------
// Sub-voxel translation refinement (a step after Algorithm 2; the paper stops
// at the voxel centre t* = k* delta_t). With the correspondences fixed at the
// pose (R, t) -- each source point paired with its nearest target, kept when
// that distance is below epsilon as in Eq. 3 -- the translation minimising the
// summed squared residual is the mean of the inlier translations:
//   t' = (1 / |I|) sum_{i in I} (y_nn(i) - R x_i).
// With no inlier t' = t. Returns |I|. Bookkeeping: n_boundary counts points
// whose nearest distance lies within band of epsilon, n_tie inlier candidates
// (distance below epsilon + band) whose second-nearest target is within band
// of the nearest; only there may an FP32 implementation pick differently.
int64_t orc_refine_translation(const double* X, int64_t N, const double* Y, int64_t M, const double* R,
                               const double* t, double eps, double band, double* t_out, int64_t* n_boundary,
                               int64_t* n_tie) {
  double sx = 0.0, sy = 0.0, sz = 0.0;
  int64_t n_in = 0, nb = 0, nt = 0;
  for (int64_t i = 0; i < N; ++i) {
    const V3 u = rot(R, X + 3 * i);
    const double qx = u.x + t[0], qy = u.y + t[1], qz = u.z + t[2];
    double d1 = std::numeric_limits<double>::infinity(), d2 = d1;
    int64_t j1 = -1;
    for (int64_t j = 0; j < M; ++j) {
      const double dx = Y[3 * j] - qx, dy = Y[3 * j + 1] - qy, dz = Y[3 * j + 2] - qz;
      const double dd = std::sqrt(dx * dx + dy * dy + dz * dz);
      if (dd < d1) {
        d2 = d1;
        d1 = dd;
        j1 = j;
      } else if (dd < d2) {
        d2 = dd;
      }
    }
    if (std::fabs(d1 - eps) <= band) ++nb;
    if (d1 < eps + band && d2 - d1 <= band) ++nt;
    if (d1 < eps) {
      sx += Y[3 * j1] - u.x;
      sy += Y[3 * j1 + 1] - u.y;
      sz += Y[3 * j1 + 2] - u.z;
      ++n_in;
    }
  }
  if (n_in > 0) {
    t_out[0] = sx / (double)n_in;
    t_out[1] = sy / (double)n_in;
    t_out[2] = sz / (double)n_in;
  } else {
    t_out[0] = t[0];
    t_out[1] = t[1];
    t_out[2] = t[2];
  }
  if (n_boundary) *n_boundary = nb;
  if (n_tie) *n_tie = nt;
  return n_in;
}

// ---------------------------------------------------------------------------
// Robust per-point error (the ERROR of Algorithm 2, the norm p of Eq. 1).

double orc_rho(const orc_params* P, double d) {
  switch (P->metric) {
    case 0:  // saturated L0 at tolerance epsilon (Eq. 3)
      return d < P->epsilon ? 0.0 : 1.0;
    case 1:  // truncated L1
      return std::min(d, P->tau);
    case 2: {  // truncated L2
      const double e = std::min(d, P->tau);
      return e * e;
    }
    case 3: {  // Huber on the truncated distance
      const double e = std::min(d, P->tau);
      return e <= P->huber_h ? 0.5 * e * e : P->huber_h * (e - 0.5 * P->huber_h);
    }
    default:  // L_p, p in (0, 1]
      return std::pow(d, P->p);
  }
}

// Error of Eq. 1 / Eq. 2 at one pose with exact (brute-force) nearest neighbours:
// sum over source points of rho(min_j ||y_j - R x_i - t||).
double orc_cost_exact(const double* X, int64_t N, const double* Y, int64_t M, const double* R, const double* t,
                      const orc_params* P) {
  std::vector<double> d((size_t)N);
  orc_nn_dist(X, N, Y, M, R, t, d.data());
  double s = 0.0;
  for (int64_t i = 0; i < N; ++i) s += orc_rho(P, d[i]);
  return s;
}

// ---------------------------------------------------------------------------
// Truncated distance grid of the target (a precomputed field standing in for
// the brute-force nearest neighbour of Algorithm 2's error loop).
// Geometry per axis: h = (extent + 2 cap) / (G - 2), lo = min - cap - h, so that
// the outermost voxel centres lie at least cap from every target point.
// D[(a G + b) G + c] = min(cap, min_j ||centre(a, b, c) - y_j||), centre =
// lo + (index + 1/2) h.

void orc_dist_grid_geometry(const double* Y, int64_t M, int G, double cap, double* lo, double* h) {
  for (int a = 0; a < 3; ++a) {
    double mn = std::numeric_limits<double>::infinity(), mx = -mn;
    for (int64_t j = 0; j < M; ++j) {
      mn = std::min(mn, Y[3 * j + a]);
      mx = std::max(mx, Y[3 * j + a]);
    }
    h[a] = (mx - mn + 2.0 * cap) / (double)(G - 2);
    lo[a] = mn - cap - h[a];
  }
}

static void dist_grid_planes(const double* Y, int64_t M, int G, double cap, const double* lo, const double* h,
                             double* D, int a0, int a1) {
  for (int a = a0; a < a1; ++a)
    for (int b = 0; b < G; ++b)
      for (int c = 0; c < G; ++c) {
        const double px = lo[0] + (a + 0.5) * h[0], py = lo[1] + (b + 0.5) * h[1], pz = lo[2] + (c + 0.5) * h[2];
        double best = std::numeric_limits<double>::infinity();
        for (int64_t j = 0; j < M; ++j) {
          const double dx = Y[3 * j] - px, dy = Y[3 * j + 1] - py, dz = Y[3 * j + 2] - pz;
          best = std::min(best, dx * dx + dy * dy + dz * dz);
        }
        D[((int64_t)a * G + b) * G + c] = std::min(cap, std::sqrt(best));
      }
}

void orc_dist_grid(const double* Y, int64_t M, int G, double cap, double* D) {
  double lo[3], h[3];
  orc_dist_grid_geometry(Y, M, G, cap, lo, h);
  dist_grid_planes(Y, M, G, cap, lo, h, D, 0, G);
}

// The same grid with its x-planes split over host threads (every voxel is
// computed as above, by one thread), for targets whose brute-force grid takes
// minutes on one core.
void orc_dist_grid_threads(const double* Y, int64_t M, int G, double cap, double* D, int threads) {
  double lo[3], h[3];
  orc_dist_grid_geometry(Y, M, G, cap, lo, h);
  const int T = std::max(1, std::min(threads, G));
  std::vector<std::thread> pool;
  for (int w = 0; w < T; ++w)
    pool.emplace_back([=]() { dist_grid_planes(Y, M, G, cap, lo, h, D, G * w / T, G * (w + 1) / T); });
  for (auto& th : pool) th.join();
}

// Trilinear interpolation between voxel centres, clamped at the outermost
// centres; points outside [lo, lo + G h] read the cap.
double orc_grid_lookup(const double* D, int G, const double* lo, const double* h, double cap, const double* p) {
  double f[3];
  int64_t i0[3];
  for (int a = 0; a < 3; ++a) {
    if (p[a] < lo[a] || p[a] > lo[a] + G * h[a]) return cap;
    double g = (p[a] - lo[a]) / h[a] - 0.5;
    g = std::min(std::max(g, 0.0), (double)(G - 1));
    int64_t i = (int64_t)std::floor(g);
    if (i > G - 2) i = G - 2;
    i0[a] = i;
    f[a] = g - (double)i;
  }
  double s = 0.0;
  for (int da = 0; da < 2; ++da)
    for (int db = 0; db < 2; ++db)
      for (int dc = 0; dc < 2; ++dc) {
        const double w = (da ? f[0] : 1 - f[0]) * (db ? f[1] : 1 - f[1]) * (dc ? f[2] : 1 - f[2]);
        s += w * D[((i0[0] + da) * G + (i0[1] + db)) * G + (i0[2] + dc)];
      }
  return s;
}

double orc_cost_grid(const double* X, int64_t N, const double* D, int G, const double* lo, const double* h,
                     double cap, const double* R, const double* t, const orc_params* P) {
  double s = 0.0;
  for (int64_t i = 0; i < N; ++i) {
    const V3 u = rot(R, X + 3 * i);
    const double q[3] = {u.x + t[0], u.y + t[1], u.z + t[2]};
    s += orc_rho(P, orc_grid_lookup(D, G, lo, h, cap, q));
  }
  return s;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Algorithm 2 end to end.

namespace {

struct RotOut {
  int k[3];
  int64_t V, M, nbp, nbm;
  double cost;
  bool cand;
};

static void eval_rotation(const double* X, int64_t N, const double* Y, int64_t M, const double* R,
                          const orc_params* P, const int* lo, const int* hi, RotOut* o) {
  orc_vote(X, N, Y, M, R, P->delta_t, lo, hi, P->band, o->k, &o->V, &o->nbp);
  const double t[3] = {o->k[0] * P->delta_t, o->k[1] * P->delta_t, o->k[2] * P->delta_t};
  orc_inliers(X, N, Y, M, R, t, P->epsilon, P->band, &o->M, &o->nbm);
  o->cost = std::numeric_limits<double>::quiet_NaN();
  o->cand = false;
}

struct Field {
  std::vector<double> D;
  double lo[3], h[3];
  int G;
  double cap;
};

static double score(const double* X, int64_t N, const double* Y, int64_t M, const double* R, const RotOut& o,
                    const orc_params* P, const Field* F) {
  if (P->metric == 0) return (double)(N - o.M);
  const double t[3] = {o.k[0] * P->delta_t, o.k[1] * P->delta_t, o.k[2] * P->delta_t};
  if (P->nn_mode == 1) return orc_cost_exact(X, N, Y, M, R, t, P);
  return orc_cost_grid(X, N, F->D.data(), F->G, F->lo, F->h, F->cap, R, t, P);
}

template <class Fn>
static void fan_out(int64_t n, int threads, Fn fn) {
  if (threads <= 1 || n < 2) {
    for (int64_t r = 0; r < n; ++r) fn(r);
    return;
  }
  std::vector<std::thread> pool;
  for (int w = 0; w < threads; ++w)
    pool.emplace_back([=]() {
      for (int64_t r = w; r < n; r += threads) fn(r);
    });
  for (auto& th : pool) th.join();
}

// Candidate selection of Algorithm 2: M* = max M, keep 1000 M >= q_milli M*
// (or the top_k by M descending, index ascending).
static void select_candidates(std::vector<RotOut>& o, size_t begin, size_t end, const orc_params* P) {
  int64_t Mstar = 0;
  for (size_t r = begin; r < end; ++r) Mstar = std::max(Mstar, o[r].M);
  if (P->top_k > 0) {
    std::vector<size_t> idx;
    for (size_t r = begin; r < end; ++r) idx.push_back(r);
    std::stable_sort(idx.begin(), idx.end(), [&](size_t a, size_t b) { return o[a].M > o[b].M; });
    for (size_t a = 0; a < idx.size() && (int64_t)a < P->top_k; ++a) o[idx[a]].cand = true;
  } else {
    for (size_t r = begin; r < end; ++r) o[r].cand = 1000LL * o[r].M >= (int64_t)P->q_milli * Mstar;
  }
}

}  // namespace

extern "C" {

static void build_field(const double* Y, int64_t M, int G, double cap, Field* F) {
  F->G = G;
  F->cap = cap;
  F->D.resize((size_t)G * G * G);
  orc_dist_grid(Y, M, G, cap, F->D.data());
  orc_dist_grid_geometry(Y, M, G, cap, F->lo, F->h);
}

// `prebuilt`: the target's distance field built beforehand (or NULL to build it here).
static int run_register(const double* X, int64_t N, const double* Y, int64_t M, const double* Rlist,
                        int64_t nR, const orc_params* P, int threads, int32_t* out_k, int64_t* out_V,
                        int64_t* out_M, double* out_cost, int64_t* out_nbp, int64_t* out_nbm,
                        orc_result* res, const Field* prebuilt = nullptr) {
  int lo[3], hi[3];
  orc_lattice_box(P->t_center, P->t_half, P->delta_t, lo, hi);
  Field Fown;
  if (!prebuilt && P->metric != 0 && P->nn_mode == 0) build_field(Y, M, P->grid_res, P->grid_cap, &Fown);
  const Field& F = prebuilt ? *prebuilt : Fown;
  const int B = P->refine_top_k > 0 ? (2 * P->refine_K + 1) * (2 * P->refine_K + 1) * (2 * P->refine_K + 1) : 0;
  const int64_t total = nR + (int64_t)P->refine_top_k * B;
  std::vector<RotOut> o((size_t)total);
  std::vector<double> Rall((size_t)total * 9);
  std::memcpy(Rall.data(), Rlist, sizeof(double) * 9 * (size_t)nR);

  // coarse pass: vote + count for every rotation, select, score candidates
  fan_out(nR, threads, [&](int64_t r) { eval_rotation(X, N, Y, M, &Rall[9 * r], P, lo, hi, &o[r]); });
  select_candidates(o, 0, (size_t)nR, P);
  fan_out(nR, threads, [&](int64_t r) {
    if (o[r].cand) o[r].cost = score(X, N, Y, M, &Rall[9 * r], o[r], P, &F);
  });
  auto better = [&](int64_t a, int64_t b) {  // lexicographic (cost, index)
    if (o[a].cost != o[b].cost) return o[a].cost < o[b].cost;
    return a < b;
  };
  // local Euler-box pass around the refine_top_k best coarse candidates
  if (P->refine_top_k > 0) {
    std::vector<int64_t> cands;
    for (int64_t r = 0; r < nR; ++r)
      if (o[r].cand) cands.push_back(r);
    std::sort(cands.begin(), cands.end(), better);
    const int64_t nc = std::min<int64_t>((int64_t)cands.size(), P->refine_top_k);
    for (int64_t c = 0; c < P->refine_top_k; ++c) {
      const int64_t centre = cands[(size_t)std::min(c, nc - 1)];
      orc_euler_box(&Rall[9 * centre], P->refine_K, P->refine_delta_r, &Rall[9 * (nR + c * B)]);
    }
    const int64_t nf = (int64_t)P->refine_top_k * B;
    fan_out(nf, threads, [&](int64_t f) { eval_rotation(X, N, Y, M, &Rall[9 * (nR + f)], P, lo, hi, &o[nR + f]); });
    select_candidates(o, (size_t)nR, (size_t)total, P);
    fan_out(nf, threads, [&](int64_t f) {
      if (o[nR + f].cand) o[nR + f].cost = score(X, N, Y, M, &Rall[9 * (nR + f)], o[nR + f], P, &F);
    });
  }
  int64_t best = -1, Vmax = 0;
  for (int64_t r = 0; r < total; ++r) {
    Vmax = std::max(Vmax, o[r].V);
    if (!o[r].cand) continue;
    if (best < 0 || better(r, best)) best = r;
  }
  for (int64_t r = 0; r < total; ++r) {
    if (out_k) { out_k[3 * r] = o[r].k[0]; out_k[3 * r + 1] = o[r].k[1]; out_k[3 * r + 2] = o[r].k[2]; }
    if (out_V) out_V[r] = o[r].V;
    if (out_M) out_M[r] = o[r].M;
    if (out_cost) out_cost[r] = o[r].cost;
    if (out_nbp) out_nbp[r] = o[r].nbp;
    if (out_nbm) out_nbm[r] = o[r].nbm;
  }
  res->status = Vmax == 0 ? -6 : 0;
  res->rot_index = best;
  std::memcpy(res->R, &Rall[9 * best], sizeof(res->R));
  for (int a = 0; a < 3; ++a) res->t[a] = o[best].k[a] * P->delta_t;
  res->votes = o[best].V;
  res->inliers = o[best].M;
  res->cost = o[best].cost;
  return res->status;
}

// Single-threaded correctness path.
int orc_register(const double* X, int64_t N, const double* Y, int64_t M, const double* Rlist, int64_t nR,
                 const orc_params* P, int32_t* out_k, int64_t* out_V, int64_t* out_M, double* out_cost,
                 int64_t* out_nbp, int64_t* out_nbm, orc_result* res) {
  return run_register(X, N, Y, M, Rlist, nR, P, 1, out_k, out_V, out_M, out_cost, out_nbp, out_nbm, res);
}

// The same computation fanned over rotations with std::thread; used only to
// time the CPU baseline on all host cores.
int orc_register_threads(const double* X, int64_t N, const double* Y, int64_t M, const double* Rlist,
                         int64_t nR, const orc_params* P, int threads, orc_result* res) {
  return run_register(X, N, Y, M, Rlist, nR, P, threads, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                      res);
}

// The same threaded computation with the per-rotation outputs of
// orc_register (each thread writes only the rotations it evaluates); used to
// write stored expected values at sizes the single-threaded path cannot
// finish in reasonable time.
int orc_register_threads_out(const double* X, int64_t N, const double* Y, int64_t M, const double* Rlist,
                             int64_t nR, const orc_params* P, int threads, int32_t* out_k, int64_t* out_V,
                             int64_t* out_M, double* out_cost, int64_t* out_nbp, int64_t* out_nbm,
                             orc_result* res) {
  return run_register(X, N, Y, M, Rlist, nR, P, threads, out_k, out_V, out_M, out_cost, out_nbp, out_nbm, res);
}

// Algorithm 1 (pure exhaustive search): every rotation of Rlist against every
// lattice translation k delta_t of the translation box, with the error
//   e(R, t) = sum over source points of rho(min_j ||y_j - R x_i - t||)
// (exact nearest neighbours; rho is non-decreasing, so the minimum of the
// per-pair errors is rho of the nearest distance). Entry r * n_t + t_idx of
// cost / count, t_idx = ((kx - lo_x) E_y + (ky - lo_y)) E_z + (kz - lo_z);
// count is the inlier count of Eq. 3 at that pose. Returns the index of the
// smallest cost (the first on ties), or -1 with no entry. near_tie receives
// how many entries lie within rel_tie (relative) of the smallest cost.
int64_t orc_exhaustive(const double* X, int64_t N, const double* Y, int64_t M, const double* Rlist, int64_t nR,
                       const orc_params* P, double* cost, int64_t* count, double rel_tie, int64_t* near_tie) {
  int lo[3], hi[3];
  orc_lattice_box(P->t_center, P->t_half, P->delta_t, lo, hi);
  const int64_t E[3] = {hi[0] - lo[0] + 1, hi[1] - lo[1] + 1, hi[2] - lo[2] + 1};
  if (E[0] < 1 || E[1] < 1 || E[2] < 1) return -1;
  const int64_t nt = E[0] * E[1] * E[2];
  std::vector<double> u(3 * (size_t)N);
  int64_t best = -1;
  for (int64_t r = 0; r < nR; ++r) {
    for (int64_t i = 0; i < N; ++i) {
      const V3 v = rot(Rlist + 9 * r, X + 3 * i);
      u[3 * i] = v.x;
      u[3 * i + 1] = v.y;
      u[3 * i + 2] = v.z;
    }
    for (int64_t a = 0; a < E[0]; ++a)
      for (int64_t b = 0; b < E[1]; ++b)
        for (int64_t c = 0; c < E[2]; ++c) {
          const double t[3] = {(double)(lo[0] + a) * P->delta_t, (double)(lo[1] + b) * P->delta_t,
                               (double)(lo[2] + c) * P->delta_t};
          double e = 0.0;
          int64_t n_in = 0;
          for (int64_t i = 0; i < N; ++i) {
            double m2 = std::numeric_limits<double>::infinity();
            for (int64_t j = 0; j < M; ++j) {
              const double dx = Y[3 * j] - u[3 * i] - t[0], dy = Y[3 * j + 1] - u[3 * i + 1] - t[1],
                           dz = Y[3 * j + 2] - u[3 * i + 2] - t[2];
              m2 = std::min(m2, dx * dx + dy * dy + dz * dz);
            }
            const double d = std::sqrt(m2);
            e += orc_rho(P, d);
            if (d < P->epsilon) ++n_in;
          }
          const int64_t idx = r * nt + (a * E[1] + b) * E[2] + c;
          cost[idx] = e;
          count[idx] = n_in;
          if (best < 0 || e < cost[best]) best = idx;
        }
  }
  if (near_tie) {
    int64_t n = 0;
    const double lim = cost[best] + rel_tie * std::max(1.0, std::fabs(cost[best]));
    for (int64_t k = 0; k < nR * nt; ++k) n += cost[k] <= lim ? 1 : 0;
    *near_tie = n;
  }
  return best;
}

// A target's distance field, built once and reused by orc_register_field_threads
// (the resident-target setting: the field is not part of a registration).
void* orc_field_create(const double* Y, int64_t M, int G, double cap) {
  Field* F = new Field();
  build_field(Y, M, G, cap, F);
  return F;
}

// The same field with the grid's x-planes split over host threads.
void* orc_field_create_threads(const double* Y, int64_t M, int G, double cap, int threads) {
  Field* F = new Field();
  F->G = G;
  F->cap = cap;
  F->D.resize((size_t)G * G * G);
  orc_dist_grid_threads(Y, M, G, cap, F->D.data(), threads);
  orc_dist_grid_geometry(Y, M, G, cap, F->lo, F->h);
  return F;
}

void orc_field_free(void* f) { delete static_cast<Field*>(f); }

int orc_register_field_threads(const double* X, int64_t N, const double* Y, int64_t M, const double* Rlist,
                               int64_t nR, const orc_params* P, const void* field, int threads, orc_result* res) {
  return run_register(X, N, Y, M, Rlist, nR, P, threads, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, res,
                      static_cast<const Field*>(field));
}

// Per-rotation evaluation at a given rotation (used by the sampled parity
// checks at sizes where the full pass is too slow on a CPU).
void orc_eval_rotation(const double* X, int64_t N, const double* Y, int64_t M, const double* R,
                       const orc_params* P, int* k, int64_t* V, int64_t* Mcount, int64_t* nbp, int64_t* nbm) {
  int lo[3], hi[3];
  orc_lattice_box(P->t_center, P->t_half, P->delta_t, lo, hi);
  RotOut o;
  eval_rotation(X, N, Y, M, R, P, lo, hi, &o);
  k[0] = o.k[0]; k[1] = o.k[1]; k[2] = o.k[2];
  *V = o.V;
  *Mcount = o.M;
  if (nbp) *nbp = o.nbp;
  if (nbm) *nbm = o.nbm;
}

}  // extern "C"
