"""Seeded synthetic point-cloud workloads.

This module only draws inputs: shapes, crops, rigid motions, noise and the
per-workload search parameters. It contains none of the registration
arithmetic, so both the CUDA path and the FP64 oracle can consume the same
arrays without sharing any of the method's code.

The shapes stand in for the ModelNet40 objects of the paper's Section V-A
(points on a closed surface, normalised into the unit sphere, 1,024 points a
side, Euler/uniform rotations, translations in [-0.5, 0.5], Gaussian noise
clipped at 0.05, a 70% half-space crop) and for the CAD gripper of Section
V-B (a ~0.3 m assembly of primitives seen from one viewpoint, with clutter).
No dataset item is reproduced: every object is a seeded random union of boxes
and ellipsoids.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# ---------------------------------------------------------------------------
# random rigid motions


def uniform_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform random rotation (Shoemake's subgroup algorithm, 1992)."""
    u1, u2, u3 = rng.random(3)
    a, b = math.sqrt(1.0 - u1), math.sqrt(u1)
    w = a * math.sin(2 * math.pi * u2)
    x = a * math.cos(2 * math.pi * u2)
    y = b * math.sin(2 * math.pi * u3)
    z = b * math.cos(2 * math.pi * u3)
    return np.array(
        [
            [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
            [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
            [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
        ]
    )


def euler_rotation(rng: np.random.Generator, max_deg: float) -> np.ndarray:
    """Rz(a) Ry(b) Rx(c) with the three angles uniform in [-max_deg, max_deg]
    (the ModelNet40 protocol of Section V-A draws Euler angles in [-45, 45] deg)."""
    a, b, c = np.radians(rng.uniform(-max_deg, max_deg, 3))
    Rz = np.array([[math.cos(a), -math.sin(a), 0], [math.sin(a), math.cos(a), 0], [0, 0, 1]])
    Ry = np.array([[math.cos(b), 0, math.sin(b)], [0, 1, 0], [-math.sin(b), 0, math.cos(b)]])
    Rx = np.array([[1, 0, 0], [0, math.cos(c), -math.sin(c)], [0, math.sin(c), math.cos(c)]])
    return Rz @ Ry @ Rx


def unit_vector(rng: np.random.Generator) -> np.ndarray:
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


# ---------------------------------------------------------------------------
# primitive surfaces


@dataclasses.dataclass
class Primitive:
    kind: str  # "box" or "ellipsoid"
    centre: np.ndarray  # (3,)
    axes: np.ndarray  # (3,3) orthonormal columns
    half: np.ndarray  # (3,) half extents / semi-axes

    def to_local(self, p: np.ndarray) -> np.ndarray:
        return (p - self.centre) @ self.axes

    def contains_strictly(self, p: np.ndarray, shrink: float = 1e-9) -> np.ndarray:
        q = self.to_local(p)
        if self.kind == "box":
            return np.all(np.abs(q) < self.half * (1 - shrink), axis=1)
        return np.sum((q / self.half) ** 2, axis=1) < 1 - shrink

    def area(self, rng: np.random.Generator) -> float:
        a, b, c = self.half
        if self.kind == "box":
            return 8.0 * (a * b + b * c + c * a)
        u = rng.normal(size=(20000, 3))
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        g = np.sqrt((b * c * u[:, 0]) ** 2 + (a * c * u[:, 1]) ** 2 + (a * b * u[:, 2]) ** 2)
        return 4.0 * math.pi * float(g.mean())

    def sample_surface(self, rng: np.random.Generator, n: int) -> np.ndarray:
        a, b, c = self.half
        if self.kind == "box":
            # faces +-x (area 4bc), +-y (4ac), +-z (4ab), chosen by area
            w = np.array([b * c, b * c, a * c, a * c, a * b, a * b])
            face = rng.choice(6, size=n, p=w / w.sum())
            q = (rng.random((n, 3)) * 2 - 1) * self.half
            axis = face // 2
            sign = np.where(face % 2 == 0, 1.0, -1.0)
            q[np.arange(n), axis] = sign * self.half[axis]
        else:
            # area-uniform on an ellipsoid: map sphere directions, accept with
            # probability proportional to the local area scale factor
            out = []
            gmax = max(b * c, a * c, a * b)
            while sum(len(o) for o in out) < n:
                u = rng.normal(size=(2 * n + 16, 3))
                u /= np.linalg.norm(u, axis=1, keepdims=True)
                g = np.sqrt((b * c * u[:, 0]) ** 2 + (a * c * u[:, 1]) ** 2 + (a * b * u[:, 2]) ** 2)
                keep = rng.random(len(u)) < g / gmax
                out.append(u[keep] * self.half)
            q = np.concatenate(out)[:n]
        return q @ self.axes.T + self.centre


def random_primitives(rng: np.random.Generator, count: int, kinds=("box", "ellipsoid")) -> list[Primitive]:
    prims = []
    for _ in range(count):
        kind = kinds[int(rng.integers(len(kinds)))]
        prims.append(
            Primitive(
                kind=kind,
                centre=rng.uniform(-0.5, 0.5, size=3),
                axes=uniform_rotation(rng),
                half=rng.uniform(0.2, 1.0, size=3),
            )
        )
    return prims


def sample_union_surface(rng: np.random.Generator, prims: list[Primitive], n: int) -> np.ndarray:
    """n points area-uniform on the outer surface of a union of primitives.

    Points of one primitive that fall strictly inside another are removed, so
    only the union's boundary is sampled.
    """
    areas = np.array([p.area(rng) for p in prims])
    total = areas.sum()
    pts = []
    need = n
    over = 3.0
    while True:
        counts = np.maximum(1, np.round(over * need * areas / total)).astype(int)
        cand = []
        for k, (p, m) in enumerate(zip(prims, counts)):
            s = p.sample_surface(rng, int(m))
            inside = np.zeros(len(s), dtype=bool)
            for l, q in enumerate(prims):
                if l != k:
                    inside |= q.contains_strictly(s)
            cand.append(s[~inside])
        pts.append(np.concatenate(cand))
        have = sum(len(x) for x in pts)
        if have >= n:
            break
        over *= 2.0
    allp = np.concatenate(pts)
    sel = rng.choice(len(allp), size=n, replace=False)
    return allp[sel]


def normalise_to_unit_sphere(points: np.ndarray, radius: float = 1.0) -> tuple[np.ndarray, np.ndarray, float]:
    """Centre on the bounding-box centre and scale so the farthest point has norm `radius`."""
    centre = 0.5 * (points.min(axis=0) + points.max(axis=0))
    p = points - centre
    scale = radius / np.linalg.norm(p, axis=1).max()
    return p * scale, centre, scale


def half_space_crop(rng: np.random.Generator, points: np.ndarray, keep_frac: float) -> np.ndarray:
    """Keep the keep_frac fraction of points farthest along a random direction in S^2."""
    d = unit_vector(rng)
    proj = points @ d
    k = int(round(keep_frac * len(points)))
    order = np.argsort(-proj, kind="stable")
    return points[np.sort(order[:k])]


def clipped_noise(rng: np.random.Generator, shape, sigma: float, clip: float | None) -> np.ndarray:
    e = rng.normal(scale=sigma, size=shape)
    if clip is not None:
        e = np.clip(e, -clip, clip)
    return e


# ---------------------------------------------------------------------------
# workloads


@dataclasses.dataclass
class Problem:
    """One registration problem: source X (partial) to target Y (full model)."""

    name: str
    X: np.ndarray  # (N,3) float32 source
    Y: np.ndarray  # (M,3) float32 target
    R_true: np.ndarray  # (3,3) float64, aligns X onto Y: y ~ R_true x + t_true
    t_true: np.ndarray  # (3,) float64
    epsilon: float
    delta_t: float
    t_center: tuple
    t_half: tuple
    hopf_n: int
    metric: str
    tau: float
    huber_h: float
    grid_res: int = 128
    grid_cap: float = 0.0  # distance-grid truncation (0 => 2*tau)
    q_milli: int = 0
    top_k: int = 0
    refine_top_k: int = 0
    refine_K: int = 0
    refine_delta_r: float = 0.0
    seed: int = 0

    @property
    def n_rotations(self) -> int:
        base = 72 * self.hopf_n**3
        return base + self.refine_top_k * (2 * self.refine_K + 1) ** 3


def _place_source(rng, shape_pts, t_range, max_euler_deg=None):
    """Apply a rotation (uniform, or Euler angles uniform in +-max_euler_deg)
    and a uniform translation to the observed points.

    Returns the moved points and the pose (R, t) with y = R x + t mapping the
    moved points back onto the model frame.
    """
    A = uniform_rotation(rng) if max_euler_deg is None else euler_rotation(rng, max_euler_deg)
    b = rng.uniform(-t_range, t_range, size=3)
    moved = shape_pts @ A.T + b
    return moved, A.T, -A.T @ b


def tiny_problem(seed: int = 0, noise: float = 0.005, hopf_n: int = 4) -> Problem:
    """256-point target, 128-point half-space crop of it as source (50%)."""
    rng = np.random.default_rng(seed)
    prims = random_primitives(rng, 3)
    Y, _, _ = normalise_to_unit_sphere(sample_union_surface(rng, prims, 256))
    Xs = half_space_crop(rng, Y, 0.5)
    X, Rt, tt = _place_source(rng, Xs, 0.5)
    X = X + clipped_noise(rng, X.shape, noise, None)
    return Problem(
        name="tiny", X=X.astype(np.float32), Y=Y.astype(np.float32), R_true=Rt, t_true=tt,
        epsilon=0.02, delta_t=0.02, t_center=(0.0, 0.0, 0.0), t_half=(0.9, 0.9, 0.9),
        hopf_n=hopf_n, metric="trunc_l1", tau=0.04, huber_h=0.02, seed=seed,
    )


def modelnet_like_problem(seed: int = 0, m: int = 1024, keep: float = 0.7, hopf_n: int = 16,
                          name: str = "modelnet_like", max_euler_deg: float | None = None,
                          rotated_frame: bool = False) -> Problem:
    """Section V-A protocol on a synthetic shape: independent 1,024-point samples of
    the same surface for source and target, noise N(0, 0.01) clipped at 0.05 on
    both clouds, a 70% half-space crop of the source, a random rotation (uniform,
    or Euler angles uniform in +-max_euler_deg as the paper draws them) and a
    translation in [-0.5, 0.5]^3. rotated_frame: both clouds are then turned by
    one more uniform rotation Q (the changed reference frame of Section V-A);
    the relative pose becomes (Q R Q^T, Q t)."""
    rng = np.random.default_rng(seed)
    prims = random_primitives(rng, 3)
    both = sample_union_surface(rng, prims, 2 * m)
    both, _, _ = normalise_to_unit_sphere(both)
    Y = both[:m] + clipped_noise(rng, (m, 3), 0.01, 0.05)
    Xs = both[m:] + clipped_noise(rng, (m, 3), 0.01, 0.05)
    Xs = half_space_crop(rng, Xs, keep)
    X, Rt, tt = _place_source(rng, Xs, 0.5, max_euler_deg)
    if rotated_frame:
        Q = uniform_rotation(rng)
        X, Y = X @ Q.T, Y @ Q.T
        Rt, tt = Q @ Rt @ Q.T, Q @ tt
    return Problem(
        name=name, X=X.astype(np.float32), Y=Y.astype(np.float32), R_true=Rt, t_true=tt,
        epsilon=0.04, delta_t=0.04, t_center=(0.0, 0.0, 0.0), t_half=(0.9, 0.9, 0.9),
        hopf_n=hopf_n, metric="trunc_l2", tau=0.05, huber_h=0.04, seed=seed,
    )


def batch_problems(seed: int = 0, count: int = 64, hopf_range=(8, 16), m_range=(512, 4096),
                   keep_range=(0.4, 0.8)) -> list[Problem]:
    """Uneven problems: target size uniform in m_range, source a keep-fraction crop
    of an independent sample, per-problem grid resolution uniform in hopf_range."""
    rng = np.random.default_rng(seed)
    out = []
    for p in range(count):
        m = int(rng.integers(m_range[0], m_range[1] + 1))
        keep = float(rng.uniform(*keep_range))
        n = int(rng.integers(hopf_range[0], hopf_range[1] + 1))
        sub = int(rng.integers(1 << 30))
        out.append(modelnet_like_problem(seed=sub, m=m, keep=keep, hopf_n=n, name=f"batch{p}"))
    return out


@dataclasses.dataclass
class ServingWorkload:
    targets: list  # list of (M,3) float32 target clouds
    requests: list  # list of (arrival_s, target_index, Problem)
    rate: float
    duration: float


def serving_workload(seed: int = 0, n_targets: int = 16, rate: float = 200.0, duration: float = 60.0,
                     hopf_n: int = 10, m_range=(1024, 8192), src_median: float = 600.0,
                     src_sigma_ln: float = 0.5, src_clip=(100, 4000)) -> ServingWorkload:
    """Poisson arrivals over resident targets; target sizes log-uniform in m_range;
    source sizes lognormal(median, sigma_ln) clipped to src_clip."""
    rng = np.random.default_rng(seed)
    targets, shapes = [], []
    for _ in range(n_targets):
        m = int(round(math.exp(rng.uniform(math.log(m_range[0]), math.log(m_range[1])))))
        prims = random_primitives(rng, 3)
        pts = sample_union_surface(rng, prims, m + src_clip[1])
        pts, _, _ = normalise_to_unit_sphere(pts)
        Y = (pts[:m] + clipped_noise(rng, (m, 3), 0.01, 0.05)).astype(np.float32)
        targets.append(Y)
        shapes.append(pts[m:])
    reqs = []
    t = 0.0
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t >= duration:
            break
        ti = int(rng.integers(n_targets))
        n = int(np.clip(round(src_median * math.exp(rng.normal(0.0, src_sigma_ln))), *src_clip))
        pool = shapes[ti]
        obs = pool[rng.choice(len(pool), size=min(len(pool), int(n / 0.7) + 1), replace=False)]
        obs = obs + clipped_noise(rng, obs.shape, 0.01, 0.05)
        obs = half_space_crop(rng, obs, 0.7)[:n]
        X, Rt, tt = _place_source(rng, obs, 0.5)
        prob = Problem(
            name=f"req{len(reqs)}", X=X.astype(np.float32), Y=targets[ti], R_true=Rt, t_true=tt,
            epsilon=0.04, delta_t=0.04, t_center=(0.0, 0.0, 0.0), t_half=(0.9, 0.9, 0.9),
            hopf_n=hopf_n, metric="trunc_l2", tau=0.05, huber_h=0.04, seed=seed,
        )
        reqs.append((t, ti, prob))
    return ServingWorkload(targets=targets, requests=reqs, rate=rate, duration=duration)


def _visible_surface(rng, surface, view_dist=1.0, image=256, keep_mm=0.002):
    """Points of a dense surface sample seen from a random viewpoint at view_dist:
    pinhole z-buffer of image x image pixels, keep points within keep_mm of the
    buffer depth at their pixel."""
    d = unit_vector(rng)
    eye = d * view_dist
    fwd = -d
    up0 = np.array([0.0, 0.0, 1.0]) if abs(fwd[2]) < 0.9 else np.array([1.0, 0.0, 0.0])
    right = np.cross(fwd, up0)
    right /= np.linalg.norm(right)
    up = np.cross(right, fwd)
    rel = surface - eye
    z = rel @ fwd
    u = (rel @ right) / z
    v = (rel @ up) / z
    half = max(np.abs(u).max(), np.abs(v).max()) * 1.02
    px = np.clip(((u / half + 1) * 0.5 * image).astype(int), 0, image - 1)
    py = np.clip(((v / half + 1) * 0.5 * image).astype(int), 0, image - 1)
    pix = py * image + px
    zbuf = np.full(image * image, np.inf)
    np.minimum.at(zbuf, pix, z)
    return surface[z <= zbuf[pix] + keep_mm]


def robot_like_problem(seed: int = 0, m: int = 20000, n_surface: int = 3500, n_clutter: int = 1500,
                       hopf_n: int = 32, refine_top_k: int = 32, refine_K: int = 3,
                       refine_delta_r_deg: float = 0.3125) -> Problem:
    """A ~0.3 m assembly of 8 primitives (the Section V-B gripper stand-in):
    20,000 model points; the source is the surface visible from one viewpoint at
    1 m (3,500 points, noise sigma 1 mm) plus 1,500 uniform clutter points in
    twice the bounding box (30%); uniform rotation, translation in +-3 cm."""
    rng = np.random.default_rng(seed)
    prims = random_primitives(rng, 8)
    dense = sample_union_surface(rng, prims, m + 200000)
    dense, _, _ = normalise_to_unit_sphere(dense)
    ext = (dense.max(axis=0) - dense.min(axis=0)).max()
    dense *= 0.3 / ext
    Y = dense[:m]
    vis = _visible_surface(rng, dense[m:], view_dist=1.0)
    vis = vis[rng.choice(len(vis), size=min(n_surface, len(vis)), replace=False)]
    vis = vis + clipped_noise(rng, vis.shape, 0.001, None)
    lo, hi = Y.min(axis=0), Y.max(axis=0)
    c, h = 0.5 * (lo + hi), (hi - lo)
    clutter = c + (rng.random((n_clutter, 3)) - 0.5) * 2.0 * h
    obs = np.concatenate([vis, clutter])
    obs = obs[rng.permutation(len(obs))]
    X, Rt, tt = _place_source(rng, obs, 0.03)
    return Problem(
        name="robot_like", X=X.astype(np.float32), Y=Y.astype(np.float32), R_true=Rt, t_true=tt,
        epsilon=0.003, delta_t=0.003, t_center=(0.0, 0.0, 0.0), t_half=(0.05, 0.05, 0.05),
        hopf_n=hopf_n, metric="huber", tau=0.010, huber_h=0.003, grid_cap=0.02,
        refine_top_k=refine_top_k, refine_K=refine_K,
        refine_delta_r=math.radians(refine_delta_r_deg), seed=seed,
    )


def dyadic_cloud(rng: np.random.Generator, n: int, scale_bits: int = 20, extent: float = 1.0,
                 min_sep_inf: float = 0.0) -> np.ndarray:
    """Points with coordinates on a 2^-scale_bits lattice (exact in FP32/FP64) in
    [-extent, extent]^3, optionally pairwise >= min_sep_inf apart in the inf-norm."""
    q = 2.0 ** (-scale_bits)
    out = []
    tries = 0
    while len(out) < n:
        tries += 1
        if tries > 200 * n + 1000:
            raise RuntimeError("could not place separated points")
        p = np.round(rng.uniform(-extent, extent, size=3) / q) * q
        if min_sep_inf > 0 and out:
            if np.min(np.max(np.abs(np.asarray(out) - p), axis=1)) < min_sep_inf:
                continue
        out.append(p)
    return np.asarray(out, dtype=np.float64)
