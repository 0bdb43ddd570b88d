"""Seeded synthetic inputs shaped like the registration workloads of
Yao et al., "Fast and Robust Non-Rigid Registration Using Accelerated
Majorization-Minimization" (Sec. 4: clean, noisy, partial and RGB-D pairs).

This module is shared by the FP64 oracle, the tests and the benchmark. It
holds only input generation (surfaces, a smooth ground-truth warp, noise,
outliers, crops, a synthetic depth grid) and none of the registration
method's arithmetic. Every array it returns is float32, the precision the
library's entry points take; the oracle promotes them exactly to float64.

Recipes (all seeded with numpy's PCG64 through ``default_rng``):

* bumpy sphere: ``s(n) = (1 + sum_k a_k exp(-|n - c_k|^2 / (2 w^2))) n`` with
  ``n`` uniform on the unit sphere, ``c_k`` uniform on the sphere and
  ``a_k = +-amp`` with random sign; normals from the analytic gradient;
* warp ``phi(x) = x + sum_{k<4} d_k exp(-|x - mu_k|^2 / (2 * 0.5^2))``,
  rescaled so that ``max |phi(x) - x|`` over the warped points equals a cap;
* dense noise: isotropic Gaussian, sigma = fraction x bbox diagonal;
* outliers: uniform in the bounding box, appended after the surface points;
* crop: a half-space with a random normal whose offset removes a fraction;
* depth grid: a 640x480 pinhole view (fx = fy = 525, cx = 319.5,
  cy = 239.5) of a height field ``z = 2 + h`` with 32 Gaussian bumps, with
  disc-shaped hole patches until a fraction of pixels is invalid.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Pair", "bumpy_sphere", "smooth_warp", "add_noise", "add_outliers",
    "crop_halfspace", "depth_scene", "sphere_pair", "tiny_pair", "island_pair",
    "workload", "WORKLOADS",
]


@dataclass
class Pair:
    """One registration problem: source/target points (+normals) and the
    ground-truth position of every source point on the target surface."""
    src: np.ndarray                      # [P,3] float32
    src_nrm: np.ndarray                  # [P,3] float32
    tgt: np.ndarray                      # [T,3] float32
    tgt_nrm: np.ndarray                  # [T,3] float32
    gt: np.ndarray                       # [P,3] float32, true match of src
    params: dict = field(default_factory=dict)
    name: str = ""
    faces: np.ndarray | None = None      # [F,3] int32 when the source is a mesh

    @property
    def P(self) -> int:
        return int(self.src.shape[0])

    @property
    def T(self) -> int:
        return int(self.tgt.shape[0])


def _unit_sphere(n: int, rng: np.random.Generator) -> np.ndarray:
    g = rng.standard_normal((n, 3))
    return g / np.linalg.norm(g, axis=1, keepdims=True)


def bumpy_sphere(n: int, n_bumps: int, amp: float, width: float,
                 rng: np.random.Generator, bumps=None):
    """Samples ``n`` points of a radially bumped unit sphere.

    Returns (xyz, normals, bumps) with bumps = (centres [K,3], amplitudes [K])
    so that a second, independent sampling of the same surface can be drawn.
    """
    if bumps is None:
        c = _unit_sphere(n_bumps, rng)
        a = amp * np.where(rng.random(n_bumps) < 0.5, -1.0, 1.0)
        bumps = (c, a)
    c, a = bumps
    nrm = _unit_sphere(n, rng)
    diff = nrm[:, None, :] - c[None, :, :]                  # [n,K,3]
    g = np.exp(-np.sum(diff * diff, axis=2) / (2.0 * width * width))
    r = 1.0 + g @ a                                         # radius
    # gradient of r(n) in R^3, projected on the tangent plane of the sphere
    grad = -np.einsum("nk,nkd->nd", g * a[None, :], diff) / (width * width)
    grad -= np.sum(grad * nrm, axis=1, keepdims=True) * nrm
    xyz = r[:, None] * nrm
    normal = r[:, None] * nrm - grad
    normal /= np.linalg.norm(normal, axis=1, keepdims=True)
    return xyz, normal, bumps


def smooth_warp(x: np.ndarray, cap: float, rng: np.random.Generator,
                lo=None, hi=None, n_rbf: int = 4, sigma: float = 0.5,
                return_field: bool = False):
    """Applies a smooth RBF displacement field whose largest displacement
    over ``x`` is exactly ``cap``. ``lo``/``hi`` bound the RBF centres
    (default: bbox of ``x``)."""
    lo = x.min(axis=0) if lo is None else lo
    hi = x.max(axis=0) if hi is None else hi
    mu = lo + (hi - lo) * rng.random((n_rbf, 3))
    d = _unit_sphere(n_rbf, rng)

    def field_at(p):
        diff = p[:, None, :] - mu[None, :, :]
        g = np.exp(-np.sum(diff * diff, axis=2) / (2.0 * sigma * sigma))
        return g @ d

    disp = field_at(x)
    scale = cap / max(float(np.linalg.norm(disp, axis=1).max()), 1e-300)
    out = x + scale * disp
    if return_field:
        return out, (lambda p: p + scale * field_at(p))
    return out


def add_noise(x: np.ndarray, frac_of_diag: float, diag: float,
              rng: np.random.Generator) -> np.ndarray:
    return x + rng.standard_normal(x.shape) * (frac_of_diag * diag)


def add_outliers(x: np.ndarray, nrm: np.ndarray, frac: float,
                 rng: np.random.Generator):
    """Appends ``round(frac * len(x))`` points uniform in the bbox of ``x``
    (normals random unit vectors)."""
    k = int(round(frac * x.shape[0]))
    lo, hi = x.min(axis=0), x.max(axis=0)
    o = lo + (hi - lo) * rng.random((k, 3))
    on = _unit_sphere(k, rng)
    return np.concatenate([x, o]), np.concatenate([nrm, on])


def crop_halfspace(x: np.ndarray, frac: float, rng: np.random.Generator):
    """Keeps the points on one side of a random plane chosen so that a
    fraction ``frac`` of them is removed. Returns the boolean keep mask."""
    if frac <= 0.0:
        return np.ones(x.shape[0], dtype=bool)
    n = _unit_sphere(1, rng)[0]
    s = x @ n
    thr = np.quantile(s, 1.0 - frac)
    return s < thr


def _bbox_diag(*arrs) -> float:
    a = np.concatenate(arrs)
    return float(np.linalg.norm(a.max(axis=0) - a.min(axis=0)))


def _f32(*arrs):
    return tuple(np.ascontiguousarray(a, dtype=np.float32) for a in arrs)


def icosphere(subdiv: int):
    """Unit icosphere: the icosahedron with every face split into four,
    ``subdiv`` times, vertices pushed onto the sphere. Returns (V [n,3]
    float64, F [m,3] int64); consistent outward orientation."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    V = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t),
         (0, -1, -t), (0, 1, -t), (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    V = [np.array(v, dtype=np.float64) / math.sqrt(1 + t * t) for v in V]
    F = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4),
         (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8),
         (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(subdiv):
        mid = {}

        def midpoint(a, b):
            k = (min(a, b), max(a, b))
            if k not in mid:
                m = V[a] + V[b]
                V.append(m / np.linalg.norm(m))
                mid[k] = len(V) - 1
            return mid[k]

        nf = []
        for a, b, c in F:
            ab, bc, ca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        F = nf
    return np.array(V), np.array(F, dtype=np.int64)


def bumpy_sphere_mesh(subdiv: int, n_bumps: int, amp: float, width: float,
                      rng: np.random.Generator, bumps=None):
    """The bumped sphere of ``bumpy_sphere`` as a triangle mesh: the
    icosphere's vertices moved radially. Returns (xyz, normals, faces,
    bumps)."""
    n, F = icosphere(subdiv)
    if bumps is None:
        c = _unit_sphere(n_bumps, rng)
        a = amp * np.where(rng.random(n_bumps) < 0.5, -1.0, 1.0)
        bumps = (c, a)
    c, a = bumps
    diff = n[:, None, :] - c[None, :, :]
    g = np.exp(-np.sum(diff * diff, axis=2) / (2.0 * width * width))
    r = 1.0 + g @ a
    grad = -np.einsum("nk,nkd->nd", g * a[None, :], diff) / (width * width)
    grad -= np.sum(grad * n, axis=1, keepdims=True) * n
    normal = r[:, None] * n - grad
    normal /= np.linalg.norm(normal, axis=1, keepdims=True)
    return r[:, None] * n, normal, F, bumps


def grid_mesh(nx: int, ny: int, h: float = 1.0, keep=None):
    """Flat triangulated grid of nx x ny vertices (spacing h, z = 0), each
    cell split along alternating diagonals; ``keep(i, j)`` selects cells (an
    L-shaped or holed domain). Returns (V [n,3] float64, F [m,3] int64,
    index dict (i, j) -> vertex); vertices of dropped cells stay unused."""
    V, idx = [], {}
    for j in range(ny):
        for i in range(nx):
            idx[(i, j)] = len(V)
            V.append((i * h, j * h, 0.0))
    F = []
    for j in range(ny - 1):
        for i in range(nx - 1):
            if keep is not None and not keep(i, j):
                continue
            a, b, c, d = idx[(i, j)], idx[(i + 1, j)], idx[(i + 1, j + 1)], idx[(i, j + 1)]
            F += [(a, b, c), (a, c, d)] if (i + j) % 2 == 0 else [(a, b, d), (b, c, d)]
    return np.array(V, dtype=np.float64), np.array(F, dtype=np.int64), idx


def cylinder_mesh(n: int, rings: int, radius: float, dz: float):
    """Open triangulated cylinder: ``rings`` rings of n vertices around the
    z axis, ring spacing dz. Vertex (ring j, k) has index j * n + k."""
    V = [(radius * math.cos(2 * math.pi * k / n), radius * math.sin(2 * math.pi * k / n), j * dz)
         for j in range(rings) for k in range(n)]
    F = []
    for j in range(rings - 1):
        for k in range(n):
            a, b = j * n + k, j * n + (k + 1) % n
            c, d = (j + 1) * n + (k + 1) % n, (j + 1) * n + k
            F += [(a, b, c), (a, c, d)]
    return np.array(V, dtype=np.float64), np.array(F, dtype=np.int64)


def cube_mesh(nd: int):
    """Surface of the unit cube [0, 1]^3, each face an nd x nd grid of
    squares split into two triangles. Returns (V, F)."""
    key, V, F = {}, [], []

    def vid(p):
        k = tuple(int(round(x * nd)) for x in p)
        if k not in key:
            key[k] = len(V)
            V.append(p)
        return key[k]

    for axis in range(3):
        for side in (0.0, 1.0):
            for a in range(nd):
                for b in range(nd):
                    def at(u, v):
                        p = [0.0, 0.0, 0.0]
                        p[axis], p[(axis + 1) % 3], p[(axis + 2) % 3] = side, u / nd, v / nd
                        return tuple(p)
                    q = [vid(at(a, b)), vid(at(a + 1, b)), vid(at(a + 1, b + 1)), vid(at(a, b + 1))]
                    F += [(q[0], q[1], q[2]), (q[0], q[2], q[3])]
    return np.array(V, dtype=np.float64), np.array(F, dtype=np.int64)


def crown_mesh(n: int, apex_angle_deg: float):
    """A fan of n triangles around an apex (vertex 0) with ring vertices
    1..n at distance 1 from it and apex angle ``apex_angle_deg`` per
    triangle, the ring zig-zagging in z so that the angles fit in 3-D (n
    even). With n * angle > 360 degrees the apex is a saddle vertex."""
    alpha = math.radians(apex_angle_deg)
    rho = math.cos(alpha / 2) / math.cos(math.pi / n)
    h = math.sqrt(max(1.0 - rho * rho, 0.0))
    V = [(0.0, 0.0, 0.0)] + [(rho * math.cos(2 * math.pi * i / n), rho * math.sin(2 * math.pi * i / n),
                              h if i % 2 else -h) for i in range(n)]
    F = [(0, 1 + i, 1 + (i + 1) % n) for i in range(n)]
    return np.array(V, dtype=np.float64), np.array(F, dtype=np.int64)


def mesh_pair(subdiv: int, T: int, n_bumps: int, amp: float, width: float, warp_cap: float,
              noise: float, outliers: float, crop: float, seed: int) -> Pair:
    """A triangle-mesh source (the bumped icosphere) and a target sampled
    independently from the same surface, warped, with noise, outliers and a
    crop as ``sphere_pair``; ``faces`` holds the source triangles."""
    rng = np.random.default_rng(seed)
    src, src_n, F, bumps = bumpy_sphere_mesh(subdiv, n_bumps, amp, width, rng)
    base, base_n, _ = bumpy_sphere(T, n_bumps, amp, width, rng, bumps)
    lo, hi = src.min(axis=0), src.max(axis=0)
    _, phi = smooth_warp(base, 1.0, rng, lo, hi, return_field=True)
    both = np.concatenate([src, base])
    disp = phi(both) - both
    s = warp_cap / float(np.linalg.norm(disp, axis=1).max())
    warp = lambda p: p + s * (phi(p) - p)
    tgt, tgt_n, gt = warp(base), base_n, warp(src)
    diag = _bbox_diag(src, tgt)
    keep = crop_halfspace(tgt, crop, rng)
    tgt, tgt_n = tgt[keep], tgt_n[keep]
    tgt = add_noise(tgt, noise, diag, rng) if noise > 0 else tgt
    if outliers > 0:
        tgt, tgt_n = add_outliers(tgt, tgt_n, outliers, rng)
    src, src_n, tgt, tgt_n, gt = _f32(src, src_n, tgt, tgt_n, gt)
    return Pair(src, src_n, tgt, tgt_n, gt, faces=F.astype(np.int32))


def sphere_pair(P: int, T: int | None, n_bumps: int, amp: float, width: float,
                warp_cap: float, noise: float, outliers: float, crop: float,
                seed: int, same_samples: bool) -> Pair:
    """Bumpy-sphere pair. With ``same_samples`` the target is the warped
    source itself (before noise/outliers/crop); otherwise the target is an
    independent sampling of the same surface of size ``T``."""
    rng = np.random.default_rng(seed)
    src, src_n, bumps = bumpy_sphere(P, n_bumps, amp, width, rng)
    lo, hi = src.min(axis=0), src.max(axis=0)
    if same_samples:
        base, base_n = src, src_n
    else:
        base, base_n, _ = bumpy_sphere(T, n_bumps, amp, width, rng, bumps)
    # one warp field, applied to the target samples and to the source (gt)
    _, phi = smooth_warp(base, 1.0, rng, lo, hi, return_field=True)
    # rescale the field so that the cap holds over the union of samples
    both = np.concatenate([src, base])
    disp = phi(both) - both
    s = warp_cap / float(np.linalg.norm(disp, axis=1).max())
    warp = lambda p: p + s * (phi(p) - p)
    tgt = warp(base)
    tgt_n = base_n
    gt = warp(src)
    diag = _bbox_diag(src, tgt)
    keep = crop_halfspace(tgt, crop, rng)
    tgt, tgt_n = tgt[keep], tgt_n[keep]
    tgt = add_noise(tgt, noise, diag, rng) if noise > 0 else tgt
    if outliers > 0:
        tgt, tgt_n = add_outliers(tgt, tgt_n, outliers, rng)
    src, src_n, tgt, tgt_n, gt = _f32(src, src_n, tgt, tgt_n, gt)
    return Pair(src, src_n, tgt, tgt_n, gt)


def depth_scene(P: int, seed: int, width_px: int = 640, height_px: int = 480,
                hole_frac: float = 0.15, warp_frac: float = 0.10,
                noise: float = 0.01, n_bumps: int = 32) -> Pair:
    """Depth-map pair: target = valid pixels of a synthetic 640x480 depth
    grid of a bumpy height field; source = ``P`` samples of the same surface
    region under a smooth warp (cap = ``warp_frac`` x bbox diagonal) plus
    Gaussian noise (``noise`` x bbox diagonal)."""
    rng = np.random.default_rng(seed)
    fx = fy = 525.0
    cx, cy = (width_px - 1) / 2.0, (height_px - 1) / 2.0
    bc = np.stack([rng.uniform(-1.3, 1.3, n_bumps),
                   rng.uniform(-1.0, 1.0, n_bumps)], axis=1)
    ba = rng.uniform(0.04, 0.12, n_bumps) * np.where(
        rng.random(n_bumps) < 0.5, -1.0, 1.0)
    bw = rng.uniform(0.12, 0.3, n_bumps)

    def surf(a, b):
        # point on the ray (a, b, 1) at depth z = 2 + h(2a, 2b)
        x0, y0 = 2.0 * a, 2.0 * b
        dx = x0[:, None] - bc[None, :, 0]
        dy = y0[:, None] - bc[None, :, 1]
        h = np.exp(-(dx * dx + dy * dy) / (2.0 * bw * bw)) @ ba
        z = 2.0 + h
        return np.stack([z * a, z * b, z], axis=1)

    uu, vv = np.meshgrid(np.arange(width_px, dtype=np.float64),
                         np.arange(height_px, dtype=np.float64))
    A = ((uu - cx) / fx).ravel()
    B = ((vv - cy) / fy).ravel()
    grid = surf(A, B).reshape(height_px, width_px, 3)
    # normals from grid cross products (central differences, clamped)
    gx = np.gradient(grid, axis=1)
    gy = np.gradient(grid, axis=0)
    gn = np.cross(gx, gy)
    gn /= np.linalg.norm(gn, axis=2, keepdims=True)
    valid = np.ones((height_px, width_px), dtype=bool)
    target_invalid = int(round(hole_frac * width_px * height_px))
    while (~valid).sum() < target_invalid:
        hx, hy = rng.uniform(0, width_px), rng.uniform(0, height_px)
        r = rng.uniform(8.0, 40.0)
        valid &= (uu - hx) ** 2 + (vv - hy) ** 2 >= r * r
    tgt = grid[valid]
    tgt_n = gn[valid]
    # source: continuous samples of the same image region
    a = (rng.uniform(0, width_px - 1, P) - cx) / fx
    b = (rng.uniform(0, height_px - 1, P) - cy) / fy
    base = surf(a, b)
    eps = 1e-4
    ta = surf(a + eps, b) - surf(a - eps, b)
    tb = surf(a, b + eps) - surf(a, b - eps)
    base_n = np.cross(ta, tb)
    base_n /= np.linalg.norm(base_n, axis=1, keepdims=True)
    diag = _bbox_diag(tgt)
    warped, phi = smooth_warp(base, warp_frac * diag, rng, return_field=True)
    src = add_noise(warped, noise, diag, rng)
    gt = base                       # source point i truly sits at base[i]
    src, src_n, tgt, tgt_n, gt = _f32(src, base_n, tgt, tgt_n, gt)
    return Pair(src, src_n, tgt, tgt_n, gt)


def tiny_pair(P: int, T: int, seed: int, noise: float = 0.0,
              outliers: float = 0.0) -> Pair:
    """Small bumpy-sphere pair for brute-force and unit tests."""
    return sphere_pair(P, T, n_bumps=4, amp=0.1, width=0.4, warp_cap=0.05,
                       noise=noise, outliers=outliers, crop=0.0, seed=seed,
                       same_samples=False)


def island_pair(P: int, T: int, seed: int, n_island: int = 60,
                offset: float = 2.5) -> Pair:
    """A tiny pair whose source also holds an island: ``n_island`` source
    points (a patch of the sphere around its +x pole) shifted by ``offset``
    along +x, far from every target point. The island's points are appended
    after the ``P`` surface points; its ground truth is the unshifted patch."""
    base = tiny_pair(P, T, seed=seed, noise=0.002, outliers=0.0)
    rng = np.random.default_rng(seed + 7919)
    src = base.src.astype(np.float64)
    pole = src[np.argmax(src[:, 0])]
    d = np.linalg.norm(src - pole, axis=1)
    patch = np.argsort(d)[:n_island]
    island = src[patch] + np.array([offset, 0.0, 0.0])
    island += 1e-4 * rng.standard_normal(island.shape)
    src2 = np.concatenate([src, island])
    nrm2 = np.concatenate([base.src_nrm, base.src_nrm[patch]])
    gt2 = np.concatenate([base.gt, base.gt[patch]])
    s32, n32, g32 = _f32(src2, nrm2, gt2)
    return Pair(s32, n32, base.tgt, base.tgt_nrm, g32, name="island")


# ---------------------------------------------------------------------------
# Named workloads (sizes and parameters of the benchmark configurations)
# ---------------------------------------------------------------------------

def _sphere5k(seed: int = 0) -> Pair:
    p = sphere_pair(5000, None, n_bumps=8, amp=0.1, width=0.3, warp_cap=0.15,
                    noise=0.01, outliers=0.05, crop=0.0, seed=seed,
                    same_samples=True)
    p.params = dict(radius=0.15, k_alpha=100.0, k_beta=1.0, aa_m=5,
                    iters=30, precision="fp64")
    p.name = "sphere5k"
    return p


def _sphere50k_partial(seed: int = 1) -> Pair:
    p = sphere_pair(50000, 60000, n_bumps=32, amp=0.1, width=0.3,
                    warp_cap=0.15, noise=0.02, outliers=0.10, crop=0.30,
                    seed=seed, same_samples=False)
    p.params = dict(radius=0.085, k_alpha=100.0, k_beta=1.0, aa_m=5,
                    iters=50, precision="mixed")
    p.name = "sphere50k_partial"
    return p


def _depth100k(seed: int = 2) -> Pair:
    p = depth_scene(100000, seed)
    p.params = dict(radius=0.062, k_alpha=10.0, k_beta=1.0, aa_m=5,
                    rel_energy_tol=1e-6, precision="mixed")
    p.name = "depth100k"
    return p


def _grad20k(seed: int = 4) -> Pair:
    p = sphere_pair(20000, 24000, n_bumps=32, amp=0.1, width=0.3,
                    warp_cap=0.15, noise=0.02, outliers=0.10, crop=0.30,
                    seed=seed, same_samples=False)
    p.params = dict(radius=0.14, k_alpha=100.0, k_beta=1.0, aa_m=0,
                    unroll=10, precision="fp64")
    p.name = "grad20k"
    return p


def batch_pairs(n_pairs: int = 64, seed: int = 1000):
    """Independent pairs with log-uniform point counts in [2000, 40000],
    crop U[0, 0.3], outliers U[0, 0.1]; otherwise built like sphere5k."""
    meta = np.random.default_rng(seed)
    out = []
    for i in range(n_pairs):
        P = int(round(math.exp(meta.uniform(math.log(2000), math.log(40000)))))
        crop = float(meta.uniform(0.0, 0.3))
        outl = float(meta.uniform(0.0, 0.1))
        n_nodes = int(meta.integers(100, 1001))
        p = sphere_pair(P, None, n_bumps=8, amp=0.1, width=0.3,
                        warp_cap=0.15, noise=0.01, outliers=outl, crop=crop,
                        seed=seed + i + 1, same_samples=True)
        # node count ~ surface area / R^2 on a near-unit sphere
        p.params = dict(radius=float(2.2 / math.sqrt(n_nodes)), k_alpha=100.0,
                        k_beta=1.0, aa_m=5, iters=30, precision="mixed")
        p.name = f"batch{i}"
        out.append(p)
    return out


def perturbed_transforms(N: int, seed: int, scale_a: float = 0.01,
                         scale_t: float = 0.005) -> np.ndarray:
    """Seeded node transforms near the identity, [N,12] float64 in the
    library's layout (rows 0..2 of each 4x3 block = A^T, row 3 = t)."""
    rng = np.random.default_rng(seed)
    X = np.zeros((N, 4, 3))
    X[:, 0, 0] = X[:, 1, 1] = X[:, 2, 2] = 1.0
    X[:, :3, :] += scale_a * rng.standard_normal((N, 3, 3))
    X[:, 3, :] += scale_t * rng.standard_normal((N, 3))
    return X.reshape(N, 12)


WORKLOADS = {
    "sphere5k": _sphere5k,
    "sphere50k_partial": _sphere50k_partial,
    "depth100k": _depth100k,
    "grad20k": _grad20k,
}


def workload(name: str, seed: int | None = None) -> Pair:
    fn = WORKLOADS[name]
    return fn() if seed is None else fn(seed)
