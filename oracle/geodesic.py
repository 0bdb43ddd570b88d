"""Exact geodesic distances on a triangle mesh and the deformation graph of
a mesh source (Sec. 3.1, Eq. InfluenceNodes, Eq. weight_data, Algorithm 1),
in FP64. Test infrastructure: a plain, slow restatement, not the product.

The geodesic distance D(a, b) is the length of the shortest path between
two vertices on the polyhedral surface. Such a path is a chain of straight
segments: inside one face a shortest path is straight, across an interior
edge it stays straight once the two faces are unfolded into a common plane,
and it can bend only at vertices (Sec. 3.1 computes D exactly; the paper
uses the VTP algorithm for it). This module takes that statement as the
definition and evaluates it literally:

* ``direct_distances(s)``: for every vertex b, the length of the shortest
  straight segment from vertex s to b through a strip of distinct faces
  unfolded into the plane of s's face (every strip that leaves s is
  enumerated; the set of directions from s that still pass through all of
  the strip's crossed edges is kept as a cone and the strip ends when the
  cone is empty or when the nearest point it can reach lies beyond
  ``limit``);
* ``geodesic_from(s)``: Dijkstra over the vertices with those direct
  distances as edge weights, i.e. the shortest chain of straight segments
  that meet at vertices.

Every path considered is a path on the surface, and every shortest path is
one of them (a shortest path crosses each face at most once and bends only
at vertices), so the result is the geodesic distance up to rounding. The
cost grows quickly with the mesh: this is for the small meshes of the tests.

Readings used for Algorithm 1 on a mesh (the paper leaves them open):

* The ball B(v) of Algorithm 1 is found by a breadth-first search along
  mesh edges from v that enters only vertices q with |v - q| < R (strict);
  the sub-mesh is every face incident to a vertex of B(v); D(v, q) is the
  geodesic distance on that sub-mesh (its boundary is a boundary of the
  sub-mesh surface: paths may bend around it but not leave it).
* A vertex q joins I(...) of node v when D(v, q) < R (strict), with the
  influence weight of Eq. (weight_data) computed from D(v, q)^2.
* l-bar is the mean length of the mesh edges (Sec. 4.1).
* Everything else (the PCA visiting order, the cap of ``max_influence``
  nearest nodes with ties to the lower id, edges from the capped sets,
  r_ij) is the point-cloud construction of ``oracle.graph``.
"""
from __future__ import annotations

import heapq
import math

import numpy as np

from . import graph as G


def mesh_edges(F: np.ndarray) -> np.ndarray:
    """Undirected edges (a < b) of the faces, sorted."""
    F = np.asarray(F, dtype=np.int64)
    e = np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]])
    e.sort(axis=1)
    return np.unique(e, axis=0)


def mean_edge_length(V: np.ndarray, F: np.ndarray) -> float:
    """l-bar of a mesh: the mean length of its edges."""
    V = np.asarray(V, dtype=np.float64)
    e = mesh_edges(F)
    d = V[e[:, 0]] - V[e[:, 1]]
    return float(np.mean(np.sqrt(d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] + d[:, 2] * d[:, 2])))


def _cross(a, b) -> float:
    return a[0] * b[1] - a[1] * b[0]


class Mesh:
    """Faces and edge adjacency of a triangle mesh (every edge in at most
    two faces)."""

    def __init__(self, V: np.ndarray, F: np.ndarray):
        self.V = np.asarray(V, dtype=np.float64)
        self.F = [tuple(int(x) for x in f) for f in np.asarray(F, dtype=np.int64)]
        self.edge_faces: dict[tuple[int, int], list[int]] = {}
        for fi, (a, b, c) in enumerate(self.F):
            for u, v in ((a, b), (b, c), (c, a)):
                self.edge_faces.setdefault((min(u, v), max(u, v)), []).append(fi)
        for k, fs in self.edge_faces.items():
            if len(fs) > 2:
                raise ValueError(f"edge {k} is shared by more than two faces")
        self.vert_faces: dict[int, list[int]] = {}
        for fi, f in enumerate(self.F):
            for v in f:
                self.vert_faces.setdefault(v, []).append(fi)

    def length(self, a: int, b: int) -> float:
        d = self.V[a] - self.V[b]
        return math.sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2])

    def other_face(self, u: int, v: int, f: int) -> int | None:
        for g in self.edge_faces[(min(u, v), max(u, v))]:
            if g != f:
                return g
        return None


def _third(f: tuple, u: int, v: int) -> int:
    for x in f:
        if x != u and x != v:
            return x
    raise ValueError("degenerate face")


def _unfold(pu, pv, lu: float, lv: float, away):
    """2D position of a point at distance lu from pu and lv from pv, on the
    side of line pu-pv opposite to point ``away``."""
    ex = (pv[0] - pu[0], pv[1] - pu[1])
    L = math.hypot(ex[0], ex[1])
    ux, uy = ex[0] / L, ex[1] / L
    x = (L * L + lu * lu - lv * lv) / (2.0 * L)
    y = math.sqrt(max(lu * lu - x * x, 0.0))
    nx, ny = -uy, ux
    side = (away[0] - pu[0]) * nx + (away[1] - pu[1]) * ny
    if side > 0:
        y = -y
    return (pu[0] + x * ux + y * nx, pu[1] + x * uy + y * ny)


def _dist_to_segment(p, q) -> float:
    """Distance from the origin to segment p-q (2D)."""
    dx, dy = q[0] - p[0], q[1] - p[1]
    L2 = dx * dx + dy * dy
    t = 0.0 if L2 == 0 else max(0.0, min(1.0, -(p[0] * dx + p[1] * dy) / L2))
    return math.hypot(p[0] + t * dx, p[1] + t * dy)


def direct_distances(mesh: Mesh, s: int, limit: float = math.inf,
                     faces: set | None = None) -> dict[int, float]:
    """Shortest straight-segment distances from vertex s to the vertices it
    sees through strips of distinct faces (restricted to ``faces`` if
    given). The source sits at the origin of the unfolding plane."""
    out: dict[int, float] = {}

    def see(v: int, p):
        d = math.hypot(p[0], p[1])
        if d < out.get(v, math.inf):
            out[v] = d

    def inside(lo, hi, p) -> bool:
        # p within the cone from direction lo counter-clockwise to hi
        return _cross(lo, p) >= 0.0 and _cross(p, hi) >= 0.0

    def cross_edge(u, v, pu, pv, f, lo, hi, used):
        # the strip enters the face beyond edge (u, v) of face f; pu, pv are
        # unfolded positions; (lo, hi) the cone of directions that reach the
        # edge through every crossed edge so far
        if _dist_to_segment(pu, pv) >= limit:
            return
        g = mesh.other_face(u, v, f)
        if g is None or g in used or (faces is not None and g not in faces):
            return
        w = _third(mesh.F[g], u, v)
        pw = _unfold(pu, pv, mesh.length(u, w), mesh.length(v, w), (0.0, 0.0))
        if inside(lo, hi, pw):
            see(w, pw)
        used2 = used | {g}
        # sub-edges (u, w) and (w, v): the cone restricted to each
        for a, b, pa, pb in ((u, w, pu, pw), (w, v, pw, pv)):
            # orient so that pa -> pb runs counter-clockwise around s
            if _cross(pa, pb) < 0:
                a, b, pa, pb = b, a, pb, pa
            nlo = lo if _cross(lo, pa) <= 0 else pa   # the later of lo, pa
            nhi = hi if _cross(hi, pb) >= 0 else pb   # the earlier of hi, pb
            if _cross(nlo, nhi) > 0 or (_cross(nlo, nhi) == 0 and nlo[0] * nhi[0] + nlo[1] * nhi[1] > 0):
                cross_edge(a, b, pa, pb, g, nlo, nhi, used2)

    for f in mesh.vert_faces.get(s, []):
        if faces is not None and f not in faces:
            continue
        a, b, c = mesh.F[f]
        u, v = (b, c) if a == s else (c, a) if b == s else (a, b)
        pu = (mesh.length(s, u), 0.0)
        pv = _unfold((0.0, 0.0), pu, mesh.length(s, v), mesh.length(u, v), (0.0, -1.0))
        see(u, pu)
        see(v, pv)
        if _cross(pu, pv) < 0:
            u, v, pu, pv = v, u, pv, pu
        cross_edge(u, v, pu, pv, f, pu, pv, {f})
    return out


def geodesic_from(mesh: Mesh, s: int, limit: float = math.inf,
                  faces: set | None = None) -> dict[int, float]:
    """Geodesic distances from vertex s (Dijkstra over the straight-segment
    distances between vertices); vertices farther than ``limit`` may be
    missing or overestimated beyond it."""
    direct = {}
    dist = {s: 0.0}
    heap = [(0.0, s)]
    done = set()
    while heap:
        d, a = heapq.heappop(heap)
        if a in done:
            continue
        done.add(a)
        if d >= limit:
            continue
        if a not in direct:
            direct[a] = direct_distances(mesh, a, limit - d, faces)
        for b, l in direct[a].items():
            nd = d + l
            if nd < dist.get(b, math.inf):
                dist[b] = nd
                heapq.heappush(heap, (nd, b))
    return dist


def ball(mesh: Mesh, v: int, R: float, adj: list) -> list[int]:
    """B(v) of Algorithm 1: breadth-first search along mesh edges from v
    through vertices strictly within Euclidean distance R of v."""
    R2 = R * R
    seen = {v}
    order = [v]
    k = 0
    while k < len(order):
        a = order[k]
        k += 1
        for b in adj[a]:
            if b in seen:
                continue
            d = mesh.V[b] - mesh.V[v]
            if d[0] * d[0] + d[1] * d[1] + d[2] * d[2] < R2:
                seen.add(b)
                order.append(b)
    return order


def build_graph_mesh(V: np.ndarray, F: np.ndarray, R: float, max_influence: int = 8) -> G.Graph:
    """Algorithm 1 on a mesh source: the PCA visiting order, a node for
    every visited vertex with no influencing node yet, its ball B(v), the
    geodesic distances on the sub-mesh of B(v), and the influence sets,
    weights, edges and r_ij of the point-cloud construction with D the
    geodesic distance."""
    V = np.asarray(V, dtype=np.float64)
    P = V.shape[0]
    mesh = Mesh(V, F)
    adj: list[list[int]] = [[] for _ in range(P)]
    for a, b in mesh_edges(F):
        adj[int(a)].append(int(b))
        adj[int(b)].append(int(a))
    order = G.pca_order(V)
    R2 = float(R) * float(R)
    infl: list[list[tuple[float, int]]] = [[] for _ in range(P)]
    nodes: list[int] = []
    for i in order:
        i = int(i)
        if nodes and infl[i]:
            continue
        j = len(nodes)
        nodes.append(i)
        B = ball(mesh, i, R, adj)
        sub = set()
        for q in B:
            sub.update(mesh.vert_faces.get(q, []))
        D = geodesic_from(mesh, i, R, sub)
        for q in B:
            d = D.get(q, math.inf)
            if d < R:
                infl[q].append((d * d, j))
    N = len(nodes)
    K = max_influence
    nidx = -np.ones((P, K), dtype=np.int64)
    w = np.zeros((P, K), dtype=np.float64)
    edge_set = set()
    for i in range(P):
        lst = sorted(infl[i])[:K]
        ids = [j for _, j in lst]
        raw = np.array([(1.0 - d2 / R2) ** 3 for d2, _ in lst])
        nidx[i, :len(ids)] = ids
        w[i, :len(ids)] = raw / raw.sum()
        for a in range(len(ids)):
            for b in range(a + 1, len(ids)):
                j, k = ids[a], ids[b]
                edge_set.add((min(j, k), max(j, k)))
    edges = np.array(sorted(edge_set), dtype=np.int64).reshape(-1, 2)
    p = V[np.array(nodes, dtype=np.int64)] if N else np.zeros((0, 3))
    both = np.concatenate([edges, edges[:, ::-1]]) if len(edges) else edges
    dpair = both[np.lexsort((both[:, 1], both[:, 0]))] if len(both) else both
    r = G.edge_normalisation(p, dpair, len(edges))
    return G.Graph(np.array(nodes, dtype=np.int64), p, nidx, w, edges, dpair, r, float(R))
