"""Deformation graph construction (Sec. 3.1, Algorithm 1) in FP64.

Readings of the paper used here (the paper works on triangle meshes with
geodesic distances; the inputs here are point clouds):

* D(.,.) is the Euclidean distance. The paper notes that the Euclidean
  distance bounds the geodesic one from below (Sec. 3.1), and the ball
  B(v_j) of Algorithm 1 is then exactly the set {q : |v_j - q| < R}.
* The PCA axis is the eigenvector of the largest eigenvalue of the FP64
  covariance (1/P) sum (v - mean)(v - mean)^T; its sign makes the entry of
  largest magnitude positive. Points are visited in ascending order of
  their projection on that axis; equal projections keep the lower index.
* Influence sets keep at most ``max_influence`` nodes, the nearest ones
  (ties to the lower node id). Edges come from the capped sets.
* Squared distances are evaluated as ``dx*dx + dy*dy + dz*dz`` left to right
  in FP64, and membership uses the strict test ``d^2 < R^2``.
* l-bar (mean edge length) of a point cloud: mean distance of every source
  point to its 6 nearest other source points.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def _sqdist_to(V: np.ndarray, q: np.ndarray) -> np.ndarray:
    dx = V[:, 0] - q[0]
    dy = V[:, 1] - q[1]
    dz = V[:, 2] - q[2]
    return dx * dx + dy * dy + dz * dz


def mean_spacing(V: np.ndarray, k: int = 6) -> float:
    """l-bar: mean distance from each point to its k nearest other points,
    by brute force over all pairs."""
    V = np.asarray(V, dtype=np.float64)
    P = V.shape[0]
    if P < 2:
        return 0.0
    kk = min(k, P - 1)
    total = 0.0
    for i in range(P):
        d2 = _sqdist_to(V, V[i])
        d2[i] = np.inf
        part = np.partition(d2, kk - 1)[:kk]
        total += float(np.sum(np.sqrt(part)))
    return total / (P * kk)


def pca_axis(V: np.ndarray) -> np.ndarray:
    """Axis of the largest eigenvalue of the covariance (Algorithm 1)."""
    V = np.asarray(V, dtype=np.float64)
    c = V - V.mean(axis=0)
    C = (c.T @ c) / V.shape[0]
    evals, evecs = np.linalg.eigh(C)
    a = evecs[:, int(np.argmax(evals))].copy()
    if a[int(np.argmax(np.abs(a)))] < 0:
        a = -a
    return a


def pca_order(V: np.ndarray) -> np.ndarray:
    a = pca_axis(V)
    V = np.asarray(V, dtype=np.float64)
    proj = V[:, 0] * a[0] + V[:, 1] * a[1] + V[:, 2] * a[2]
    idx = np.arange(V.shape[0])
    return np.lexsort((idx, proj))


@dataclass
class Graph:
    nodes: np.ndarray        # [N] source index of each node
    p: np.ndarray            # [N,3] node positions (float64)
    nidx: np.ndarray         # [P,K] node ids of I(v_i), -1 padded, by (d^2, id)
    w: np.ndarray            # [P,K] weights of Eq. (weight_data), 0 padded
    edges: np.ndarray        # [|E_G|,2] undirected edges j<k, sorted
    dpair: np.ndarray        # [2|E_G|,2] directed pairs (i,j), sorted by (i,j)
    r: np.ndarray            # [2|E_G|] normalisation weight r_ij
    radius: float

    @property
    def N(self) -> int:
        return int(self.nodes.shape[0])

    @property
    def n_edges(self) -> int:
        return int(self.edges.shape[0])


def build_graph(V: np.ndarray, R: float, max_influence: int = 8) -> Graph:
    """Algorithm 1 with Euclidean distances, then the edge weights r_ij."""
    V = np.asarray(V, dtype=np.float64)
    P = V.shape[0]
    R2 = float(R) * float(R)
    order = pca_order(V)
    infl: list[list[tuple[float, int]]] = [[] for _ in range(P)]
    nodes: list[int] = []
    for i in order:
        if len(nodes) == 0 or len(infl[i]) == 0:
            j = len(nodes)
            nodes.append(int(i))
            d2 = _sqdist_to(V, V[i])
            for q in np.nonzero(d2 < R2)[0]:
                infl[int(q)].append((float(d2[q]), j))
    N = len(nodes)
    K = max_influence
    nidx = -np.ones((P, K), dtype=np.int64)
    w = np.zeros((P, K), dtype=np.float64)
    edge_set = set()
    for i in range(P):
        lst = sorted(infl[i])[:K]
        ids = [j for _, j in lst]
        # Eq. (weight_data): (1 - D^2/R^2)^3, normalised over I(v_i)
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
    r = edge_normalisation(p, dpair, len(edges))
    return Graph(np.array(nodes, dtype=np.int64), p, nidx, w, edges, dpair,
                 r, float(R))


def edge_normalisation(p: np.ndarray, dpair: np.ndarray,
                       n_edges: int) -> np.ndarray:
    """r_ij of Sec. 3.2: 2|E_G| |p_i - p_j|^-1 divided by the sum of
    |p_i - p_j|^-1 over all directed neighbour pairs."""
    if len(dpair) == 0:
        return np.zeros(0)
    d = p[dpair[:, 0]] - p[dpair[:, 1]]
    inv = 1.0 / np.sqrt(d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] + d[:, 2] * d[:, 2])
    return 2.0 * n_edges * inv / inv.sum()
