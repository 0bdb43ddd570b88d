"""Pins of the oracle's exact geodesic distances and of Algorithm 1 on a mesh
source (Sec. 3.1: D of Eq. InfluenceNodes is the geodesic distance on the
source surface, computed exactly). Each pin is a surface whose geodesic
distances have a closed form, chosen so that a plausible mistake fails one:

* flat grid: D is the Euclidean distance (any error in unfolding a strip
  of faces into the plane, or a strip cut short, shows);
* L-shaped flat domain: the shortest path bends at the reflex corner
  (paths that may not bend at vertices would be too long);
* open cylinder: developable, D is the distance in the unrolled strip of
  polygon chords (unfolding across edges onto the wrong side fails);
* cube surface: D between corners and edge points by unfolding two faces
  (sqrt(5) between opposite corners);
* saddle crown: eight triangles of 50 degrees around an apex (400 degrees
  in total); ring vertices whose angular separation exceeds 180 degrees are
  joined through the apex (D = 2), the others straight across the fan.
"""
import math

import numpy as np
import pytest

import synth
from oracle import geodesic as GD


def test_flat_grid_is_euclidean():
    V, F, idx = synth.grid_mesh(6, 5)
    m = GD.Mesh(V, F)
    for s in (idx[(0, 0)], idx[(2, 3)]):
        D = GD.geodesic_from(m, s)
        for v in range(len(V)):
            assert abs(D[v] - np.linalg.norm(V[v] - V[s])) < 1e-12


def test_l_shape_bends_at_the_reflex_corner():
    V, F, idx = synth.grid_mesh(5, 5, keep=lambda i, j: i < 2 or j < 2)
    m = GD.Mesh(V, F)
    s, t, c = idx[(4, 0)], idx[(0, 4)], idx[(2, 2)]
    D = GD.geodesic_from(m, s)
    assert abs(D[t] - (np.linalg.norm(V[s] - V[c]) + np.linalg.norm(V[c] - V[t]))) < 1e-12
    # points that see each other inside the domain stay Euclidean
    assert abs(D[idx[(4, 1)]] - 1.0) < 1e-12
    assert abs(D[idx[(0, 2)]] - np.linalg.norm(V[s] - V[idx[(0, 2)]])) < 1e-12
    u = idx[(1, 4)]   # hidden behind the corner as well
    assert abs(D[u] - (np.linalg.norm(V[s] - V[c]) + np.linalg.norm(V[c] - V[u]))) < 1e-12


def test_cylinder_unrolls():
    n, rings, r, dz = 12, 4, 1.0, 0.7
    V, F = synth.cylinder_mesh(n, rings, r, dz)
    m = GD.Mesh(V, F)
    D = GD.geodesic_from(m, 0)
    chord = 2 * r * math.sin(math.pi / n)
    for j in range(rings):
        for k in range(n):
            assert abs(D[j * n + k] - math.hypot(min(k, n - k) * chord, j * dz)) < 1e-12


def test_cube_unfolds_two_faces():
    V, F = synth.cube_mesh(2)
    m = GD.Mesh(V, F)
    at = {tuple(p): i for i, p in enumerate(V)}
    D = GD.geodesic_from(m, at[(0.0, 0.0, 0.0)])
    assert abs(D[at[(1.0, 1.0, 1.0)]] - math.sqrt(5.0)) < 1e-12
    assert abs(D[at[(1.0, 0.5, 1.0)]] - math.hypot(1.0, 1.5)) < 1e-12
    assert abs(D[at[(1.0, 1.0, 0.0)]] - math.sqrt(2.0)) < 1e-12
    assert abs(D[at[(0.5, 1.0, 1.0)]] - math.hypot(1.0, 1.5)) < 1e-12


def test_saddle_crown_paths_through_the_apex():
    n, a = 8, 50.0
    V, F = synth.crown_mesh(n, a)
    assert abs(np.linalg.norm(V[1]) - 1.0) < 1e-12
    assert abs(np.linalg.norm(V[1] - V[2]) - 2 * math.sin(math.radians(a) / 2)) < 1e-12
    m = GD.Mesh(V, F)
    D = GD.geodesic_from(m, 1)
    for k in range(1, n):
        sep = min(k, n - k) * a   # degrees around the apex, the short way
        want = 2.0 if sep >= 180.0 else 2 * math.sin(math.radians(sep) / 2)
        assert abs(D[1 + k] - want) < 1e-12, (k, D[1 + k], want)


def test_limit_only_drops_far_vertices():
    V, F = synth.cylinder_mesh(10, 5, 1.0, 0.5)
    m = GD.Mesh(V, F)
    full = GD.geodesic_from(m, 3)
    lim = GD.geodesic_from(m, 3, limit=1.2)
    for v, d in full.items():
        if d < 1.2:
            assert abs(lim[v] - d) < 1e-12


def test_mesh_graph_invariants_and_flat_reduction():
    """On a flat convex grid D is Euclidean, so the mesh construction and the
    point-cloud construction give the same graph when every ball found by
    the breadth-first search is the whole Euclidean ball (the grid is
    convex, R small against it); and in general every point is influenced,
    the weights are a partition of unity, a node influences itself first."""
    V, F, idx = synth.grid_mesh(12, 10, h=0.1)
    # interior vertices moved in the plane (no exact distance ties; the
    # rectangle stays convex)
    rng = np.random.default_rng(1)
    for (i, j), v in idx.items():
        if 0 < i < 11 and 0 < j < 9:
            V[v, :2] += rng.uniform(-0.02, 0.02, 2)
    from oracle import graph as OG
    gm = GD.build_graph_mesh(V, F, 0.35, 8)
    gp = OG.build_graph(V, 0.35, 8)
    assert np.array_equal(gm.nodes, gp.nodes)
    assert np.array_equal(gm.nidx, gp.nidx)
    assert np.abs(gm.w - gp.w).max() < 1e-12
    assert np.array_equal(gm.edges, gp.edges)
    rng = np.random.default_rng(0)
    V2, _, F2, _ = synth.bumpy_sphere_mesh(2, 5, 0.15, 0.4, rng)
    g = GD.build_graph_mesh(V2, F2, 0.6, 6)
    assert np.all(g.nidx[:, 0] >= 0)
    assert np.allclose(g.w.sum(axis=1), 1.0, atol=1e-14)
    for j, v in enumerate(g.nodes):
        assert g.nidx[v, 0] == j


def test_mean_edge_length():
    V, F, _ = synth.grid_mesh(3, 3)
    # 12 axis edges of length 1 and 4 diagonals of length sqrt(2)
    assert abs(GD.mean_edge_length(V, F) - (12 + 4 * math.sqrt(2)) / 16) < 1e-15
