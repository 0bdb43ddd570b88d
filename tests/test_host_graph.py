"""The library's deformation graph (Algorithm 1 with Euclidean distances,
Sec. 3.1; weights of Eq. (weight_data); r_ij of Sec. 3.2) built on the host
through nrr_graph_build, without a GPU, against the oracle's graph builder:
identical nodes, influence sets and edges, weights to rounding. The same
host code builds the graph inside nrr_create."""
import numpy as np
import pytest

import synth
from oracle import graph as OG
from paper_2206_03410_gb300 import build as B
from paper_2206_03410_gb300 import nrr


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    nrr.load()


def relmax(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("case", [("sphere5k", 0.15, 8), ("tiny", 0.3, 4), ("tiny", 0.0, 8)])
def test_host_graph_matches_oracle(case):
    name, R, K = case
    pair = synth.workload("sphere5k") if name == "sphere5k" else synth.tiny_pair(700, 720, seed=5)
    V = pair.src.astype(np.float64)           # the library reads float32, exactly representable
    g = nrr.build_graph(pair.src, radius=R, max_influence=K)
    lbar = OG.mean_spacing(V)
    assert abs(g.lbar - lbar) < 1e-12 * lbar
    og = OG.build_graph(V, R if R > 0 else 5.0 * lbar, K)
    assert np.array_equal(g.nodes, og.nodes)
    assert np.array_equal(g.nidx, og.nidx)
    assert np.array_equal(g.edges, og.edges)
    assert relmax(g.w, og.w) < 1e-13
    assert relmax(g.r, og.r) < 1e-12
    # invariants of the construction: every point is influenced, weights
    # form a partition of unity
    assert np.all(g.nidx[:, 0] >= 0)
    assert np.allclose(g.w.sum(axis=1), 1.0, atol=1e-13)


def test_host_graph_rejects_bad_arguments():
    pts = np.zeros((10, 3), dtype=np.float32)
    with pytest.raises(nrr.NrrError) as e:
        nrr.build_graph(pts[:0], radius=0.1)
    assert e.value.code == nrr.NRR_E_INVALID
    bad = pts.copy()
    bad[3, 1] = np.nan
    with pytest.raises(nrr.NrrError) as e:
        nrr.build_graph(bad, radius=0.1)
    assert e.value.code == nrr.NRR_E_INVALID
    with pytest.raises(nrr.NrrError) as e:
        nrr.build_graph(pts, radius=float("inf"))
    assert e.value.code == nrr.NRR_E_INVALID
    with pytest.raises(nrr.NrrError) as e:
        nrr.build_graph(pts, radius=0.1, max_influence=9)
    assert e.value.code == nrr.NRR_E_INVALID


def test_host_graph_default_radius_needs_spread_points():
    """With the default radius 5 lbar, identical points give lbar = 0 and no
    valid radius: the call fails instead of building a degenerate graph."""
    pts = np.repeat(np.array([[0.1, 0.2, 0.3]], np.float32), 20, axis=0)
    with pytest.raises(nrr.NrrError) as e:
        nrr.build_graph(pts, radius=0.0)
    assert e.value.code == nrr.NRR_E_INVALID
    g = nrr.build_graph(pts, radius=0.1)      # an explicit radius works
    assert len(g.nodes) == 1 and g.lbar == 0.0


# ---- triangle-mesh source: geodesic D (nrr_graph_build_mesh) ----------------

def _mesh_cases():
    rng = np.random.default_rng(3)
    V3, _, F3, _ = synth.bumpy_sphere_mesh(3, 6, 0.15, 0.4, rng)
    V2, _, F2, _ = synth.bumpy_sphere_mesh(2, 4, 0.2, 0.5, rng)
    Vg, Fg, idx = synth.grid_mesh(14, 12, h=0.1, keep=lambda i, j: not (4 <= i < 8 and 3 <= j < 7))
    rg = np.random.default_rng(4)
    for v in range(len(Vg)):
        Vg[v] += rg.uniform(-0.01, 0.01, 3) * np.array([1.0, 1.0, 2.0])
    # symmetric meshes are jittered: a tie in the PCA axis or in the
    # projections would make the visiting order depend on rounding
    Vc, Fc = synth.cylinder_mesh(16, 6, 0.5, 0.2)
    Vk, Fk = synth.crown_mesh(8, 50.0)
    Vq, Fq = synth.cube_mesh(3)
    for Vx in (Vc, Vk, Vq):
        Vx += rg.uniform(-2e-3, 2e-3, Vx.shape)
    return {
        "icosphere3_5lbar": (V3, F3, 0.0, 8),
        "icosphere3_3lbar": (V3, F3, 3.0, 8),
        "icosphere2_K4": (V2, F2, 0.5, 4),
        "holed_grid": (Vg, Fg, 0.33, 8),        # boundary around a hole: paths bend there
        "cylinder": (Vc, Fc, 0.55, 8),
        "saddle_crown": (Vk, Fk, 1.3, 8),
        "cube": (Vq, Fq, 0.9, 8),
    }


@pytest.mark.parametrize("name", list(_mesh_cases().keys()))
def test_host_mesh_graph_matches_oracle(name):
    from oracle import geodesic as GD
    V, F, R, K = _mesh_cases()[name]
    V32 = V.astype(np.float32)
    V64 = V32.astype(np.float64)
    lbar = GD.mean_edge_length(V64, F)
    if name == "icosphere3_3lbar":
        R = 3.0 * lbar
    g = nrr.build_graph(V32, radius=R, max_influence=K, faces=F)
    assert abs(g.lbar - lbar) < 1e-13 * lbar
    og = GD.build_graph_mesh(V64, F, R if R > 0 else 5.0 * lbar, K)
    assert np.array_equal(g.nodes, og.nodes)
    assert np.array_equal(g.nidx, og.nidx)
    assert np.array_equal(g.edges, og.edges)
    assert relmax(g.w, og.w) < 1e-12
    assert relmax(g.r, og.r) < 1e-12


def test_host_mesh_graph_rejects_bad_meshes():
    V, F, _ = synth.grid_mesh(4, 4)
    V32 = V.astype(np.float32)
    bad = {
        "index out of range": np.vstack([F, [[0, 1, 99]]]),
        "repeated vertex": np.vstack([F, [[0, 0, 1]]]),
        "non-manifold edge": np.vstack([F, [[0, 5, 15]]]),   # (0, 5) is the diagonal of cell (0, 0)
    }
    for why, Fb in bad.items():
        with pytest.raises(nrr.NrrError) as e:
            nrr.build_graph(V32, radius=1.5, faces=Fb)
        assert e.value.code == nrr.NRR_E_INVALID, why
    # a zero-length edge (two vertices at one position)
    Vz = V32.copy()
    Vz[1] = Vz[0]
    with pytest.raises(nrr.NrrError):
        nrr.build_graph(Vz, radius=1.5, faces=F)
    lib = nrr.load()
    g = nrr._VP()
    assert lib.nrr_graph_build_mesh(None, nrr._ptr(V32), 16, nrr._ptr(F.astype(np.int32)), len(F), 1.0, 8) \
        == nrr.NRR_E_INVALID
    assert lib.nrr_graph_build_mesh(g, nrr._ptr(V32), 16, None, len(F), 1.0, 8) == nrr.NRR_E_INVALID
    assert lib.nrr_graph_build_mesh(g, nrr._ptr(V32), 16, nrr._ptr(F.astype(np.int32)), 0, 1.0, 8) \
        == nrr.NRR_E_INVALID


def test_host_graph_from_concurrent_threads():
    """The host construction runs its parallel loops on one pool of worker
    threads shared by every caller: graphs built from several Python
    threads at once (ctypes releases the GIL during the call) are those
    built one after another, bit for bit."""
    import concurrent.futures
    srcs = [synth.tiny_pair(6000 + 500 * k, 100, seed=30 + k).src for k in range(6)]
    radii = [0.12, 0.15, 0.1, 0.13, 0.11, 0.14]
    ref = [nrr.build_graph(s, radius=r) for s, r in zip(srcs, radii)]
    with concurrent.futures.ThreadPoolExecutor(max_workers=6) as ex:
        got = list(ex.map(lambda a: nrr.build_graph(a[0], radius=a[1]), zip(srcs, radii)))
    for a, b in zip(got, ref):
        assert np.array_equal(a.nodes, b.nodes)
        assert np.array_equal(a.nidx, b.nidx)
        assert np.array_equal(a.w, b.w)
        assert np.array_equal(a.edges, b.edges)
        assert np.array_equal(a.r, b.r)
        assert a.lbar == b.lbar
