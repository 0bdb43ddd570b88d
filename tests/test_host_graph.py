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
