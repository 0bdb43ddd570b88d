"""Algorithm 1 on the GPU (nrr_graph_build_gpu, and nrr_create with
graph_on_gpu = 1) against the host construction and the FP64 oracle: the
same nodes (the greedy sampling's lexicographically first maximal
independent set in PCA order), the same influence sets and edges, and the
weights bit for bit and r_ij to rounding; on the 5,000-point sphere (also against the
oracle), a small pair with a capped influence width and with the default
radius 5 l-bar, the full-size depth workload, a 250,000-point sphere (the
greedy sampling with its states in global memory) and pairs of the batched
workload."""
import numpy as np
import pytest

import synth
from oracle import graph as OG

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _nrr():
    from paper_2206_03410_gb300 import nrr
    nrr.load()
    return nrr


def relmax(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300))


def _same(gg, gh):
    assert np.array_equal(gg.nodes, gh.nodes)
    assert np.array_equal(gg.nidx, gh.nidx)
    assert np.array_equal(gg.edges, gh.edges)
    # the same distances, cube (two products) and normalisation order
    assert np.array_equal(gg.w, gh.w)
    if len(gh.r):
        assert relmax(gg.r, gh.r) < 1e-12


def _cases():
    out = [("sphere5k", synth.workload("sphere5k").src, 0.15, 8),
           ("tiny_k4", synth.tiny_pair(700, 720, seed=5).src, 0.3, 4),
           ("tiny_default_radius", synth.tiny_pair(700, 720, seed=5).src, 0.0, 8),
           ("depth100k", synth.workload("depth100k").src, 0.062, 8),
           # beyond the shared-memory greedy sampling's 200,000 points
           ("sphere250k", synth.tiny_pair(250000, 1000, seed=3).src, 0.08, 8)]
    for p in synth.batch_pairs(64)[:6]:
        out.append((p.name, p.src, p.params["radius"], 8))
    return out


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c[0])
def test_gpu_graph_equals_host_graph(case):
    nrr = _nrr()
    name, src, R, K = case
    gh = nrr.build_graph(src, radius=R, max_influence=K)
    gg = nrr.build_graph(torch.from_numpy(src).cuda(), radius=R, max_influence=K, on_gpu=True)
    _same(gg, gh)
    # l-bar: with a given radius computed on the GPU on the graph's grid (the
    # host's per-point values, summed in another order)
    assert abs(gg.lbar - gh.lbar) < 1e-12 * gh.lbar


def test_gpu_lbar_matches_oracle_and_falls_back():
    """l-bar on the GPU against the oracle's brute-force mean 6-NN spacing;
    points whose six nearest others are not within R (far outliers) are
    searched by brute force on the GPU, and with more of them than the GPU
    lists (4,096) the host computes l-bar: the same result each way."""
    nrr = _nrr()
    src = synth.tiny_pair(700, 720, seed=5).src
    gg = nrr.build_graph(torch.from_numpy(src).cuda(), radius=0.3, on_gpu=True)
    lo = OG.mean_spacing(src.astype(np.float64))
    assert abs(gg.lbar - lo) < 1e-12 * lo
    far = np.concatenate([src, np.array([[40.0, 40.0, 40.0]], dtype=np.float32)])
    gg = nrr.build_graph(torch.from_numpy(far).cuda(), radius=0.3, on_gpu=True)
    gh = nrr.build_graph(far, radius=0.3)
    lo = OG.mean_spacing(far.astype(np.float64))
    assert abs(gg.lbar - lo) < 1e-12 * lo and abs(gh.lbar - lo) < 1e-12 * lo
    # a sparse cloud: every point uncertified, some 60 or all 5,000 of them
    rng = np.random.default_rng(8)
    for n_far in (60, 5000):
        pts = np.concatenate([src, rng.uniform(-50, 50, (n_far, 3)).astype(np.float32)])
        gg = nrr.build_graph(torch.from_numpy(pts).cuda(), radius=0.3, on_gpu=True)
        gh = nrr.build_graph(pts, radius=0.3)
        lo = OG.mean_spacing(pts.astype(np.float64))
        assert abs(gg.lbar - lo) < 1e-12 * lo and abs(gh.lbar - lo) < 1e-12 * lo, n_far


def test_gpu_graph_equals_oracle():
    nrr = _nrr()
    src = synth.workload("sphere5k").src
    og = OG.build_graph(src.astype(np.float64), 0.15)
    gg = nrr.build_graph(src, radius=0.15, on_gpu=True)
    assert np.array_equal(gg.nodes, og.nodes)
    assert np.array_equal(gg.nidx, og.nidx)
    assert np.array_equal(gg.edges, og.edges)
    assert relmax(gg.w, og.w) < 1e-13
    assert relmax(gg.r, og.r) < 1e-12


def test_create_with_graph_on_gpu():
    """nrr_create builds the same context with either construction: the same
    graph and the same first pass (to rounding)."""
    nrr = _nrr()
    pair = synth.workload("sphere5k")
    kw = dict(radius=0.15, aa_m=5, precision="fp64")
    a = nrr.Registration(pair.src, pair.tgt, **kw)
    b = nrr.Registration(pair.src, pair.tgt, graph_on_gpu=1, **kw)
    _same(b.graph(), a.graph())
    # r_ij agrees to rounding (its sum order differs between the
    # constructions), so the first pass agrees to rounding
    ia, ib = a.step(), b.step()
    assert abs(ia.E - ib.E) < 1e-12 * abs(ia.E)
    assert relmax(b.transforms(), a.transforms()) < 1e-11
    a.close()
    b.close()
