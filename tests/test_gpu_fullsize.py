"""Parity at the full benchmark sizes, in the launch configuration bench.py
times (mixed precision, default launch shapes), on outputs the oracle can
compute one by one: the whole deformation graph, the regularisation and
rotation terms, and the closest points and distances of a random sample of
source points (brute force over all targets for each sampled point)."""
import numpy as np
import pytest

import synth
from oracle import graph as OG, model as M

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


@pytest.mark.parametrize("name", ["depth100k", "sphere50k_partial"])
def test_full_size_sampled_parity(name):
    from paper_2206_03410_gb300 import nrr
    pair = synth.workload(name)
    kw = {k: v for k, v in pair.params.items() if k not in ("precision", "iters", "unroll")}
    reg = nrr.Registration(torch.from_numpy(pair.src).cuda(), torch.from_numpy(pair.tgt).cuda(),
                           precision="mixed", **kw)
    V = pair.src.astype(np.float64)
    U = pair.tgt.astype(np.float64)
    g = OG.build_graph(V, kw["radius"])
    gg = reg.graph()
    assert np.array_equal(gg.nodes, g.nodes) and np.array_equal(gg.nidx, g.nidx)
    assert np.array_equal(gg.edges, g.edges)
    X = synth.perturbed_transforms(reg.N, seed=23, scale_a=0.003, scale_t=0.002)
    X = X.astype(np.float32).astype(np.float64)
    e = reg.energy(X)
    info = reg.info()
    # regularisation and rotation terms over all pairs and nodes
    D = M.reg_residuals(g.p, g.dpair, g.r, X)
    e_reg = float(np.sum(M.welsch(np.sum(D * D, axis=1), info.nu_r)))
    A = M.A_of(X)
    e_rot = float(np.sum((A - M.proj_rotation(A)) ** 2))
    assert abs(e[2] - e_reg) < 1e-5 * e_reg
    assert abs(e[3] - e_rot) < 1e-5 * e_rot
    # closest points of 1,500 random source points
    rng = np.random.default_rng(7)
    idx = np.sort(rng.choice(reg.P, size=1500, replace=False))
    vh_o = M.deform(V[idx], g.nidx[idx], g.w[idx], g.p, X)
    rho_o, d2_o = M.closest_points(vh_o, U)
    rho, d2 = reg.correspondence()
    vh = reg.deformed()
    assert np.abs(vh[idx] - vh_o).max() < 4e-6
    diff = np.nonzero(rho[idx] != rho_o)[0]
    if len(diff):
        # a different index must be the exact minimiser for the GPU's float point
        rb, db = M.closest_points(vh[idx][diff], U)
        dg = np.sum((vh[idx][diff] - U[rho[idx][diff]]) ** 2, axis=1)
        assert np.all(dg <= db * (1 + 1e-6) + 1e-15)
    assert len(diff) <= 3
    # distances to the same target point: by the triangle inequality they
    # differ by at most |v_hat_gpu - v_hat_oracle|, plus float rounding
    same = rho[idx] == rho_o
    dg, do = np.sqrt(d2[idx][same]), np.sqrt(d2_o[same])
    dv = np.linalg.norm(vh[idx][same] - vh_o[same], axis=1)
    assert np.all(np.abs(dg - do) <= dv * (1 + 1e-6) + 2e-7 * do + 1e-9)
    reg.close()
