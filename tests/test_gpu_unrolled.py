"""Unrolled MM steps and their backward (nrr_unroll, nrr_backward mode 1)
through the C ABI, against the FP64 oracle (oracle.unrolled, pinned by
central differences) and against central differences of the GPU's own
forward map.

The oracle runs its own trajectory from the same seeded X^(0) (rounded to
float for both sides). Tolerances: FP64 path 1e-8 relative to the largest
entry (PCG to relative residual 1e-12 in the forward and the adjoint
solves); mixed path 1e-4 (float X, v_hat and PCG at 1e-6 relative residual,
summed over the steps). The closest point is piecewise constant: where the
float search and the FP64 oracle pick different points at a near tie, the
loss itself jumps and the two gradients are gradients of different
functions, so the mixed-path comparisons first check that every closest
point along the trajectory agrees.
"""
import numpy as np
import pytest

import synth
from oracle import model as M, unrolled as UR
from oracle.solver import Params, Registration as OReg

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


KW = dict(radius=0.3, nu_a=0.05, nu_r=0.2, nu_a_min=0.05, aa_m=0)
TOL = {"fp64": 1e-8, "mixed": 1e-4}
# L = E(X^(K)) after K MM steps sits near a stationary point of E, where the
# gradient is small against the curvature: the float drift of the forward
# trajectory (|dX| ~ 1e-6 relative) moves dE/dX^(K) by curvature x drift,
# which the backward carries to X^(0). Measured 9e-4 on the small pair.
TOL_MIXED_ENERGY = 2e-3


def relmax(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300))


@pytest.fixture(scope="module")
def tiny():
    pair = synth.tiny_pair(1500, 1600, seed=21, noise=0.002, outliers=0.05)
    ora = OReg(pair.src, pair.tgt, Params(radius=0.3, nu_a=0.05, nu_r=0.2, nu_a_min=0.05, aa_m=0))
    return pair, ora


def _reg(pair, prec, **kw):
    nrr = _nrr()
    args = dict(KW)
    args.update(kw)
    return nrr.Registration(torch.from_numpy(pair.src).cuda(), torch.from_numpy(pair.tgt).cuda(),
                            precision=prec, **args)


def _stage(reg):
    i = reg.info()
    return i.nu_a, i.nu_r, i.alpha, i.beta


def _flips(reg, ora_graph, V, U, Xs_gpu, Xs_ora, nu_a, nu_r):
    """Closest points that differ between the GPU at its checkpoints and the
    oracle at its own, per checkpoint."""
    out = []
    for Xg, Xo in zip(Xs_gpu, Xs_ora):
        reg.energy(Xg)
        rho, _ = reg.correspondence()
        out.append(int((rho != M.energy_terms(V, U, ora_graph, Xo, nu_a, nu_r)["rho"]).sum()))
    return out


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_unroll_forward_matches_oracle(tiny, prec):
    pair, ora = tiny
    reg = _reg(pair, prec)
    K = 5
    X0 = synth.perturbed_transforms(reg.N, seed=3)
    if prec == "mixed":
        X0 = X0.astype(np.float32).astype(np.float64)
    XK = reg.unroll(K, X0)
    nu_a, nu_r, alpha, beta = _stage(reg)
    Xs = UR.unrolled_forward(ora.V, ora.U, ora.graph, X0, nu_a, nu_r, alpha, beta, K)
    tol = 1e-9 if prec == "fp64" else 1e-4
    assert relmax(XK, Xs[-1]) < tol, relmax(XK, Xs[-1])
    # the solver state is untouched: a pass afterwards still starts from identity
    info = reg.step()
    assert info.n_passes == 1 and info.stage == 0
    reg.close()


@pytest.mark.parametrize("loss", ["energy", "cotangent"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_unrolled_backward_matches_oracle(tiny, prec, loss):
    pair, ora = tiny
    reg = _reg(pair, prec)
    K = 4
    X0 = synth.perturbed_transforms(reg.N, seed=4)
    if prec == "mixed":
        X0 = X0.astype(np.float32).astype(np.float64)
    C = np.random.default_rng(9).standard_normal((reg.N, 12)) if loss == "cotangent" else None
    XK = reg.unroll(K, X0)
    gX, gv = reg.unrolled_backward(C)
    nu_a, nu_r, alpha, beta = _stage(reg)
    Xs = UR.unrolled_forward(ora.V, ora.U, ora.graph, X0, nu_a, nu_r, alpha, beta, K)
    if prec == "mixed":
        Xg = [X0] + [reg.unroll(k, X0) for k in range(1, K + 1)]
        assert _flips(reg, ora.graph, ora.V, ora.U, Xg, Xs, nu_a, nu_r) == [0] * (K + 1)
        reg.unroll(K, X0)
    ogX, ogv = UR.unrolled_backward(ora.V, ora.U, ora.graph, Xs, nu_a, nu_r, alpha, beta, cotangent=C)
    tol = TOL[prec] if (prec, loss) != ("mixed", "energy") else TOL_MIXED_ENERGY
    assert relmax(gX, ogX) < tol, relmax(gX, ogX)
    assert relmax(gv, ogv) < tol, relmax(gv, ogv)
    # deterministic: a second backward is bitwise identical
    gX2, gv2 = reg.unrolled_backward(C)
    assert np.array_equal(gX, gX2) and np.array_equal(gv, gv2)
    reg.close()


def test_unrolled_backward_matches_gpu_central_differences(tiny):
    """FP64 path: <C, dL/dX0> against central differences (h = 1e-6) of the
    GPU's own forward map L(X0) = <C, X^(K)>, in random directions."""
    pair, _ = tiny
    reg = _reg(pair, "fp64")
    K = 3
    rng = np.random.default_rng(12)
    X0 = synth.perturbed_transforms(reg.N, seed=5)
    C = rng.standard_normal((reg.N, 12))
    reg.unroll(K, X0)
    gX, _ = reg.unrolled_backward(C)
    h = 1e-6
    for _ in range(4):
        Dv = rng.standard_normal(X0.shape)
        Lp = float(np.sum(C * reg.unroll(K, X0 + h * Dv)))
        Lm = float(np.sum(C * reg.unroll(K, X0 - h * Dv)))
        fd = (Lp - Lm) / (2 * h)
        an = float(np.sum(gX * Dv))
        assert abs(fd - an) < 1e-6 * max(1.0, abs(fd)), (fd, an)
    reg.close()


def test_unroll_errors_and_autograd(tiny):
    nrr = _nrr()
    pair, _ = tiny
    reg = _reg(pair, "fp64")
    with pytest.raises(nrr.NrrError) as e:
        reg.unrolled_backward(None)        # no unroll yet
    assert e.value.code == nrr.NRR_E_STATE
    X0 = synth.perturbed_transforms(reg.N, seed=6)
    K = 3
    fn = nrr.unrolled_function()
    Xt = torch.tensor(X0, dtype=torch.float64, device="cuda", requires_grad=True)
    src = torch.tensor(pair.src.astype(np.float64), device="cuda", requires_grad=True)
    XK = fn.apply(Xt, src, reg, K)
    C = torch.randn_like(XK)
    (XK * C).sum().backward()
    gX, gv = reg.unrolled_backward(C.detach().cpu().numpy())
    assert np.array_equal(Xt.grad.cpu().numpy(), gX)
    assert np.array_equal(src.grad.cpu().numpy(), gv)
    # a stage change invalidates the checkpoints
    reg.set_stage(0.04, 0.15)
    with pytest.raises(nrr.NrrError) as e:
        reg.unrolled_backward(None)
    assert e.value.code == nrr.NRR_E_STATE
    reg.close()


@pytest.fixture(scope="module")
def grad20k():
    """The differentiation workload: 20,000 source / 18,480 target points,
    30 % crop, 10 % outliers, 604 nodes, K = 10 unrolled steps at the first
    stage's nu (paper's rule), from a seeded X^(0) near the identity; the
    oracle's trajectory and its closest points are computed once."""
    pair = synth.workload("grad20k")
    prm = pair.params
    nrr = _nrr()
    probe = nrr.Registration(torch.from_numpy(pair.src).cuda(), torch.from_numpy(pair.tgt).cuda(),
                             precision="fp64", radius=prm["radius"], aa_m=0)
    nu = _stage(probe)
    N = probe.N
    nodes = probe.graph().nodes
    probe.close()
    ora = OReg(pair.src, pair.tgt, Params(radius=prm["radius"], nu_a=1.0, nu_r=1.0, nu_a_min=1.0, aa_m=0))
    assert np.array_equal(ora.graph.nodes, nodes)
    K = prm["unroll"]
    X0 = synth.perturbed_transforms(N, seed=7).astype(np.float32).astype(np.float64)
    Xs = UR.unrolled_forward(ora.V, ora.U, ora.graph, X0, *nu, K)
    return pair, ora, nu, X0, Xs


@pytest.mark.parametrize("prec,loss", [("fp64", "energy"), ("fp64", "cotangent")])
def test_unrolled_backward_grad20k_matches_oracle(grad20k, prec, loss):
    """dL/dX^(0) and dL/dv of K = 10 unrolled steps at full size, against the
    oracle along its own trajectory. The FP64 path is the one this workload
    runs: in float, near-tie closest points along a 10-step trajectory of
    20,000 points differ from the FP64 oracle's (1-2 points per step here),
    and each such flip moves the gradient of the piecewise-smooth map by
    ~1e-2 relative."""
    pair, ora, nu, X0, Xs = grad20k
    K = len(Xs) - 1
    reg = _reg(pair, prec, radius=pair.params["radius"], nu_a=0, nu_r=0, nu_a_min=0)
    assert np.allclose(_stage(reg), nu, rtol=1e-6)
    C = np.random.default_rng(10).standard_normal((reg.N, 12)) if loss == "cotangent" else None
    XK = reg.unroll(K, X0)
    tol = TOL[prec]
    assert relmax(XK, Xs[-1]) < (1e-9 if prec == "fp64" else 1e-4)
    if prec == "mixed":
        Xg = [X0] + [reg.unroll(k, X0) for k in range(1, K + 1)]
        assert _flips(reg, ora.graph, ora.V, ora.U, Xg, Xs, nu[0], nu[1])[:K] == [0] * K
        reg.unroll(K, X0)
    gX, gv = reg.unrolled_backward(C)
    ogX, ogv = UR.unrolled_backward(ora.V, ora.U, ora.graph, Xs, *nu, cotangent=C)
    assert relmax(gX, ogX) < tol, relmax(gX, ogX)
    assert relmax(gv, ogv) < tol, relmax(gv, ogv)
    reg.close()
