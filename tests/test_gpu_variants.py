"""The robust-norm variants of Sec. 4.2 (NRR_L2, NRR_L2_TRUNCATED) and the
fixed-nu schedules (Welsch-fmax/fmin/fmed) through the C ABI, against the
FP64 oracle: stage parameters, energy terms, the surrogate system and its
solution, a short trajectory of Algorithm 2, and the unrolled backward.

Tolerances as in test_gpu_parity: FP64 path to rounding (energies 1e-10,
K and B 1e-11, transforms 1e-9 relative to the largest entry), mixed path
1e-5 (energies, K, B) and 1e-4 (transforms). The truncated variant decides
each alignment weight by comparing d^2 with 9 nu_a^2; the mixed-path checks
first assert that no point lies within float rounding of that threshold
(where the two precisions may decide differently).
"""
import numpy as np
import pytest

import synth
from oracle import model as M, surrogate as S, unrolled as UR
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


def relmax(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300))


@pytest.fixture(scope="module")
def pair():
    return synth.tiny_pair(2000, 2200, seed=71, noise=0.002, outliers=0.05)


BASE = dict(radius=0.25, aa_m=5)


def _both(pair, prec, **kw):
    args = dict(BASE)
    args.update(kw)
    nrr = _nrr()
    reg = nrr.Registration(pair.src, pair.tgt, precision=prec, **args)
    ora = OReg(pair.src, pair.tgt, Params(**args))
    return reg, ora


@pytest.mark.parametrize("kw", [dict(robust="l2"), dict(robust="l2r"), dict(nu_fixed="max"),
                                dict(nu_fixed="min"), dict(nu_fixed="med"),
                                dict(robust="l2r", nu_fixed="min")])
def test_stage_parameters_match_oracle(pair, kw):
    reg, ora = _both(pair, "fp64", **kw)
    info = reg.info()
    a, b = ora.weights()
    for g, o in [(info.nu_a, ora.nu_a), (info.nu_r, ora.nu_r), (info.alpha, a), (info.beta, b)]:
        assert abs(g - o) <= 1e-12 * abs(o), (kw, g, o)
    reg.close()


def _near_cutoff(d2, nu_a):
    return np.abs(d2 - 9 * nu_a * nu_a) <= 1e-5 * 9 * nu_a * nu_a


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("robust", ["l2", "l2r"])
def test_energy_system_and_solution_match_oracle(pair, robust, prec):
    """At the same iterate X: E terms, K, B (from one pass) and the
    minimiser G of the surrogate."""
    # for the truncation, a nu_a whose 3 nu_a cut-off excludes some points
    extra = dict(nu_a=0.015, nu_a_min=0.015) if robust == "l2r" else {}
    reg, ora = _both(pair, prec, robust=robust, **extra)
    X = synth.perturbed_transforms(reg.N, seed=72)
    if prec == "mixed":
        X = X.astype(np.float32).astype(np.float64)
    reg.set_transforms(X)
    info = reg.step()
    assert info.solved == 1
    t = ora.terms(X)
    if robust == "l2r":
        assert not _near_cutoff(t["d2"], ora.nu_a).any()
        assert (t["d2"] >= 9 * ora.nu_a ** 2).sum() > 0       # the truncation acts
    a, b = ora.weights()
    Eo = M.total_energy(t, a, b)
    tolE = 1e-10 if prec == "fp64" else 1e-5
    assert abs(info.E - Eo) <= tolE * abs(Eo), (info.E, Eo)
    assert abs(info.E_align - t["E_align"]) <= tolE * abs(t["E_align"])
    rho, _ = reg.correspondence()
    assert (rho == t["rho"]).mean() > 0.999
    K, B = reg.system(dense=True)
    Ko, Bo, _ = S.normal_equations(ora.V, ora.U, ora.graph, t, ora.nu_a, ora.nu_r, a, b, robust=robust)
    tolK = 1e-11 if prec == "fp64" else 1e-5
    assert relmax(K, Ko.toarray()) < tolK and relmax(B, np.asarray(Bo)) < tolK
    G = reg.mm_solution()
    Go = S.solve_normal_equations(Ko, Bo)
    assert relmax(G, Go) < (1e-9 if prec == "fp64" else 1e-4)
    reg.close()


@pytest.mark.parametrize("kw", [dict(robust="l2"), dict(robust="l2r"), dict(nu_fixed="min")])
def test_fp64_trajectory_matches_oracle(pair, kw):
    """Six passes of Algorithm 2 (MM + AA + safeguard) from X = I."""
    reg, ora = _both(pair, "fp64", **kw)
    for k in range(6):
        info = reg.step()
        rec = ora.step()
        assert info.kept == int(rec.kept), (kw, k)
        assert abs(info.E - rec.E) <= 1e-9 * abs(rec.E), (kw, k, info.E, rec.E)
        assert relmax(reg.transforms(), ora.X) < 1e-6, (kw, k)
    reg.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("robust", ["l2", "l2r"])
def test_variants_converge(pair, robust, prec):
    reg, _ = _both(pair, prec, robust=robust, rel_energy_tol=1e-6)
    info = reg.solve(3000)
    assert info.done == 1 and info.status == 0
    reg.close()


@pytest.mark.parametrize("robust", ["l2", "l2r"])
def test_unrolled_backward_matches_oracle(pair, robust):
    reg, ora = _both(pair, "fp64", robust=robust, aa_m=0)
    K = 3
    X0 = synth.perturbed_transforms(reg.N, seed=73)
    C = np.random.default_rng(74).standard_normal((reg.N, 12))
    XK = reg.unroll(K, X0)
    gX, gv = reg.unrolled_backward(C)
    info = reg.info()
    a, b = info.alpha, info.beta
    Xs = UR.unrolled_forward(ora.V, ora.U, ora.graph, X0, info.nu_a, info.nu_r, a, b, K, robust=robust)
    assert relmax(XK, Xs[-1]) < 1e-9
    ogX, ogv = UR.unrolled_backward(ora.V, ora.U, ora.graph, Xs, info.nu_a, info.nu_r, a, b,
                                    cotangent=C, robust=robust)
    assert relmax(gX, ogX) < 1e-8 and relmax(gv, ogv) < 1e-8
    reg.close()
