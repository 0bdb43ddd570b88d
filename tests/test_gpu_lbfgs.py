"""The preliminary version's solver (closest points held at X^k, inner
L-BFGS with a backtracking line search; Sec. 3.3.4 and Sec. 4.3) on the GPU
through the C ABI against the FP64 oracle's restatement: outer iteration by
outer iteration in FP64 (energies 1e-9, iterates 1e-8: the line searches
take the same decisions), a whole run in both precisions, and argument
checks."""
import numpy as np
import pytest

import synth
from oracle.lbfgs import LbfgsParams, LbfgsRegistration
from oracle.solver import Params

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


def test_fp64_outer_iterations_match_oracle():
    nrr = _nrr()
    pair = synth.tiny_pair(800, 880, seed=31, noise=0.002, outliers=0.05)
    # four stages (nu_a 0.05, 0.025, 0.0125, 0.01) of at most three outer
    # iterations: the run below crosses a stage end
    kw = dict(radius=0.3, aa_m=5, max_iters_per_stage=3, nu_a=0.05, nu_r=0.2, nu_a_min=0.01)
    ora = LbfgsRegistration(pair.src, pair.tgt, Params(**kw), LbfgsParams(max_inner=8))
    reg = nrr.Registration(pair.src, pair.tgt, precision="fp64", **kw)
    for k in range(5):
        rec = ora.step()
        assert rec is not None
        info = reg.solve_lbfgs(1, max_inner=8)
        # info.stage is the stage after the pass (a stage end moves it on)
        assert info.n_passes == k + 1 and info.stage == ora.stage, k
        assert abs(info.E - rec.E) < 1e-9 * abs(rec.E), (k, info.E, rec.E)
        X = reg.transforms()
        assert relmax(X, ora.X) < 1e-8, (k, relmax(X, ora.X))
        if rec.max_disp == rec.max_disp:
            assert abs(info.max_disp - rec.max_disp) < 1e-8 * rec.max_disp + 1e-14, k
    reg.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_lbfgs_run_converges(prec):
    """A whole run of the stage loop with the relative-energy stopping rule:
    it returns, the energy falls from the first to the last outer iterate,
    and it ends within 1 % of the oracle's final energy (the two
    trajectories take different float paths)."""
    nrr = _nrr()
    pair = synth.tiny_pair(600, 660, seed=43, noise=0.002, outliers=0.05)
    kw = dict(radius=0.3, rel_energy_tol=1e-4, max_iters_per_stage=15)
    reg = nrr.Registration(pair.src, pair.tgt, precision=prec, **kw)
    E0 = reg.energy()[0]
    info = reg.solve_lbfgs(0, max_inner=10)
    assert info.done == 1 and info.status == 0
    ora = LbfgsRegistration(pair.src, pair.tgt, Params(**kw), LbfgsParams(max_inner=10))
    ora.solve()
    ora.nu_a, ora.nu_r = info.nu_a, info.nu_r
    Eg, _ = ora.energy(reg.transforms())
    Eo, _ = ora.energy(ora.X)
    assert Eg < E0
    assert abs(Eg - Eo) < 1e-2 * Eo, (Eg, Eo)
    # the Algorithm 2 passes may follow the comparison solver
    reg.reset()
    assert reg.step().status == 0
    reg.close()


def test_lbfgs_rejects_bad_parameters():
    nrr = _nrr()
    pair = synth.tiny_pair(300, 320, seed=44)
    reg = nrr.Registration(pair.src, pair.tgt, precision="mixed", radius=0.4)
    for bad in (dict(m=0), dict(m=9), dict(c1=0.0), dict(c1=1.0), dict(g_tol=1.0), dict(max_inner=0),
                dict(max_halvings=61)):
        with pytest.raises(nrr.NrrError) as e:
            reg.solve_lbfgs(1, **bad)
        assert e.value.code == nrr.NRR_E_INVALID, bad
    reg.close()
