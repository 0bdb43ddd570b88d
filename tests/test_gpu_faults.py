"""Failure detection without a GPU fault: the grid-wide solve's barrier wait
is bounded. With the host-side test knob NRR_FAULT_BARRIER (read when a
context is created), one CTA skips its first arrival; every CTA's wait then
runs out after about two seconds, the kernel records NRR_E_TIMEOUT in the
context's device state and returns, and the host reports the code. The
device stays usable: a new context solves normally afterwards."""
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def test_bounded_barrier_wait_reports_timeout(monkeypatch):
    from paper_2206_03410_gb300 import nrr
    nrr.load()
    pair = synth.tiny_pair(3000, 3200, seed=81, noise=0.002, outliers=0.05)
    kw = dict(radius=0.2, aa_m=5, precision="mixed")
    monkeypatch.setenv("NRR_FAULT_BARRIER", "1")
    reg = nrr.Registration(pair.src, pair.tgt, **kw)
    monkeypatch.delenv("NRR_FAULT_BARRIER")
    reg.set_launch_config(8, 0)            # the grid-wide solve (software barrier)
    with pytest.raises(nrr.NrrError) as e:
        reg.step()
    assert e.value.code == nrr.NRR_E_TIMEOUT
    with pytest.raises(nrr.NrrError) as e2:
        reg.step()                          # the context is marked failed
    assert e2.value.code == nrr.NRR_E_STATE
    reg.close()
    torch.cuda.synchronize()
    ok = nrr.Registration(pair.src, pair.tgt, **kw)
    ok.set_launch_config(8, 0)
    info = ok.solve(3000)
    assert info.done == 1 and info.status == 0
    ok.close()


def test_bounded_halo_wait_reports_timeout(monkeypatch):
    """The cluster solve's halo wait is bounded too. With the host-side knob
    NRR_FAULT_HALO (read when a context is created), CTA 1 of the cluster
    does not push the halo rows of the first preconditioned residual; its
    neighbours' mbarrier waits run out after about two seconds, they record
    NRR_E_TIMEOUT and add NaN to the next cluster reduction, so every CTA
    leaves the solve at the same point and the kernel returns."""
    from paper_2206_03410_gb300 import nrr
    nrr.load()
    pair = synth.workload("sphere5k")
    kw = dict(radius=0.15, aa_m=5, precision="mixed")
    monkeypatch.setenv("NRR_FAULT_HALO", "1")
    reg = nrr.Registration(pair.src, pair.tgt, **kw)
    monkeypatch.delenv("NRR_FAULT_HALO")
    assert reg.launch_config().solve_ctas > 2      # CTA 1 has neighbours to push to
    with pytest.raises(nrr.NrrError) as e:
        reg.step()
    assert e.value.code == nrr.NRR_E_TIMEOUT
    reg.close()
    torch.cuda.synchronize()
    ok = nrr.Registration(pair.src, pair.tgt, **kw)
    info = ok.solve(3000)
    assert info.done == 1 and info.status == 0
    ok.close()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_pcg_iteration_cap_is_reported_not_fatal(prec):
    """Injected PCG non-convergence: with pcg_max_iters = 2 the solve stops
    after two CG iterations, far above its tolerance; the pass reports the
    iteration count and the residual reached, the MM step is taken from
    that inexact solve, and the run continues without an error status (the
    energy safeguard of Algorithm 2 still decides every kept iterate)."""
    from paper_2206_03410_gb300 import nrr
    nrr.load()
    pair = synth.tiny_pair(3000, 3200, seed=83, noise=0.002, outliers=0.05)
    reg = nrr.Registration(pair.src, pair.tgt, radius=0.2, aa_m=5, precision=prec, pcg_max_iters=2)
    info = reg.step()
    assert info.solved == 1 and info.status == 0
    assert info.pcg_iters == 2
    assert info.pcg_rel_residual > 1e-6
    for _ in range(4):
        info = reg.step()
        assert info.status == 0 and info.E == info.E   # finite, no NaN
    reg.close()
