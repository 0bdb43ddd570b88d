"""Checkpoint / resume through the C ABI: a solve saved after some passes
and resumed in a fresh context of the same problem ends bitwise where the
uninterrupted solve ends; a state from another problem (other sizes, or
the same sizes with another target or other parameters) is rejected."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_resume_is_bitwise_identical(prec):
    from paper_2206_03410_gb300 import nrr
    pair = synth.tiny_pair(2500, 2700, seed=91, noise=0.002, outliers=0.05)
    kw = dict(radius=0.25, aa_m=5, precision=prec, rel_energy_tol=1e-6)
    a = nrr.Registration(pair.src, pair.tgt, **kw)
    for _ in range(17):                     # mid-stage, Anderson history filled
        a.step()
    state = a.save_state()
    ia = a.solve(5000)
    Xa = a.transforms()
    b = nrr.Registration(pair.src, pair.tgt, **kw)
    b.load_state(state)
    i17 = b.info()
    assert i17.n_passes == 17
    ib = b.solve(5000)
    assert ib.n_passes == ia.n_passes and ib.n_solves == ia.n_solves and ib.stage == ia.stage
    assert np.array_equal(b.transforms(), Xa)
    assert ib.E == ia.E
    # a state from another problem (other sizes) is rejected
    other = synth.tiny_pair(1200, 1300, seed=92)
    c = nrr.Registration(other.src, other.tgt, **kw)
    with pytest.raises(nrr.NrrError) as e:
        c.load_state(state)                 # header names other sizes
    assert e.value.code == nrr.NRR_E_INVALID
    with pytest.raises(nrr.NrrError) as e:
        b.load_state(state[: len(state) // 2])   # short buffer
    assert e.value.code == nrr.NRR_E_INVALID
    # the same sizes but another problem: a different target, or the same
    # pair with other parameters (the header's hash differs)
    tgt2 = pair.tgt.copy()
    tgt2[:, 0] += 0.01
    d = nrr.Registration(pair.src, tgt2, **kw)
    assert (d.P, d.N) == (a.P, a.N)
    with pytest.raises(nrr.NrrError) as e:
        d.load_state(state)
    assert e.value.code == nrr.NRR_E_INVALID
    e2 = nrr.Registration(pair.src, pair.tgt, **dict(kw, k_alpha=50.0))
    with pytest.raises(nrr.NrrError) as e:
        e2.load_state(state)
    assert e.value.code == nrr.NRR_E_INVALID
    for r in (a, b, c, d, e2):
        r.close()
