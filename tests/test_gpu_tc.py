"""The tensor-core candidate search (mixed path) against the exact pruned
search, through the C ABI: the closest points, their float squared
distances, the deformed source and the energy terms are bitwise equal (the
tensor cores only choose each query's candidates; the winner comes from the
same exact float keys), on the 5,000-point sphere, on ragged sizes with
duplicated targets (ties to the lowest index) and on the full-size depth
workload; whole trajectories of Algorithm 2 stay bitwise equal. The exact
search itself is checked against the FP64 oracle in test_gpu_parity.py."""
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


def _nrr():
    from paper_2206_03410_gb300 import nrr
    nrr.load()
    return nrr


def _pair(case):
    if case == "sphere5k":
        p = synth.workload("sphere5k")
        return p.src, p.tgt, dict(radius=0.15, aa_m=5)
    if case == "ragged_dup":
        p = synth.tiny_pair(1037, 613, seed=33)
        return p.src, np.concatenate([p.tgt, p.tgt]), dict(radius=0.3, aa_m=3)
    p = synth.workload("depth100k")
    kw = {k: v for k, v in p.params.items() if k not in ("precision", "iters", "unroll")}
    return p.src, p.tgt, kw


def _pair_of_contexts(nrr, case, monkeypatch=None):
    src, tgt, kw = _pair(case)
    s, t = torch.from_numpy(src).cuda(), torch.from_numpy(tgt).cuda()
    exact = nrr.Registration(s, t, precision="mixed", **kw)
    if monkeypatch is not None:
        monkeypatch.setenv("NRR_NN_STATS", "1")
    tc = nrr.Registration(s, t, precision="mixed", **kw)
    if monkeypatch is not None:
        monkeypatch.delenv("NRR_NN_STATS")
    lc = exact.launch_config()
    tc.set_launch_config(lc.nn_lanes_per_query, lc.solve_ctas, 1)
    assert tc.launch_config().nn_tensor_cores == 1 and exact.launch_config().nn_tensor_cores == 0
    return exact, tc


def _same_search(a, b):
    ra, da = a.correspondence()
    rb, db = b.correspondence()
    assert np.array_equal(ra, rb), int((ra != rb).sum())
    assert np.array_equal(da, db)
    assert np.array_equal(a.deformed(), b.deformed())


@pytest.mark.parametrize("case", ["sphere5k", "ragged_dup", "depth100k"])
def test_tc_search_bitwise_equal_to_exact(case, monkeypatch):
    nrr = _nrr()
    exact, tc = _pair_of_contexts(nrr, case, monkeypatch)
    Xs = [None, synth.perturbed_transforms(exact.N, seed=7),
          synth.perturbed_transforms(exact.N, seed=8, scale_a=0.05, scale_t=0.03)]
    for k, X in enumerate(Xs):
        if X is not None:
            X = X.astype(np.float32).astype(np.float64)
        ea = exact.energy(X)
        eb = tc.energy(X)
        assert np.array_equal(ea, eb), (case, k, ea, eb)
        _same_search(exact, tc)
    # the tensor cores did the candidate work: per CTA {cycles, candidate
    # leaves, chunks, exact fallbacks}
    stats = nrr.nrr_get_search_stats(tc.ctx)
    assert stats is not None and stats.shape[0] == (tc.P + 127) // 128
    assert stats[:, 2].sum() > 0
    if case != "ragged_dup":   # duplicated targets tie in pairs, which widens windows
        assert stats[:, 3].sum() <= 0.01 * tc.P, int(stats[:, 3].sum())
    exact.close()
    tc.close()


@pytest.mark.parametrize("case", ["sphere5k", "depth100k"])
def test_tc_trajectory_bitwise_equal_to_exact(case):
    """Passes of Algorithm 2 (closest points, energy, safeguard, assembly,
    solve, Anderson) with either search: the same iterates bit for bit."""
    nrr = _nrr()
    exact, tc = _pair_of_contexts(nrr, case)
    for k in range(12):
        ia = exact.step()
        ib = tc.step()
        assert (ia.kept, ia.stage, ia.E) == (ib.kept, ib.stage, ib.E), k
        assert np.array_equal(exact.transforms(), tc.transforms()), k
    _same_search(exact, tc)
    exact.close()
    tc.close()


def test_tc_search_needs_the_mixed_path():
    nrr = _nrr()
    p = synth.tiny_pair(500, 520, seed=2)
    reg = nrr.Registration(p.src, p.tgt, precision="fp64", radius=0.3)
    with pytest.raises(nrr.NrrError) as e:
        reg.set_launch_config(8, reg.launch_config().solve_ctas, 1)
    assert e.value.code == nrr.NRR_E_INVALID
    reg.close()
