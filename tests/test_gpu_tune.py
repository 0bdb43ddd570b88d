"""The autotuner (nrr_tune, nrr_batch_tune, nrr_set_launch_config) through
the C ABI: it picks valid launch shapes, restarts the solve, reuses a
tuning table, and a solve with the tuned shapes is bitwise the solve with
the same shapes set by hand."""
import os
import tempfile

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


KW = dict(radius=0.25, aa_m=5, precision="mixed", max_iters_per_stage=20)


@pytest.fixture(scope="module")
def pair():
    return synth.tiny_pair(3000, 3200, seed=41, noise=0.002, outliers=0.05)


def test_tune_picks_valid_shapes_and_restarts(pair):
    nrr = _nrr()
    reg = nrr.Registration(pair.src, pair.tgt, **KW)
    reg.step()
    cfg = reg.tune(reps=3)
    assert cfg.nn_lanes_per_query in (1, 2, 4, 8)
    assert 0 <= cfg.solve_ctas <= 16
    assert cfg.nn_ms > 0 and cfg.solve_ms > 0
    now = reg.launch_config()
    assert (now.nn_lanes_per_query, now.solve_ctas) == (cfg.nn_lanes_per_query, cfg.solve_ctas)
    assert reg.info().n_passes == 0          # restarted
    info = reg.solve(3000)
    assert info.done == 1 and info.status == 0
    X_tuned = reg.transforms()
    # the same shapes set by hand give bitwise the same solve
    other = nrr.Registration(pair.src, pair.tgt, **KW)
    other.set_launch_config(cfg.nn_lanes_per_query, cfg.solve_ctas)
    info2 = other.solve(3000)
    assert info2.n_passes == info.n_passes
    assert np.array_equal(other.transforms(), X_tuned)
    reg.close()
    other.close()


def test_tune_table_is_written_and_reused(pair):
    nrr = _nrr()
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "tune.txt")
        a = nrr.Registration(pair.src, pair.tgt, **KW)
        ca = a.tune(path, reps=2)
        lines = open(path).read().splitlines()
        assert len(lines) == 1 and lines[0].startswith("nrr-tune ")
        b = nrr.Registration(pair.src, pair.tgt, **KW)
        cb = b.tune(path, reps=2)
        assert cb.nn_ms == 0.0                      # taken from the table, not timed
        assert (cb.nn_lanes_per_query, cb.solve_ctas) == (ca.nn_lanes_per_query, ca.solve_ctas)
        assert len(open(path).read().splitlines()) == 1
        a.close()
        b.close()


def test_set_launch_config_rejects_bad_shapes(pair):
    nrr = _nrr()
    reg = nrr.Registration(pair.src, pair.tgt, **KW)
    for lpq, ctas in [(3, 1), (8, 17), (8, -2)]:
        with pytest.raises(nrr.NrrError) as e:
            reg.set_launch_config(lpq, ctas)
        assert e.value.code == nrr.NRR_E_INVALID
    reg.set_launch_config(2, 0)                     # grid-wide solve
    info = reg.solve(3000)
    assert info.done == 1 and info.status == 0
    reg.close()


def test_batch_tune():
    nrr = _nrr()
    pairs = [synth.tiny_pair(P, T, seed=60 + k, noise=0.002, outliers=0.03)
             for k, (P, T) in enumerate([(900, 1000), (2500, 2400), (400, 450)])]
    batch = nrr.BatchRegistration([(p.src, p.tgt) for p in pairs], params=KW)
    cfg = batch.tune(reps=2)
    assert cfg.nn_lanes_per_query in (2, 4, 8) and cfg.solve_ctas in (-2, -1, 0)
    assert cfg.pass_ms > 0
    infos = batch.solve(3000)
    assert all(i.done == 1 and i.status == 0 for i in infos)
    # whatever policy the tuner chose (smallest, largest or balanced
    # clusters), each pair ends bitwise where a single context with the same
    # lanes per query and cluster size ends
    for k, p in enumerate(pairs):
        c = nrr.nrr_get_launch_config(batch.context(k))
        single = nrr.Registration(p.src, p.tgt, **KW)
        single.set_launch_config(c.nn_lanes_per_query, c.solve_ctas)
        si = single.solve(3000)
        assert (si.n_passes, si.n_solves) == (infos[k].n_passes, infos[k].n_solves)
        assert np.array_equal(single.transforms(), nrr.nrr_get_transforms(batch.context(k)))
        single.close()
    batch.close()


@pytest.mark.parametrize("lpq", [8, 4, 1])
def test_search_and_solve_counters(pair, lpq, monkeypatch):
    """The opt-in per-warp search counters and the solve's phase stamps
    cover every warp a search launches, for any lanes-per-query setting,
    and leave the results unchanged."""
    nrr = _nrr()
    ref = nrr.Registration(pair.src, pair.tgt, **KW)
    ref.set_launch_config(lpq, ref.launch_config().solve_ctas)
    monkeypatch.setenv("NRR_NN_STATS", "1")
    monkeypatch.setenv("NRR_SOLVE_STATS", "1")
    reg = nrr.Registration(pair.src, pair.tgt, **KW)
    reg.set_launch_config(lpq, reg.launch_config().solve_ctas)
    for _ in range(3):
        reg.step()
        ref.step()
    assert np.array_equal(reg.transforms(), ref.transforms())
    s = nrr.nrr_get_search_stats(reg.ctx)
    per_warp = 32 // lpq
    assert s.shape == (-(-pair.P // per_warp), 4)
    assert np.all(s[:, 0] > 0)                      # every warp ran and stamped its cycles
    assert np.all(s[:, 2] >= s[:, 3])               # scanned leaves were staged first
    assert s[:, 3].sum() > 0
    if reg.launch_config().solve_ctas > 0:          # the cluster solve stamps its phases
        t = nrr.nrr_get_solve_stats(reg.ctx)
        n = int(t[63])
        assert 2 <= n < 64 and np.all(np.diff(t[:n]) >= 0)
    reg.close()
    ref.close()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_cluster_halo_matches_remote_reads(prec, monkeypatch):
    """The cluster solve reads neighbouring CTAs' z rows from halo copies
    pushed into its own shared memory; with the halo off (every such row
    read from the owner CTA) the products are summed in the same order, so
    the two runs agree bit for bit."""
    nrr = _nrr()
    pair = synth.workload("sphere5k")
    kw = dict(radius=0.15, aa_m=5, precision=prec)
    out = []
    for off in (False, True):
        if off:
            monkeypatch.setenv("NRR_NO_HALO", "1")
        reg = nrr.Registration(pair.src, pair.tgt, **kw)
        assert reg.launch_config().solve_ctas > 1
        infos = [reg.step() for _ in range(4)]
        out.append((reg.transforms(), [i.pcg_iters for i in infos]))
        reg.close()
    assert out[0][1] == out[1][1]
    assert np.array_equal(out[0][0], out[1][0])
