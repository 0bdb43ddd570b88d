"""The device-side pass loop: nrr_solve and nrr_batch_solve repeat the pass
graph inside one graph launch (a conditional WHILE node whose body is one
pass and a control kernel) instead of launching it from the host. The
passes are the same kernels on the same inputs, so the iterates must be
bitwise those of the host-launched loop (NRR_HOST_LOOP=1, read when the
pass graph is captured), with the same pass counts; a cap of k passes must
run exactly k passes."""
import os

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


class _host_loop:
    def __enter__(self):
        os.environ["NRR_HOST_LOOP"] = "1"

    def __exit__(self, *a):
        os.environ.pop("NRR_HOST_LOOP", None)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_device_loop_matches_host_loop(precision):
    nrr = _nrr()
    p = synth.workload("sphere5k")
    kw = {k: v for k, v in p.params.items() if k not in ("precision", "iters")}
    kw.update(precision=precision, max_iters_per_stage=40)
    dev = nrr.Registration(p.src, p.tgt, **kw)
    with _host_loop():
        host = nrr.Registration(p.src, p.tgt, **kw)
    # a capped call first: exactly k passes, then the rest of the run
    i3 = dev.solve(3)
    with _host_loop():
        h3 = host.solve(3)
    assert i3.n_passes == 3 and h3.n_passes == 3 and not i3.done
    a = dev.solve(100000)
    with _host_loop():
        b = host.solve(100000)
    assert a.done == 1 and b.done == 1
    assert (a.n_passes, a.n_solves, a.n_rejected, a.stage) == (b.n_passes, b.n_solves, b.n_rejected, b.stage)
    assert np.array_equal(dev.transforms(), host.transforms())
    assert a.E == b.E
    # a solved context stays solved: no further pass runs
    again = dev.solve(100000)
    assert again.n_passes == a.n_passes
    dev.close()
    host.close()


def test_device_loop_batch_matches_host_loop():
    """Uneven pairs: the device loop returns to the host when half of the
    captured pairs are done, the host recaptures the rest; the pairs end
    bitwise where the host-launched batch ends them."""
    nrr = _nrr()
    pairs = [synth.tiny_pair(P, T, seed=70 + k, noise=0.002, outliers=0.03)
             for k, (P, T) in enumerate([(700, 800), (1500, 1400), (300, 350), (2100, 2300), (900, 950)])]
    kw = dict(radius=0.3, aa_m=5, precision="mixed", max_iters_per_stage=20)
    dev = nrr.BatchRegistration([(q.src, q.tgt) for q in pairs], params=kw)
    with _host_loop():
        host = nrr.BatchRegistration([(q.src, q.tgt) for q in pairs], params=kw)
    ia = dev.solve(3000)
    with _host_loop():   # the host recaptures when half of the pairs are done
        ib = host.solve(3000)
    for k in range(len(pairs)):
        assert ia[k].done == 1 and ib[k].done == 1
        assert (ia[k].n_passes, ia[k].n_solves) == (ib[k].n_passes, ib[k].n_solves)
        assert np.array_equal(nrr.nrr_get_transforms(dev.context(k)), nrr.nrr_get_transforms(host.context(k)))
    dev.close()
    host.close()


def test_device_loop_batch_cap():
    """A batch call capped at k passes runs k passes of every running pair."""
    nrr = _nrr()
    pairs = [synth.tiny_pair(P, T, seed=90 + k, noise=0.002, outliers=0.03)
             for k, (P, T) in enumerate([(600, 650), (1200, 1300)])]
    kw = dict(radius=0.3, aa_m=5, precision="mixed", max_iters_per_stage=20)
    b = nrr.BatchRegistration([(q.src, q.tgt) for q in pairs], params=kw)
    infos = b.solve(4)
    for k in range(len(pairs)):
        assert infos[k].n_passes == 4 and not infos[k].done
    b.close()


def test_device_loop_history_matches_steps():
    """nrr_get_history returns, pass by pass, the state nrr_step reports for
    the same passes (recorded on the device by the loop's control kernel);
    a capped call records only its own passes, the host-launched loop none."""
    nrr = _nrr()
    p = synth.workload("sphere5k")
    kw = {k: v for k, v in p.params.items() if k not in ("precision", "iters")}
    kw.update(precision="mixed", max_iters_per_stage=30)
    a = nrr.Registration(p.src, p.tgt, **kw)
    info = a.solve(100000)
    hist = a.history()
    # one record per pass the loop ran: the counted passes, then the pass
    # whose stopping test returns (done, not counted)
    assert info.done == 1 and len(hist) == info.n_passes + 1
    assert hist[-1].done == 1 and all(h.done == 0 for h in hist[:-1])
    b = nrr.Registration(p.src, p.tgt, **kw)
    for k, h in enumerate(hist):
        s = b.step()
        assert h.as_dict() == s.as_dict(), k
    assert hist[-1].as_dict() == info.as_dict()
    a.reset()
    a.solve(5)
    h5 = a.history()
    assert [h.n_passes for h in h5] == [1, 2, 3, 4, 5]
    with _host_loop():
        c = nrr.Registration(p.src, p.tgt, **kw)
        c.solve(5)
    assert c.history() == []
    a.close()
    b.close()
    c.close()


def test_batch_create_parallel_contexts():
    """nrr_batch_create builds the pairs' contexts on several host threads:
    each pair's graph is the one a single context builds (also with the
    graph on the GPU, several constructions then sharing the device), and
    a bad pair is reported with the lowest failing index."""
    nrr = _nrr()
    pairs = [synth.tiny_pair(P, T, seed=110 + k, noise=0.002, outliers=0.03)
             for k, (P, T) in enumerate([(800, 900), (1600, 1500), (500, 520), (1200, 1250),
                                         (2000, 2100), (700, 760), (1000, 980), (1400, 1450),
                                         (600, 640)])]
    for on_gpu in (0, 1):
        kw = dict(radius=0.3, aa_m=5, precision="mixed", graph_on_gpu=on_gpu)
        b = nrr.BatchRegistration([(q.src, q.tgt) for q in pairs], params=kw)
        for k, q in enumerate(pairs):
            single = nrr.Registration(q.src, q.tgt, **kw)
            gb, gs = nrr.nrr_get_graph(b.context(k)), single.graph()
            assert np.array_equal(gb.nodes, gs.nodes) and np.array_equal(gb.edges, gs.edges)
            assert np.array_equal(gb.nidx, gs.nidx) and np.array_equal(gb.w, gs.w)
            assert np.array_equal(gb.r, gs.r)
            single.close()
        b.close()
    bad = [(q.src.copy(), q.tgt) for q in pairs]
    bad[5][0][3, 1] = np.nan
    bad[7][0][0, 0] = np.inf
    with pytest.raises(nrr.NrrError) as e:
        nrr.BatchRegistration(bad, params=dict(radius=0.3, aa_m=5, precision="mixed"))
    assert e.value.code == nrr.NRR_E_INVALID
    assert "pair 5" in str(e.value)
