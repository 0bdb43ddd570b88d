"""The allocation-free entry point nrr_align_energy_noalloc, for callers that
cannot call cudaMalloc (preallocated real-time loops, host frameworks that
own every device allocation, work issued during CUDA graph capture).

It must give the same alignment energy as the context-based path
(nrr_energy) on the same closest-point distances, on two calls in a row
(its static scratch keeps the previous call's contents), and reject sizes
beyond its fixed scratch with NRR_E_INVALID. This file is collected last so
that a failure here never hides the results of the other GPU tests.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_noalloc_align_energy_matches_context_path():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_2206_03410_gb300 import nrr
    nrr.load()
    pair = synth.tiny_pair(3000, 3300, seed=41, noise=0.003, outliers=0.05)
    reg = nrr.Registration(pair.src, pair.tgt, precision="mixed", radius=0.25, aa_m=5)
    X = synth.perturbed_transforms(reg.N, seed=5).astype(np.float32).astype(np.float64)
    terms = reg.energy(X)
    info = reg.info()
    _, d2 = reg.correspondence()          # float32 values of the mixed path, as doubles
    d2_t = torch.from_numpy(d2.astype(np.float32)).cuda()
    assert np.array_equal(d2_t.double().cpu().numpy(), d2)
    stream = torch.cuda.Stream()
    for call in range(2):
        w = torch.full_like(d2_t, -1.0)
        E = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        nrr.nrr_align_energy_noalloc(d2_t, info.nu_a, w, E, stream=stream.cuda_stream)
        stream.synchronize()
        e = float(E.cpu()[0])
        # same float terms, summed in a different order: 1e-10 relative
        assert abs(e - terms[1]) < 1e-10 * terms[1], (call, e, terms[1])
        ia = 1.0 / (2.0 * info.nu_a ** 2)
        w_ref = np.exp(-d2 * ia) * ia
        assert np.allclose(w.cpu().numpy(), w_ref, rtol=1e-5, atol=0), call
    # sizes beyond the static scratch are rejected with a clear error
    lib = nrr.load()
    code = lib.nrr_align_energy_noalloc(d2_t.data_ptr(), 33423361, info.nu_a, w.data_ptr(),
                                        E.data_ptr(), None)
    assert code == nrr.NRR_E_INVALID
    assert b"scratch" in lib.nrr_last_error(None)
    reg.close()
