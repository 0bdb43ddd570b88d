"""CPU checks of the C-ABI library: it builds, loads, exports every entry
point declared in include/nrr.h, its structs match the header's layout, and
argument validation that needs no GPU returns the documented codes."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

from paper_2206_03410_gb300 import build as B
from paper_2206_03410_gb300 import nrr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nrr.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nrr_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    path = B.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(nrr_[a-z0-9_]+)", out))
    declared = _declared()
    assert len(declared) >= 15
    missing = [s for s in declared if s not in exported]
    assert not missing, missing
    # the binding declares exactly the header's entry points
    bound = {name for name, _, _ in nrr._SIGS}
    assert bound == set(declared)


def test_struct_layout_matches_header():
    src = ('#include <stdio.h>\n#include <stddef.h>\n#include "nrr.h"\n'
           'int main(){printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(nrr_params), sizeof(nrr_step_info),'
           ' offsetof(nrr_params, pcg_max_iters), offsetof(nrr_step_info, status),'
           ' sizeof(nrr_launch_config), offsetof(nrr_params, nu_schedule));}\n')
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "p.c")
        exe = os.path.join(d, "p")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        vals = [int(x) for x in subprocess.run([exe], capture_output=True, text=True,
                                               check=True).stdout.split()]
    assert vals[0] == ctypes.sizeof(nrr.NrrParams)
    assert vals[1] == ctypes.sizeof(nrr.NrrStepInfo)
    assert vals[2] == nrr.NrrParams.pcg_max_iters.offset
    assert vals[3] == nrr.NrrStepInfo.status.offset
    assert vals[4] == ctypes.sizeof(nrr.NrrLaunchConfig)
    assert vals[5] == nrr.NrrParams.nu_schedule.offset


def test_params_default_values():
    p = nrr.params_default()
    assert p.max_influence == 8 and p.aa_m == 5 and p.max_iters_per_stage == 100
    assert p.k_alpha == 100.0 and p.k_beta == 1.0 and p.alpha < 0 and p.beta < 0
    assert p.anneal == 1 and p.precision == nrr.NRR_MIXED and p.pcg_max_iters == 500


def test_create_rejects_bad_arguments_without_gpu():
    lib = nrr.load()
    ctx = ctypes.c_void_p()
    p = nrr.params_default()
    buf = (ctypes.c_float * 30)()
    assert lib.nrr_create(None, buf, None, 10, buf, None, 10, ctypes.byref(p), None) == nrr.NRR_E_INVALID
    assert lib.nrr_create(ctypes.byref(ctx), None, None, 10, buf, None, 10, ctypes.byref(p), None) == nrr.NRR_E_INVALID
    assert lib.nrr_create(ctypes.byref(ctx), buf, None, 0, buf, None, 10, ctypes.byref(p), None) == nrr.NRR_E_INVALID
    assert lib.nrr_create(ctypes.byref(ctx), buf, None, 10, buf, None, 0, ctypes.byref(p), None) == nrr.NRR_E_INVALID
    for field, bad in [("aa_m", 9), ("max_influence", 0), ("precision", 7),
                       ("pcg_max_iters", 0), ("nu_a", float("nan"))]:
        q = nrr.params_default()
        setattr(q, field, bad)
        code = lib.nrr_create(ctypes.byref(ctx), buf, None, 10, buf, None, 10, ctypes.byref(q), None)
        assert code == nrr.NRR_E_INVALID, field
        assert lib.nrr_last_error(None)
    assert lib.nrr_step(None, None) == nrr.NRR_E_INVALID
    assert lib.nrr_solve(None, 0, None) == nrr.NRR_E_INVALID
    assert lib.nrr_energy(None, None, None) == nrr.NRR_E_INVALID


def test_unrolled_entry_points_reject_bad_arguments_without_gpu():
    lib = nrr.load()
    X = (ctypes.c_double * 12)()
    assert lib.nrr_unroll(None, 3, X, None) == nrr.NRR_E_INVALID
    assert lib.nrr_backward(None, 1, None, None, None) == nrr.NRR_E_INVALID
    assert lib.nrr_last_error(None)


def test_tuner_entry_points_reject_bad_arguments_without_gpu():
    lib = nrr.load()
    cfg = nrr.NrrLaunchConfig()
    assert lib.nrr_tune(None, None, 0, ctypes.byref(cfg)) == nrr.NRR_E_INVALID
    assert lib.nrr_batch_tune(None, None, 0, ctypes.byref(cfg)) == nrr.NRR_E_INVALID
    assert lib.nrr_get_launch_config(None, ctypes.byref(cfg)) == nrr.NRR_E_INVALID
    assert lib.nrr_set_launch_config(None, ctypes.byref(cfg)) == nrr.NRR_E_INVALID


def test_noalloc_wrapper_rejects_wrong_buffers_before_launch():
    """The binding of nrr_align_energy_noalloc passes raw device pointers, so
    it checks the buffers first: wrong dtype, too few elements or host
    memory raise ValueError and nothing reaches the library."""
    torch = pytest.importorskip("torch")
    f32 = torch.zeros(16, dtype=torch.float32)
    f64 = torch.zeros(1, dtype=torch.float64)
    cases = [
        (f32.double(), f32, f64, "float32"),            # d2 float64
        (f32, f32.double(), f64, "float32"),            # w_a float64
        (f32, f32, f64.float(), "float64"),             # E_align float32
        (f32, torch.zeros(15, dtype=torch.float32), f64, "fewer"),
        (f32, f32, torch.zeros(0, dtype=torch.float64), "one element"),
        (torch.zeros(0, dtype=torch.float32), f32, f64, "non-empty"),
        (torch.zeros(16, 2, dtype=torch.float32)[:, 0], f32, f64, "contiguous"),
        (f32, f32, f64, "CUDA"),                        # host tensors
        (f32.numpy(), f32, f64, "torch tensor"),
    ]
    for d2, w, E, msg in cases:
        with pytest.raises(ValueError, match=msg):
            nrr.nrr_align_energy_noalloc(d2, 0.1, w, E)
