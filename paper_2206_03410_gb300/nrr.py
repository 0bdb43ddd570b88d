"""ctypes binding of libnrr (include/nrr.h).

Argument marshalling only: every computation of the registration runs in the
library's CUDA kernels. The functions keep the C names (``nrr_create``,
``nrr_step``, ``nrr_solve``, ``nrr_energy``, ``nrr_backward`` ...); the
``Registration`` class is a thin owner of one context.

Inputs may be numpy arrays (host) or torch tensors (host or CUDA); outputs
are returned as numpy arrays. The library is loaded from the in-tree build
(``_build/libnrr.so``); if it cannot be built or loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

NRR_OK = 0
NRR_E_INVALID = 1
NRR_E_CUDA = 2
NRR_E_OOM = 3
NRR_E_SINGULAR = 4
NRR_E_TIMEOUT = 5
NRR_E_NOT_CONVERGED = 6
NRR_E_STATE = 7

NRR_FP64 = 0
NRR_MIXED = 1
ROBUST = {"welsch": 0, "l2": 1, "l2r": 2}
NU_SCHEDULE = {"": 0, "anneal": 0, "max": 1, "min": 2, "med": 3}


class NrrParams(ctypes.Structure):
    _fields_ = [
        ("graph_radius", ctypes.c_double),
        ("max_influence", ctypes.c_int),
        ("nu_a", ctypes.c_double),
        ("nu_r", ctypes.c_double),
        ("nu_a_min", ctypes.c_double),
        ("anneal", ctypes.c_int),
        ("k_alpha", ctypes.c_double),
        ("k_beta", ctypes.c_double),
        ("alpha", ctypes.c_double),
        ("beta", ctypes.c_double),
        ("aa_m", ctypes.c_int),
        ("max_iters_per_stage", ctypes.c_int),
        ("max_total_passes", ctypes.c_int),
        ("eps", ctypes.c_double),
        ("rel_energy_tol", ctypes.c_double),
        ("precision", ctypes.c_int),
        ("pcg_tol", ctypes.c_double),
        ("pcg_max_iters", ctypes.c_int),
        ("solve_ctas", ctypes.c_int),
        ("robust", ctypes.c_int),
        ("nu_schedule", ctypes.c_int),
        ("graph_on_gpu", ctypes.c_int),
        ("src_faces", ctypes.c_void_p),
        ("n_src_faces", ctypes.c_int64),
    ]


class NrrLbfgsParams(ctypes.Structure):
    _fields_ = [
        ("m", ctypes.c_int),
        ("c1", ctypes.c_double),
        ("g_tol", ctypes.c_double),
        ("max_inner", ctypes.c_int),
        ("max_halvings", ctypes.c_int),
    ]


class NrrLaunchConfig(ctypes.Structure):
    _fields_ = [
        ("nn_lanes_per_query", ctypes.c_int),
        ("solve_ctas", ctypes.c_int),
        ("nn_ms", ctypes.c_double),
        ("solve_ms", ctypes.c_double),
        ("pass_ms", ctypes.c_double),
        ("launches_per_pass", ctypes.c_int),
        ("nn_tensor_cores", ctypes.c_int),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class NrrStepInfo(ctypes.Structure):
    _fields_ = [
        ("E", ctypes.c_double),
        ("E_align", ctypes.c_double),
        ("E_reg", ctypes.c_double),
        ("E_rot", ctypes.c_double),
        ("nu_a", ctypes.c_double),
        ("nu_r", ctypes.c_double),
        ("alpha", ctypes.c_double),
        ("beta", ctypes.c_double),
        ("max_disp", ctypes.c_double),
        ("pcg_rel_residual", ctypes.c_double),
        ("kept", ctypes.c_int),
        ("solved", ctypes.c_int),
        ("stage", ctypes.c_int),
        ("done", ctypes.c_int),
        ("pcg_iters", ctypes.c_int),
        ("aa_mk", ctypes.c_int),
        ("n_passes", ctypes.c_int),
        ("n_solves", ctypes.c_int),
        ("n_rejected", ctypes.c_int),
        ("status", ctypes.c_int),
        ("warning", ctypes.c_int),
        ("n_singular", ctypes.c_int),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


# (name, restype, argtypes) of every entry point declared in include/nrr.h
_VP = ctypes.c_void_p
_I64 = ctypes.c_int64
_SIGS = [
    ("nrr_params_default", None, [ctypes.POINTER(NrrParams)]),
    ("nrr_create", ctypes.c_int, [ctypes.POINTER(_VP), _VP, _VP, _I64, _VP, _VP, _I64,
                                  ctypes.POINTER(NrrParams), _VP]),
    ("nrr_destroy", None, [_VP]),
    ("nrr_step", ctypes.c_int, [_VP, ctypes.POINTER(NrrStepInfo)]),
    ("nrr_solve", ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(NrrStepInfo)]),
    ("nrr_enqueue_passes", ctypes.c_int, [_VP, ctypes.c_int]),
    ("nrr_reset", ctypes.c_int, [_VP]),
    ("nrr_time_kernels", ctypes.c_int, [_VP, ctypes.c_int, _VP]),
    ("nrr_energy", ctypes.c_int, [_VP, _VP, _VP]),
    ("nrr_backward", ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, _VP]),
    ("nrr_unroll", ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP]),
    ("nrr_get_state_size", ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_size_t)]),
    ("nrr_save_state", ctypes.c_int, [_VP, _VP, ctypes.c_size_t]),
    ("nrr_load_state", ctypes.c_int, [_VP, _VP, ctypes.c_size_t]),
    ("nrr_set_transforms", ctypes.c_int, [_VP, _VP]),
    ("nrr_set_stage", ctypes.c_int, [_VP, ctypes.c_double, ctypes.c_double]),
    ("nrr_get_transforms", ctypes.c_int, [_VP, _VP]),
    ("nrr_get_deformed", ctypes.c_int, [_VP, _VP]),
    ("nrr_get_correspondence", ctypes.c_int, [_VP, _VP, _VP]),
    ("nrr_get_sizes", ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP]),
    ("nrr_get_graph", ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    ("nrr_graph_build", ctypes.c_int, [ctypes.POINTER(_VP), _VP, _I64, ctypes.c_double, ctypes.c_int]),
    ("nrr_graph_build_gpu", ctypes.c_int, [ctypes.POINTER(_VP), _VP, _I64, ctypes.c_double, ctypes.c_int, _VP]),
    ("nrr_graph_build_mesh", ctypes.c_int, [ctypes.POINTER(_VP), _VP, _I64, _VP, _I64, ctypes.c_double,
                                             ctypes.c_int]),
    ("nrr_graph_sizes", ctypes.c_int, [_VP, _VP, _VP, _VP, _VP]),
    ("nrr_graph_get", ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    ("nrr_graph_destroy", None, [_VP]),
    ("nrr_get_system", ctypes.c_int, [_VP, _VP, _VP]),
    ("nrr_get_mm_solution", ctypes.c_int, [_VP, _VP]),
    ("nrr_get_info", ctypes.c_int, [_VP, ctypes.POINTER(NrrStepInfo)]),
    ("nrr_get_history", ctypes.c_int, [_VP, _VP, ctypes.c_int, _VP]),
    ("nrr_get_search_stats", ctypes.c_int, [_VP, _VP, _I64, _VP]),
    ("nrr_get_solve_stats", ctypes.c_int, [_VP, _VP]),
    ("nrr_align_energy_noalloc", ctypes.c_int, [_VP, _I64, ctypes.c_double, _VP, _VP, _VP]),
    ("nrr_batch_create", ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_int, _VP, _VP, _VP, _VP, _VP,
                                        ctypes.c_int, _VP]),
    ("nrr_batch_solve", ctypes.c_int, [_VP, ctypes.c_int, _VP]),
    ("nrr_batch_reset", ctypes.c_int, [_VP]),
    ("nrr_batch_get_context", ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(_VP)]),
    ("nrr_batch_destroy", None, [_VP]),
    ("nrr_get_launch_config", ctypes.c_int, [_VP, ctypes.POINTER(NrrLaunchConfig)]),
    ("nrr_set_launch_config", ctypes.c_int, [_VP, ctypes.POINTER(NrrLaunchConfig)]),
    ("nrr_tune", ctypes.c_int, [_VP, ctypes.c_char_p, ctypes.c_int, ctypes.POINTER(NrrLaunchConfig)]),
    ("nrr_batch_tune", ctypes.c_int, [_VP, ctypes.c_char_p, ctypes.c_int, ctypes.POINTER(NrrLaunchConfig)]),
    ("nrr_lbfgs_params_default", None, [ctypes.POINTER(NrrLbfgsParams)]),
    ("nrr_solve_lbfgs", ctypes.c_int, [_VP, ctypes.POINTER(NrrLbfgsParams), ctypes.c_int,
                                       ctypes.POINTER(NrrStepInfo)]),
    ("nrr_last_error", ctypes.c_char_p, [_VP]),
]

_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Loads libnrr.so (building it first if needed). Raises on failure."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libnrr.so not found at {path}")
    lib = ctypes.CDLL(path)
    for name, res, args in _SIGS:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class NrrError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"nrr error {code}: {msg}")
        self.code = code


def _check(code: int, ctx=None, ok=(NRR_OK,)):
    if code not in ok:
        msg = load().nrr_last_error(ctx)
        raise NrrError(code, msg.decode() if msg else "")
    return code


def _ptr(a):
    """Device or host pointer of a numpy array or torch tensor (contiguous)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous()
        return a.data_ptr()
    raise TypeError(type(a))


def params_default() -> NrrParams:
    p = NrrParams()
    load().nrr_params_default(ctypes.byref(p))
    return p


def make_params(**kw) -> NrrParams:
    p = params_default()
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = NRR_FP64 if v.lower() == "fp64" else NRR_MIXED
        if k == "robust" and isinstance(v, str):
            v = ROBUST[v]
        if k in ("nu_fixed", "nu_schedule"):
            k = "nu_schedule"
            if isinstance(v, str):
                v = NU_SCHEDULE[v]
        if k in ("radius",):
            k = "graph_radius"
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


# ---------------------------------------------------------------------------
# C-named wrappers
# ---------------------------------------------------------------------------

def nrr_create(src, tgt, params: NrrParams, src_nrm=None, tgt_nrm=None, stream=None):
    lib = load()
    ctx = _VP()
    P = int(src.shape[0])
    T = int(tgt.shape[0])
    _check(lib.nrr_create(ctypes.byref(ctx), _ptr(src), _ptr(src_nrm), P, _ptr(tgt),
                          _ptr(tgt_nrm), T, ctypes.byref(params), stream))
    return ctx


def nrr_destroy(ctx):
    load().nrr_destroy(ctx)


def nrr_step(ctx) -> NrrStepInfo:
    info = NrrStepInfo()
    _check(load().nrr_step(ctx, ctypes.byref(info)), ctx)
    return info


def nrr_solve(ctx, max_passes: int = 0) -> NrrStepInfo:
    info = NrrStepInfo()
    _check(load().nrr_solve(ctx, int(max_passes), ctypes.byref(info)), ctx,
           ok=(NRR_OK, NRR_E_NOT_CONVERGED))
    return info


def nrr_solve_lbfgs(ctx, max_outer: int = 0, **lbfgs) -> NrrStepInfo:
    """The preliminary version's solver (fixed closest points + inner
    L-BFGS) from the current state; keyword arguments override the fields of
    nrr_lbfgs_params (m, c1, g_tol, max_inner, max_halvings)."""
    p = NrrLbfgsParams()
    load().nrr_lbfgs_params_default(ctypes.byref(p))
    for k, v in lbfgs.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    info = NrrStepInfo()
    _check(load().nrr_solve_lbfgs(ctx, ctypes.byref(p), int(max_outer), ctypes.byref(info)), ctx,
           ok=(NRR_OK, NRR_E_NOT_CONVERGED))
    return info


def nrr_enqueue_passes(ctx, n: int):
    _check(load().nrr_enqueue_passes(ctx, int(n)), ctx)


def nrr_reset(ctx):
    _check(load().nrr_reset(ctx), ctx)


# the steps of a pass in launch order; "solve_kernel" is the PCG solve and
# the free-translation kernel after it, the last is two kernels
# (aa_dots_kernel, aa_mix_kernel)
KERNELS = ("nn_kernel", "xterm_kernel", "energy_kernel", "assemble_kernel", "solve_kernel", "aa_kernels")


def nrr_time_kernels(ctx, n: int = 1) -> np.ndarray:
    """Milliseconds spent in each step of a pass (KERNELS), summed over n
    passes (event-timed on the context's stream)."""
    out = np.zeros(len(KERNELS), dtype=np.float64)
    _check(load().nrr_time_kernels(ctx, int(n), _ptr(out)), ctx)
    return out


def nrr_energy(ctx, X=None) -> np.ndarray:
    out = np.zeros(4, dtype=np.float64)
    Xa = None if X is None else np.ascontiguousarray(X, dtype=np.float64)
    _check(load().nrr_energy(ctx, _ptr(Xa), _ptr(out)), ctx)
    return out


def nrr_backward(ctx, X=None, mode: int = 0, want_src: bool = True):
    P, _, N, _, _ = nrr_get_sizes(ctx)
    gX = np.zeros((N, 12), dtype=np.float64)
    gv = np.zeros((P, 3), dtype=np.float64) if want_src else None
    Xa = None if X is None else np.ascontiguousarray(X, dtype=np.float64)
    _check(load().nrr_backward(ctx, int(mode), _ptr(Xa), _ptr(gX), _ptr(gv)), ctx)
    return gX, gv


def nrr_unroll(ctx, K: int, X0):
    """K plain MM steps from X0 (checkpoints kept for nrr_backward mode 1);
    returns X^(K) [N, 12] float64."""
    _, _, N, _, _ = nrr_get_sizes(ctx)
    X0a = np.ascontiguousarray(X0, dtype=np.float64)
    XK = np.zeros((N, 12), dtype=np.float64)
    _check(load().nrr_unroll(ctx, int(K), _ptr(X0a), _ptr(XK)), ctx)
    return XK


def nrr_save_state(ctx) -> bytes:
    """Checkpoint of the solve (see nrr_save_state in nrr.h)."""
    n = ctypes.c_size_t()
    _check(load().nrr_get_state_size(ctx, ctypes.byref(n)), ctx)
    buf = (ctypes.c_ubyte * n.value)()
    _check(load().nrr_save_state(ctx, ctypes.cast(buf, _VP), n), ctx)
    return bytes(buf)


def nrr_load_state(ctx, state: bytes):
    buf = (ctypes.c_ubyte * len(state)).from_buffer_copy(state)
    _check(load().nrr_load_state(ctx, ctypes.cast(buf, _VP), len(state)), ctx)


def nrr_get_launch_config(ctx) -> NrrLaunchConfig:
    out = NrrLaunchConfig()
    _check(load().nrr_get_launch_config(ctx, ctypes.byref(out)), ctx)
    return out


def nrr_set_launch_config(ctx, nn_lanes_per_query: int, solve_ctas: int, nn_tensor_cores: int = 0):
    cfg = NrrLaunchConfig(nn_lanes_per_query=int(nn_lanes_per_query), solve_ctas=int(solve_ctas),
                          nn_tensor_cores=int(nn_tensor_cores))
    _check(load().nrr_set_launch_config(ctx, ctypes.byref(cfg)), ctx)


def nrr_tune(ctx, table: str | None = None, reps: int = 0) -> NrrLaunchConfig:
    out = NrrLaunchConfig()
    path = table.encode() if table else None
    _check(load().nrr_tune(ctx, path, int(reps), ctypes.byref(out)), ctx)
    return out


def nrr_batch_tune(batch, table: str | None = None, reps: int = 0) -> NrrLaunchConfig:
    out = NrrLaunchConfig()
    path = table.encode() if table else None
    _check(load().nrr_batch_tune(batch, path, int(reps), ctypes.byref(out)))
    return out


def nrr_align_energy_noalloc(d2, nu_a: float, w_a, E_align, stream=None):
    """Allocation-free alignment energy and surrogate weights. d2, w_a:
    float32 CUDA tensors [P] (w_a at least P elements); E_align: float64
    CUDA tensor with at least one element; all three contiguous and on the
    same device. Enqueues on ``stream`` (raw cudaStream_t, None = legacy
    default stream). Buffers of the wrong kind raise ValueError before
    anything is launched: the library reads and writes them as raw device
    pointers."""
    import torch
    bufs = {"d2": d2, "w_a": w_a, "E_align": E_align}
    for name, t in bufs.items():
        if not isinstance(t, torch.Tensor):
            raise ValueError(f"{name} must be a torch tensor")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    if d2.dtype != torch.float32 or w_a.dtype != torch.float32:
        raise ValueError("d2 and w_a must be float32")
    if E_align.dtype != torch.float64:
        raise ValueError("E_align must be float64")
    if d2.dim() != 1 or d2.numel() < 1:
        raise ValueError("d2 must be a non-empty 1-D tensor [P]")
    P = int(d2.numel())
    if w_a.numel() < P:
        raise ValueError(f"w_a holds {w_a.numel()} elements, fewer than P = {P}")
    if E_align.numel() < 1:
        raise ValueError("E_align must hold one element")
    for name, t in bufs.items():
        if not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
    if not (d2.device == w_a.device == E_align.device):
        raise ValueError("d2, w_a and E_align must be on the same device")
    _check(load().nrr_align_energy_noalloc(_ptr(d2), P, float(nu_a), _ptr(w_a), _ptr(E_align), stream))


def nrr_set_transforms(ctx, X):
    Xa = np.ascontiguousarray(X, dtype=np.float64)
    _check(load().nrr_set_transforms(ctx, _ptr(Xa)), ctx)


def nrr_set_stage(ctx, nu_a: float, nu_r: float):
    _check(load().nrr_set_stage(ctx, float(nu_a), float(nu_r)), ctx)


def nrr_get_sizes(ctx):
    P, T, N, E = (ctypes.c_int64() for _ in range(4))
    K = ctypes.c_int32()
    _check(load().nrr_get_sizes(ctx, ctypes.byref(P), ctypes.byref(T), ctypes.byref(N),
                                ctypes.byref(E), ctypes.byref(K)), ctx)
    return P.value, T.value, N.value, E.value, K.value


def nrr_get_transforms(ctx) -> np.ndarray:
    _, _, N, _, _ = nrr_get_sizes(ctx)
    X = np.zeros((N, 12), dtype=np.float64)
    _check(load().nrr_get_transforms(ctx, _ptr(X)), ctx)
    return X


def nrr_get_mm_solution(ctx) -> np.ndarray:
    _, _, N, _, _ = nrr_get_sizes(ctx)
    X = np.zeros((N, 12), dtype=np.float64)
    _check(load().nrr_get_mm_solution(ctx, _ptr(X)), ctx)
    return X


def nrr_get_deformed(ctx) -> np.ndarray:
    P, _, _, _, _ = nrr_get_sizes(ctx)
    v = np.zeros((P, 3), dtype=np.float64)
    _check(load().nrr_get_deformed(ctx, _ptr(v)), ctx)
    return v


def nrr_get_correspondence(ctx):
    P, _, _, _, _ = nrr_get_sizes(ctx)
    rho = np.zeros(P, dtype=np.int32)
    d2 = np.zeros(P, dtype=np.float64)
    _check(load().nrr_get_correspondence(ctx, _ptr(rho), _ptr(d2)), ctx)
    return rho, d2


@dataclass
class GraphView:
    nodes: np.ndarray
    nidx: np.ndarray
    w: np.ndarray
    edges: np.ndarray
    r: np.ndarray
    lbar: float


def nrr_get_graph(ctx) -> GraphView:
    P, _, N, E, K = nrr_get_sizes(ctx)
    nodes = np.zeros(N, dtype=np.int32)
    nidx = np.zeros((P, K), dtype=np.int32)
    w = np.zeros((P, K), dtype=np.float64)
    edges = np.zeros((E, 2), dtype=np.int32)
    r = np.zeros(2 * E, dtype=np.float64)
    lbar = ctypes.c_double()
    _check(load().nrr_get_graph(ctx, _ptr(nodes), _ptr(nidx), _ptr(w), _ptr(edges), _ptr(r),
                                ctypes.byref(lbar)), ctx)
    return GraphView(nodes, nidx, w, edges, r, lbar.value)


def _faces_array(faces) -> np.ndarray:
    F = np.ascontiguousarray(np.asarray(faces, dtype=np.int32))
    if F.ndim != 2 or F.shape[1] != 3 or F.shape[0] < 1:
        raise ValueError("faces must be [n_faces, 3] with n_faces >= 1")
    return F


def build_graph(src, radius: float = 0.0, max_influence: int = 0, on_gpu: bool = False,
                stream=None, faces=None) -> GraphView:
    """The deformation graph of the source points src [P,3] (Algorithm 1,
    Sec. 3.1-3.2): the graph nrr_create would build with the same radius
    (<= 0: 5 lbar) and influence cap (<= 0: 8), built by the library on the
    host (nrr_graph_build, no GPU needed) or on the GPU
    (nrr_graph_build_gpu); with ``faces`` [n,3] the source is a triangle
    mesh and D is the exact geodesic distance (nrr_graph_build_mesh, host)."""
    lib = load()
    g = _VP()
    if faces is not None:
        if on_gpu:
            raise ValueError("a mesh graph is built on the host (on_gpu must be False)")
        v = np.ascontiguousarray(np.asarray(src, dtype=np.float32))
        if v.ndim != 2 or v.shape[1] != 3:
            raise ValueError("src must be [P, 3]")
        P = int(v.shape[0])
        F = _faces_array(faces)
        _check(lib.nrr_graph_build_mesh(ctypes.byref(g), _ptr(v), P, _ptr(F), int(F.shape[0]), float(radius),
                                        int(max_influence)))
    elif on_gpu and hasattr(src, "data_ptr"):
        v = src.contiguous()
        P = int(v.shape[0])
        _check(lib.nrr_graph_build_gpu(ctypes.byref(g), _ptr(v), P, float(radius), int(max_influence), stream))
    else:
        v = np.ascontiguousarray(np.asarray(src, dtype=np.float32))
        if v.ndim != 2 or v.shape[1] != 3:
            raise ValueError("src must be [P, 3]")
        P = int(v.shape[0])
        if on_gpu:
            _check(lib.nrr_graph_build_gpu(ctypes.byref(g), _ptr(v), P, float(radius), int(max_influence), stream))
        else:
            _check(lib.nrr_graph_build(ctypes.byref(g), _ptr(v), P, float(radius), int(max_influence)))
    try:
        N, E, K = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        R = ctypes.c_double()
        _check(lib.nrr_graph_sizes(g, ctypes.byref(N), ctypes.byref(E), ctypes.byref(K), ctypes.byref(R)))
        nodes = np.zeros(N.value, dtype=np.int32)
        nidx = np.zeros((P, K.value), dtype=np.int32)
        w = np.zeros((P, K.value), dtype=np.float64)
        edges = np.zeros((E.value, 2), dtype=np.int32)
        r = np.zeros(2 * E.value, dtype=np.float64)
        lbar = ctypes.c_double()
        _check(lib.nrr_graph_get(g, _ptr(nodes), _ptr(nidx), _ptr(w), _ptr(edges), _ptr(r), ctypes.byref(lbar)))
    finally:
        lib.nrr_graph_destroy(g)
    return GraphView(nodes, nidx, w, edges, r, lbar.value)


def nrr_get_system(ctx, dense: bool = True):
    _, _, N, _, _ = nrr_get_sizes(ctx)
    K = np.zeros((4 * N, 4 * N), dtype=np.float64) if dense else None
    B = np.zeros((4 * N, 3), dtype=np.float64)
    _check(load().nrr_get_system(ctx, _ptr(K), _ptr(B)), ctx)
    return K, B


def nrr_get_search_stats(ctx):
    """Per-warp counters of the last closest-point search ([warps, 4]:
    cycles, super tiles, leaves staged, leaves scanned) or None."""
    n = ctypes.c_int64()
    _check(load().nrr_get_search_stats(ctx, None, 0, ctypes.byref(n)), ctx)
    if n.value == 0:
        return None
    out = np.zeros((n.value, 4), dtype=np.uint64)
    _check(load().nrr_get_search_stats(ctx, _ptr(out), n.value, ctypes.byref(n)), ctx)
    return out


def nrr_get_solve_stats(ctx) -> np.ndarray:
    out = np.zeros(64, dtype=np.int64)
    _check(load().nrr_get_solve_stats(ctx, _ptr(out)), ctx)
    return out


def nrr_get_info(ctx) -> NrrStepInfo:
    info = NrrStepInfo()
    _check(load().nrr_get_info(ctx, ctypes.byref(info)), ctx)
    return info


def nrr_get_history(ctx) -> list:
    """Per-pass records (NrrStepInfo) of the last nrr_solve call."""
    lib = load()
    n = ctypes.c_int()
    _check(lib.nrr_get_history(ctx, None, 0, ctypes.byref(n)), ctx)
    recs = (NrrStepInfo * max(n.value, 1))()
    got = ctypes.c_int()
    _check(lib.nrr_get_history(ctx, ctypes.cast(recs, ctypes.c_void_p), n.value, ctypes.byref(got)), ctx)
    return list(recs)[:got.value]


class Registration:
    """Owner of one nrr context.

    >>> reg = Registration(src, tgt, precision="fp64", radius=0.15)
    >>> info = reg.solve()
    >>> X = reg.transforms()
    """

    def __init__(self, src, tgt, src_nrm=None, tgt_nrm=None, stream=None, faces=None, **params):
        self._p = make_params(**params)
        F = None
        if faces is not None:
            # a triangle-mesh source: geodesic influence (host int32 faces)
            F = _faces_array(faces)
            self._p.src_faces = F.ctypes.data
            self._p.n_src_faces = int(F.shape[0])
        self._keep = (src, tgt, src_nrm, tgt_nrm, F)
        self.ctx = nrr_create(src, tgt, self._p, src_nrm, tgt_nrm, stream)
        self.P, self.T, self.N, self.n_edges, self.K = nrr_get_sizes(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            nrr_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def step(self) -> NrrStepInfo:
        return nrr_step(self.ctx)

    def solve(self, max_passes: int = 0) -> NrrStepInfo:
        return nrr_solve(self.ctx, max_passes)

    def solve_lbfgs(self, max_outer: int = 0, **lbfgs) -> NrrStepInfo:
        return nrr_solve_lbfgs(self.ctx, max_outer, **lbfgs)

    def enqueue_passes(self, n: int):
        nrr_enqueue_passes(self.ctx, n)

    def reset(self):
        nrr_reset(self.ctx)

    def time_kernels(self, n: int = 1) -> np.ndarray:
        return nrr_time_kernels(self.ctx, n)

    def energy(self, X=None) -> np.ndarray:
        return nrr_energy(self.ctx, X)

    def backward(self, X=None, want_src: bool = True):
        return nrr_backward(self.ctx, X, 0, want_src)

    def save_state(self) -> bytes:
        return nrr_save_state(self.ctx)

    def load_state(self, state: bytes):
        nrr_load_state(self.ctx, state)

    def tune(self, table: str | None = None, reps: int = 0) -> NrrLaunchConfig:
        """Autotunes the launch shapes on this problem (restarts the solve)."""
        return nrr_tune(self.ctx, table, reps)

    def launch_config(self) -> NrrLaunchConfig:
        return nrr_get_launch_config(self.ctx)

    def set_launch_config(self, nn_lanes_per_query: int, solve_ctas: int, nn_tensor_cores: int = 0):
        nrr_set_launch_config(self.ctx, nn_lanes_per_query, solve_ctas, nn_tensor_cores)

    def unroll(self, K: int, X0) -> np.ndarray:
        return nrr_unroll(self.ctx, K, X0)

    def unrolled_backward(self, cotangent=None, want_src: bool = True):
        """dL/dX^(0), dL/dv of the last unroll; cotangent = dL/dX^(K) or
        None for L = E(X^(K))."""
        return nrr_backward(self.ctx, cotangent, 1, want_src)

    def set_transforms(self, X):
        nrr_set_transforms(self.ctx, X)

    def set_stage(self, nu_a, nu_r):
        nrr_set_stage(self.ctx, nu_a, nu_r)

    def transforms(self) -> np.ndarray:
        return nrr_get_transforms(self.ctx)

    def mm_solution(self) -> np.ndarray:
        return nrr_get_mm_solution(self.ctx)

    def deformed(self) -> np.ndarray:
        return nrr_get_deformed(self.ctx)

    def correspondence(self):
        return nrr_get_correspondence(self.ctx)

    def graph(self) -> GraphView:
        return nrr_get_graph(self.ctx)

    def system(self, dense: bool = True):
        return nrr_get_system(self.ctx, dense)

    def info(self) -> NrrStepInfo:
        return nrr_get_info(self.ctx)

    def history(self) -> list:
        """Per-pass records of the last solve() (device-side loop)."""
        return nrr_get_history(self.ctx)


def energy_function():
    """torch.autograd.Function computing E(X) of a registration with the
    hand-written gradient kernel as its backward (closest points held at X).

    Usage: E = energy_function().apply(X, reg) with X a float64 tensor
    [N, 12] (requires_grad) and reg a Registration; E.backward() fills
    X.grad with dE/dX from nrr_backward. Imported lazily so that the binding
    itself does not need torch."""
    import torch

    class NrrEnergy(torch.autograd.Function):
        @staticmethod
        def forward(ctx, X, reg):
            Xh = X.detach().cpu().numpy().astype(np.float64)
            ctx.reg = reg
            ctx.Xh = Xh
            e = reg.energy(Xh)
            return torch.tensor(e[0], dtype=X.dtype, device=X.device)

        @staticmethod
        def backward(ctx, grad_out):
            gX, _ = ctx.reg.backward(ctx.Xh, want_src=False)
            g = torch.from_numpy(gX).to(device=grad_out.device, dtype=grad_out.dtype)
            return grad_out * g, None

    return NrrEnergy


def unrolled_function():
    """torch.autograd.Function for K unrolled MM steps: XK = fn.apply(X0, src,
    reg, K) runs nrr_unroll from X0 [N, 12] (float64 tensor) and returns
    X^(K); its backward calls nrr_backward mode 1 with the incoming gradient
    as the cotangent and returns dL/dX0 and dL/dsrc. ``src`` [P, 3] must be
    the source the registration was created from (it carries the source
    gradient; the library uses its own copy). Imported lazily so that the
    binding itself does not need torch."""
    import torch

    class NrrUnrolled(torch.autograd.Function):
        @staticmethod
        def forward(ctx, X0, src, reg, K):
            ctx.reg = reg
            ctx.src_meta = (src.dtype, src.device)
            XK = reg.unroll(int(K), X0.detach().cpu().numpy().astype(np.float64))
            return torch.from_numpy(XK).to(device=X0.device, dtype=X0.dtype)

        @staticmethod
        def backward(ctx, grad_out):
            C = grad_out.detach().cpu().numpy().astype(np.float64)
            gX, gv = ctx.reg.unrolled_backward(np.ascontiguousarray(C))
            dt, dev = ctx.src_meta
            return (torch.from_numpy(gX).to(device=grad_out.device, dtype=grad_out.dtype),
                    torch.from_numpy(gv).to(device=dev, dtype=dt), None, None)

    return NrrUnrolled


class BatchRegistration:
    """Independent pairs advanced together by one CUDA-graph launch per pass
    (nrr_batch_*). ``pairs`` is a list of (src, tgt) arrays; ``params`` a
    dict applied to every pair or a list of dicts, one per pair."""

    def __init__(self, pairs, params=None, stream=None):
        lib = load()
        n = len(pairs)
        self._keep = [(np.ascontiguousarray(s, dtype=np.float32) if isinstance(s, np.ndarray) else s,
                       np.ascontiguousarray(t, dtype=np.float32) if isinstance(t, np.ndarray) else t)
                      for s, t in pairs]
        srcp = (_VP * n)(*[_ptr(s) for s, _ in self._keep])
        tgtp = (_VP * n)(*[_ptr(t) for _, t in self._keep])
        P = (ctypes.c_int64 * n)(*[int(s.shape[0]) for s, _ in self._keep])
        T = (ctypes.c_int64 * n)(*[int(t.shape[0]) for _, t in self._keep])
        if params is None:
            pp, per = None, 0
        elif isinstance(params, dict):
            pp, per = ctypes.byref(make_params(**params)), 0
        else:
            arr = (NrrParams * n)(*[make_params(**p) for p in params])
            pp, per = arr, 1
            self._params = arr
        self.b = _VP()
        _check(lib.nrr_batch_create(ctypes.byref(self.b), n, srcp, P, tgtp, T, pp, per, stream))
        self.n = n

    def solve(self, max_passes: int = 0):
        infos = (NrrStepInfo * self.n)()
        _check(load().nrr_batch_solve(self.b, int(max_passes), infos), None,
               ok=(NRR_OK, NRR_E_NOT_CONVERGED))
        return list(infos)

    def reset(self):
        _check(load().nrr_batch_reset(self.b))

    def tune(self, table: str | None = None, reps: int = 0) -> NrrLaunchConfig:
        """Autotunes the batch's launch policy (restarts every pair)."""
        return nrr_batch_tune(self.b, table, reps)

    def context(self, i: int):
        c = _VP()
        _check(load().nrr_batch_get_context(self.b, int(i), ctypes.byref(c)))
        return c

    def close(self):
        if getattr(self, "b", None):
            load().nrr_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
