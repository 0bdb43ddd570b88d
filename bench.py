#!/usr/bin/env python
"""Benchmark: MM iterations/s and time-to-converge of Welsch-norm MM
non-rigid registration with Anderson acceleration on one GB300.

Workload (default ``depth100k``): target = valid pixels of a synthetic
640x480 depth grid of a bumpy height field with 15% hole patches (261,104
points), source = 100,000 samples of the same surface under a smooth warp
(10% of the bbox diagonal) with 1% noise; deformation graph radius 0.062
(about 3,000 nodes), k_alpha = 10, k_beta = 1, Anderson m = 5, stages end on
a relative energy change below 1e-6.

A step is one pass of Algorithm 2 (closest points, energy, safeguard,
weights, assembly, PCG solve, Anderson mix). ``value`` = solves (MM
iterations) per second over K device-timed passes of the mixed-precision
path, with L2 flushed (256 MiB write) before every timed pass. The JSON line
also carries the time-to-converge of the mixed and FP64 paths, the energy
gap between their results, the end-to-end rate through the public API from
pinned host buffers, a roofline entry for the dominant kernel, the sampled
clocks and the FP64 CPU oracle timed on a bounded sample.

N > 1 GPUs (torchrun): every rank registers its own copy of the workload
(replicas, no collective on the data path); value = all ranks' iterations /
max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "MM iters/s and time-to-converge at 100k pts, mixed vs FP64 GPU, same energy"

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of
# the kernels of a pass from one ncu capture of this benchmark's workload,
# with the SHA-256 prefix of the kernel's source file at capture time; a
# figure whose source has changed since is reported as null.
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic_depth100k.txt")
KERNEL_SOURCES = {"nn_kernel": "kernels_nn.cu", "xterm_kernel": "kernels_system.cu",
                  "energy_kernel": "kernels_system.cu",
                  "assemble_kernel": "kernels_system.cu", "solve_kernel": "kernels_solve.cu",
                  "aa_kernels": "kernels_aa.cu"}


def measured_traffic(kernel: str):
    """Per-launch DRAM bytes of ``kernel`` from the committed ncu summary, or
    None if there is none or the kernel's source changed after the capture."""
    import hashlib
    try:
        lines = open(TRAFFIC_FILE).read().splitlines()
    except OSError:
        return None
    src = os.path.join(ROOT, "paper_2206_03410_gb300", "csrc", KERNEL_SOURCES[kernel])
    digest = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    for ln in lines:
        parts = ln.split()
        if len(parts) >= 3 and parts[0] == kernel and not ln.startswith("#"):
            return int(float(parts[1])) if parts[2] == digest else None
    return None
UNIT = "MM iters/s"
FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="depth100k")
    ap.add_argument("--no-ttc", action="store_true", help="skip time-to-converge runs")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-pair batch run")
    ap.add_argument("--ttc-seeds", type=int, default=3,
                    help="extra seeds of the workload for the mixed-vs-FP64 energy comparison")
    ap.add_argument("--no-tune", action="store_true", help="keep the default launch shapes")
    ap.add_argument("--no-variants", action="store_true", help="skip the robust-norm variants run")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample of the workload
# ---------------------------------------------------------------------------
_GRAPH_CACHE = {}


def oracle_pass_seconds(pair, kw, n_sample: int = 1000, seed: int = 0) -> dict:
    """Seconds of one oracle pass on the full workload, estimated from a
    bounded sample: the brute-force closest points of ``n_sample`` random
    source points (scaled to all P), plus one full evaluation of the
    regularisation/rotation terms, the normal equations and their sparse
    direct solve. The closest points that feed the normal equations come
    from a kd-tree (an untimed stand-in with the same result)."""
    import scipy.spatial
    from oracle import graph as OG, model as M, surrogate as S
    V = pair.src.astype(np.float64)
    U = pair.tgt.astype(np.float64)
    key = (pair.name, kw["radius"])
    if key not in _GRAPH_CACHE:          # setup, not part of a pass
        _GRAPH_CACHE[key] = OG.build_graph(V, kw["radius"])
    g = _GRAPH_CACHE[key]
    X = M.identity_X(g.N)
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(V.shape[0], size=min(n_sample, V.shape[0]), replace=False))
    t0 = time.perf_counter()
    vh = M.deform(V[idx], g.nidx[idx], g.w[idx], g.p, X)
    M.closest_points(vh, U)
    t_nn = (time.perf_counter() - t0) * V.shape[0] / len(idx)
    _, rho = scipy.spatial.cKDTree(U).query(M.deform(V, g.nidx, g.w, g.p, X))
    nu_a, nu_r = 0.01, 0.1
    t0 = time.perf_counter()
    terms = M.energy_terms(V, U, g, X, nu_a, nu_r, rho=rho)
    K, B, _ = S.normal_equations(V, U, g, terms, nu_a, nu_r, 1.0, 1.0)
    S.solve_normal_equations(K, B)
    t_rest = time.perf_counter() - t0
    return {"seconds": t_nn + t_rest, "t_nn_scaled": t_nn, "t_rest": t_rest,
            "n_sample": len(idx), "N": g.N}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def algorithmic_bytes(P, T, N, nblk, nnz_infl, pcg_iters, n_ent, esz=4, aa_m=5):
    """Algorithmic HBM bytes per launch of each kernel of a pass (mixed path,
    esz = 4): data each kernel must read or write at least once."""
    nn = P * (3 * esz + 4 + 3 * esz) + nnz_infl * (4 + esz) + T * 16 + \
        P * (4 + esz + 3 * esz + 3 * esz + 3 * esz) + N * 15 * esz
    assemble = n_ent * 4 + P * (3 * esz + esz + 3 * esz) + nnz_infl * (4 + esz) + nblk * 16 * esz + N * 12 * esz
    # per PCG iteration: K once, z gathered, p, q, r, x, z own rows read+written
    solve = max(pcg_iters, 1) * (nblk * 16 * esz + 12 * N * esz * 8) + nblk * 16 * esz
    # Anderson: differences and dots (G, X, F_prev, G_prev and m-1 stored dF
    # read; dF, dG written), then the mix (G, X and m dG read; X, F, G written)
    aa = 12 * N * esz * ((4 + aa_m - 1 + 2) + (2 + aa_m + 3))
    xterm = (nblk - N) * (4 + 4 + esz + esz) + N * (12 + 9) * esz
    energy = P * (esz + esz)
    return {"nn_kernel": nn, "xterm_kernel": xterm, "energy_kernel": energy, "assemble_kernel": assemble,
            "solve_kernel": solve, "aa_kernels": aa}


def tuned(cfg) -> dict:
    """Launch shapes chosen by the library's autotuner."""
    return {"nn_lanes_per_query": cfg.nn_lanes_per_query, "solve_ctas": cfg.solve_ctas,
            **({"nn_ms": round(cfg.nn_ms, 4), "solve_ms": round(cfg.solve_ms, 4)} if cfg.nn_ms else {}),
            **({"pass_ms": round(cfg.pass_ms, 4)} if cfg.pass_ms else {})}


def ttc_pair(nrr, pair, kw, stream, args) -> dict:
    """Time-to-converge of the mixed and FP64 paths on one pair and the
    signed relative gap of their final energies (both in FP64 at the FP64
    run's final nu)."""
    import torch
    src = torch.from_numpy(pair.src).cuda()
    tgt = torch.from_numpy(pair.tgt).cuda()
    out = {}
    finals = {}
    regs = {}
    for name, prec, extra in ARMS:
        r = nrr.Registration(src, tgt, stream=stream.cuda_stream, precision=prec, **kw, **extra)
        if not args.no_tune:
            r.tune()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = r.solve(20000)
        torch.cuda.synchronize()
        out[name + "_ms"] = round((time.perf_counter() - t0) * 1e3, 2)
        out[name + "_iters"] = info.n_solves
        finals[name] = (r.transforms(), info)
        regs[name] = r
    r64 = regs["fp64"]
    i64 = finals["fp64"][1]
    r64.set_stage(i64.nu_a, i64.nu_r)
    e64 = r64.energy(finals["fp64"][0])[0]
    e32 = r64.energy(finals["mixed"][0])[0]
    ec = r64.energy(finals[CONTROL][0])[0]
    for r in regs.values():
        r.close()
    out["gap"] = float((e32 - e64) / abs(e64))
    out["gap_" + CONTROL] = float((ec - e64) / abs(e64))
    out["speedup"] = round(out["fp64_ms"] / out["mixed_ms"], 2)
    return out


# time-to-converge arms: the mixed path, the FP64 path (PCG to 1e-12), and a
# control in FP64 arithmetic with the mixed path's PCG tolerance (1e-6): the
# gap of the control to the FP64 arm is what the solve tolerance alone does
# to the end point of the trajectory
CONTROL = "fp64_pcg1e-6"
ARMS = (("mixed", "mixed", {}), ("fp64", "fp64", {}), (CONTROL, "fp64", dict(pcg_tol=1e-6)))


VARIANTS = [("welsch", {}), ("l2", dict(robust="l2")), ("l2r", dict(robust="l2r")),
            ("welsch_fmax", dict(nu_fixed="max")), ("welsch_fmin", dict(nu_fixed="min")),
            ("welsch_fmed", dict(nu_fixed="med"))]


def run_variants(nrr, stream) -> dict:
    """Sec. 4.2's comparison on the partial-overlap workload (50,000 source
    points, 30 % of the target cropped, 2 % noise, 10 % outliers), mixed
    precision: wall time of nrr_solve to convergence and the RMSE of the
    deformed source against the generator's ground truth (Eq. gt_metric)."""
    import torch
    pair = synth.workload("sphere50k_partial")
    kw = {k: v for k, v in pair.params.items() if k not in ("precision", "iters", "unroll")}
    kw["rel_energy_tol"] = 1e-6
    src = torch.from_numpy(pair.src).cuda()
    tgt = torch.from_numpy(pair.tgt).cuda()
    gt = pair.gt.astype(np.float64)
    out = {"workload": "sphere50k_partial: P=%d, T=%d, 30 %% crop, 2 %% noise, 10 %% outliers, mixed, "
                       "stages end at relative dE < 1e-6" % (pair.P, pair.T)}
    for name, extra in VARIANTS:
        r = nrr.Registration(src, tgt, stream=stream.cuda_stream, precision="mixed", **kw, **extra)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = r.solve(20000)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        vh = r.deformed()
        rmse = float(np.sqrt(np.mean(np.sum((vh - gt) ** 2, axis=1))))
        out[name] = {"ms": round(dt * 1e3, 2), "iters": info.n_solves, "stages": info.stage + 1,
                     "rmse": rmse, "done": info.done}
        r.close()
    return out


def reduce_over_ranks(total_ms: float, iters: float, device) -> tuple[float, float]:
    """Whole-job numbers over the ranks of a replica run: the slowest rank's
    timed milliseconds and the sum of every rank's iterations."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(total_ms), float(iters)
    tmax = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    tsum = torch.tensor([float(iters)], dtype=torch.float64, device=device)
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(tsum[0])


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2206_03410_gb300 import nrr

    ws, rank, local = dist_env()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    pair = synth.workload(args.workload)
    kw = {k: v for k, v in pair.params.items() if k not in ("precision", "iters", "unroll")}
    stream = torch.cuda.Stream()
    src = torch.from_numpy(pair.src).cuda()
    tgt = torch.from_numpy(pair.tgt).cuda()
    reg = nrr.Registration(src, tgt, stream=stream.cuda_stream, precision="mixed", **kw)
    launch = {}
    if not args.no_tune:
        launch["mixed"] = tuned(reg.tune())
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- steady-state MM iteration throughput (device-timed) -------------
    reg.reset()
    reg.enqueue_passes(args.warmup)
    barrier()
    i0 = reg.info()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clocks = Clocks(dev)
    clocks.start()
    barrier()
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            reg.enqueue_passes(1)
            ev[k][1].record(stream)
    barrier()
    clk = clocks.stop()
    total_ms = sum(a.elapsed_time(b) for a, b in ev)
    i1 = reg.info()
    iters = i1.n_solves - i0.n_solves
    passes = i1.n_passes - i0.n_passes
    total_ms_all, iters_all = reduce_over_ranks(total_ms, iters, "cuda")
    value = iters_all / (total_ms_all / 1e3)

    # ---- per-kernel durations (events on the library's stream) ----------
    reg.reset()
    reg.enqueue_passes(args.warmup)
    torch.cuda.synchronize()
    ms = np.zeros(len(nrr.KERNELS))
    ks0 = reg.info()
    pcg_sum = 0   # CG iterations of the timed solve launches (0 for a pass that did not solve)
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(float(k))
        ms += reg.time_kernels(1)
        inf = reg.info()
        if inf.solved:
            pcg_sum += int(inf.pcg_iters)
    ks1 = reg.info()
    kt_passes = max(ks1.n_passes - ks0.n_passes, 1)
    solves_k = max(ks1.n_solves - ks0.n_solves, 1)
    per_launch_ms = ms / args.steps
    top = int(np.argmax(ms))
    names = list(nrr.KERNELS)
    result = {"rank": rank, "iters": iters, "passes": passes, "total_ms": total_ms}

    if rank == 0:
        g = reg.graph()
        nnz = int((g.nidx >= 0).sum())
        E2 = 2 * reg.n_edges
        nblk = reg.N + E2
        K_, _ = None, None
        # contributions per block list: sum over points of |I(v_i)|^2
        k_i = (g.nidx >= 0).sum(axis=1)
        n_ent = int(np.sum(k_i * k_i))
        # CG iterations per solve launch, over the launches whose durations
        # make per_launch_ms (the algorithmic bytes scale with them)
        avg_pcg = pcg_sum / max(args.steps, 1)
        ab = algorithmic_bytes(reg.P, reg.T, reg.N, nblk, nnz, avg_pcg, n_ent)
        peaks = {}
        try:
            peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        except OSError:
            pass
        hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
        top_name = names[top]
        achieved = ab[top_name] / (per_launch_ms[top] / 1e3) / 1e9
        roofline = {"kernel": top_name, "bound": "hbm", "achieved": round(achieved, 2),
                    "peak": hbm_peak, "unit": "GB/s", "frac": round(achieved / hbm_peak, 5),
                    "traffic": measured_traffic(top_name),
                    "peak_source": "measured" if peaks else "fallback",
                    "algorithmic_bytes_per_launch": int(ab[top_name]),
                    "avg_launch_ms": round(float(per_launch_ms[top]), 4),
                    "launch_ms": {n: round(float(v), 4) for n, v in zip(names, per_launch_ms)},
                    "share": {n: round(float(v / ms.sum()), 4) for n, v in zip(names, ms)},
                    "launch_ms_note": "steps timed one after the other; in the pass graph xterm_kernel "
                                      "runs beside nn_kernel"}
        # the solve is latency-bound: time per CG iteration and the
        # cluster-wide synchronisations each iteration needs
        cl_ctas = reg.launch_config().solve_ctas
        solve_ms = float(per_launch_ms[names.index("solve_kernel")])
        pcg = {"cg_iters_per_launch": round(avg_pcg, 2),
               "us_per_cg_iter": round(solve_ms * 1e3 / avg_pcg, 3) if avg_pcg > 0 else None,
               "syncs_per_cg_iter": 1 if cl_ctas > 0 else 2,
               "solver": f"cluster of {cl_ctas} CTAs" if cl_ctas > 0 else "grid-wide"}
        result.update(dict(roofline=roofline, P=reg.P, T=reg.T, N=reg.N, n_edges=reg.n_edges,
                           pcg=pcg, clocks=clk, launch=launch,
                           launches_per_pass=reg.launch_config().launches_per_pass))

        # ---- time-to-converge: mixed vs FP64, same energy -----------------
        if not args.no_ttc:
            ttc = {}
            finals = {}
            reg64 = nrr.Registration(src, tgt, stream=stream.cuda_stream, precision="fp64", **kw)
            if not args.no_tune:
                launch["fp64"] = tuned(reg64.tune())
            for name, r in (("mixed", reg), ("fp64", reg64)):
                r.reset()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                info = r.solve(20000)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                ttc[name] = {"ms": round(dt * 1e3, 2), "iters": info.n_solves, "passes": info.n_passes,
                             "rejected": info.n_rejected, "stages": info.stage + 1, "done": info.done}
                finals[name] = (r.transforms(), info)
            i64 = finals["fp64"][1]
            reg64.set_stage(i64.nu_a, i64.nu_r)
            e64 = reg64.energy(finals["fp64"][0])[0]
            e32 = reg64.energy(finals["mixed"][0])[0]
            ttc["speedup_mixed_vs_fp64"] = round(ttc["fp64"]["ms"] / ttc["mixed"]["ms"], 3)
            ttc["energy_rel_gap"] = float(abs(e32 - e64) / abs(e64))
            ttc["E_fp64"] = float(e64)
            ttc["E_mixed_in_fp64"] = float(e32)
            reg64.close()
            # the same comparison on further seeds of the workload: signed
            # relative gap (E_mixed - E_fp64) / E_fp64 at the FP64 run's final nu
            seeds = []
            for sd in range(args.ttc_seeds):
                seeds.append(ttc_pair(nrr, synth.workload(args.workload, seed=100 + sd), kw, stream, args))
            if seeds:
                ttc["seeds"] = seeds
                gaps = [x["gap"] for x in seeds] + [float((e32 - e64) / abs(e64))]
                ttc["signed_gaps_all"] = gaps
                ttc["mixed_not_worse"] = int(sum(g <= 1e-5 for g in gaps))
                ttc["runs"] = len(gaps)
                ctl = [x["gap_" + CONTROL] for x in seeds]
                ttc["control"] = {"arm": CONTROL + ": FP64 arithmetic, PCG to relative residual 1e-6",
                                  "signed_gaps": ctl,
                                  "mean_abs_gap": float(np.mean(np.abs(ctl))),
                                  "mixed_mean_abs_gap": float(np.mean(np.abs([x["gap"] for x in seeds])))}
            result["ttc"] = ttc

        # ---- batched pairs (64 independent pairs, one graph launch per pass) ----
        if not args.no_batch:
            pairs = synth.batch_pairs(64)
            prm = [dict(radius=p.params["radius"], k_alpha=100.0, k_beta=1.0, aa_m=5,
                        precision="mixed") for p in pairs]
            t0 = time.perf_counter()
            bt = nrr.BatchRegistration([(p.src, p.tgt) for p in pairs], params=prm,
                                       stream=stream.cuda_stream)
            t_create = time.perf_counter() - t0
            if not args.no_tune:
                launch["batch"] = tuned(bt.tune())
            runs = []
            for _ in range(2):
                bt.reset()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                infos = bt.solve(20000)
                torch.cuda.synchronize()
                runs.append(time.perf_counter() - t0)
            dt = min(runs)
            its = sum(i.n_solves for i in infos)
            result["batch"] = {"workload": "64 sphere pairs, P log-uniform 2k-40k (sum %d), N 100-1000, "
                                           "crop 0-30 %%, outliers 0-10 %%, mixed" % sum(p.P for p in pairs),
                               "ms_to_converge_all": round(dt * 1e3, 2), "pairs_per_s": round(64 / dt, 2),
                               "mm_iters_per_s": round(its / dt, 1), "iters": its,
                               "all_done": all(i.done for i in infos), "create_s": round(t_create, 2)}
            bt.close()

        # ---- robust-norm variants (Sec. 4.2) on the partial-overlap workload ----
        if not args.no_variants:
            result["variants"] = run_variants(nrr, stream)

        # ---- end to end through the public API from pinned host buffers ----
        hs = torch.from_numpy(pair.src).pin_memory()
        ht = torch.from_numpy(pair.tgt).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r2 = nrr.Registration(hs, ht, stream=stream.cuda_stream, precision="mixed", **kw)
        info2 = r2.solve(20000)
        Xh = r2.transforms()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        # the inputs go up once and the transforms come back once per
        # registration: per step, the bytes averaged over its MM iterations
        h2d = int(hs.numel() * 4 + ht.numel() * 4)
        d2h = int(Xh.size * 8)
        n_it = max(int(info2.n_solves), 1)
        result["e2e"] = {"value": round(info2.n_solves / dt, 3), "unit": UNIT,
                         "h2d_bytes_per_step": int(round(h2d / n_it)),
                         "d2h_bytes_per_step": int(round(d2h / n_it)),
                         "h2d_bytes_per_registration": h2d, "d2h_bytes_per_registration": d2h,
                         "seconds": round(dt, 4), "iters": info2.n_solves,
                         "includes": "nrr_create from pinned host buffers (graph + search structures) + "
                                     "nrr_solve to convergence + nrr_get_transforms to host"}
        r2.close()
    reg.close()
    return value, total_ms_all, result, ws, rank


def cpu_baseline(pair, kw):
    t0 = time.perf_counter()
    s = oracle_pass_seconds(pair, kw, n_sample=1000)
    return {"value": round(1.0 / s["seconds"], 5), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": (f"one oracle pass of {pair.name}: brute-force closest points of "
                       f"{s['n_sample']} random source points scaled to all {pair.P} "
                       f"({s['t_nn_scaled']:.1f} s), plus normal equations and sparse direct "
                       f"solve on the full problem ({s['t_rest']:.1f} s); numpy/scipy single-threaded"),
            "wall_s": round(time.perf_counter() - t0, 1)}




def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    value, total_ms, res, ws, rank = run_ours(args)
    if rank != 0:
        return
    pair = synth.workload(args.workload)
    kw = {k: v for k, v in pair.params.items() if k not in ("precision", "iters", "unroll")}
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(total_ms / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (seeded depth-grid pair, see synth.depth_scene)",
        "config": {"workload": f"{args.workload}: P={res['P']} source, T={res['T']} target "
                   f"(640x480 depth grid, 15% holes), N={res['N']} nodes, |E_G|={res['n_edges']}, "
                   "mixed precision (f32 closest points/assembly/PCG, f64 energy+AA)",
                   "parallelism": "replicas" if ws > 1 else "single",
                   "l2": "flushed before every timed pass (256 MiB write); inputs L2-resident otherwise",
                   "iters_timed": res["iters"], "passes_timed": res["passes"]},
        "roofline": res["roofline"],
        "pcg": res["pcg"],
        "clocks": res["clocks"],
        "gpu_launches": res["launches_per_pass"] * args.steps,
        "e2e": res.get("e2e"),
        "ttc": res.get("ttc"),
        "batch": res.get("batch"),
        "launch": res.get("launch"),
        "variants": res.get("variants"),
    }
    if ws == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(pair, kw)
    print(json.dumps(line))


def run_reference(args):
    """Reference arm: the FP64 CPU oracle as it stands, on the host cores,
    each step a bounded sample of the same workload."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    pair = synth.workload(args.workload)
    kw = {k: v for k, v in pair.params.items() if k not in ("precision", "iters", "unroll")}
    total = 0.0
    samp = None
    for k in range(args.warmup + args.steps):
        s = oracle_pass_seconds(pair, kw, n_sample=200, seed=k)
        if k >= args.warmup:
            total += s["seconds"]
            samp = s
    value = args.steps / total
    desc = (f"each step: one oracle pass of {pair.name} estimated from brute-force closest "
            f"points of {samp['n_sample']} random source points scaled to all {pair.P}, plus "
            "normal equations and sparse direct solve on the full problem; single-threaded")
    line = {"metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * total / args.steps, 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": pair.name, "parallelism": "single"},
            "impl": "reference",
            "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
