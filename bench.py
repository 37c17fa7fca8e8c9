#!/usr/bin/env python
"""GLBM throughput benchmark: lattice node updates per second (GLUPS) and the
fused step kernel's fraction of the HBM roofline, on one two-phase shale
medium per GPU.

One benchmark step = one ``glbm_step`` call of ``--chunk`` time steps
(the fused stream+collide kernel ``--chunk`` times, the last one also
producing the FP64 mean-velocity partials, plus the reduction finalize),
i.e. every step of the hot path; the Darcy permeability is read at the end.

Default workload: 4096x4096 D2Q9 lattice, two-phase OM/IOM medium (OM
fraction 0.2 grown with correlation length 8 nodes, eps 0.10/0.15, K
log-uniform [1e-4,1e-3] / [5e-4,5e-3]), G = 1e-6 along x, tau = 1, walls in
y, FP32 deviation storage.  Inputs (1.3 GB of distributions) are far larger
than the 129 MB L2, so no flush is needed between iterations.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Multi-GPU (torchrun): every rank advances its own medium (seed = rank);
there is no exchange on the data path (weak scaling).  The printed value is
the node updates of all ranks over the slowest rank's time.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "GLBM GLUPS & % HBM roofline; time-to-permeability (warm/low-prec vs plain)"
UNIT = "GLUPS"
G = 1e-6
TAU = 1.0
# bytes moved per node update by the fused step kernel (algorithmic):
# 9 populations read + 9 written, plus the packed coefficients (alpha, eps).
ELEM = {"f32": 4, "f64": 8, "f16": 2, "bf16": 2}
NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e, nominal (context beside the measured copy bandwidth)
COEF = {"f32": 8, "f64": 16, "f16": 8, "bf16": 8}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def args_():
    p = argparse.ArgumentParser(description=__doc__,
                                formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--nx", type=int, default=4096)
    p.add_argument("--ny", type=int, default=4096)
    p.add_argument("--chunk", type=int, default=500,
                   help="lattice time steps per benchmark step")
    p.add_argument("--storage", default="f32", choices=list(ELEM))
    p.add_argument("--om-fraction", type=float, default=0.2)
    p.add_argument("--corr-len", type=float, default=8.0)
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--cpu-seconds", type=float, default=15.0,
                   help="CPU-oracle sample budget")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-ttc", action="store_true",
                   help="skip the time-to-converged comparison of the storage formats")
    p.add_argument("--ttc-n", type=int, default=4096,
                   help="lattice side of the time-to-converged runs")
    p.add_argument("--no-warm", action="store_true",
                   help="skip the learned warm-start study")
    p.add_argument("--no-batch", action="store_true",
                   help="skip the batched-media (DGM/GMS sweep) measurement")
    p.add_argument("--batch-count", type=int, default=512)
    p.add_argument("--batch-steps", type=int, default=500)
    p.add_argument("--jsonl", metavar="PATH",
                   help="also append the result line to this JSON-lines file (one record per run)")
    p.add_argument("--sweep", type=int, default=0, metavar="STEPS",
                   help="also run the 25-cell medium sweep (OM fraction x correlation length at nx x ny), "
                        "each cell up to STEPS time steps or converged (off by default: minutes)")
    return p.parse_args()


def workload(a, rank=0):
    return {
        "workload": (f"GLBM D2Q9 {a.nx}x{a.ny} two-phase OM/IOM medium "
                     f"(OM fraction {a.om_fraction}, correlation length "
                     f"{a.corr_len:g}, eps 0.10/0.15, K log-uniform "
                     f"[1e-4,1e-3]/[5e-4,5e-3], seed {a.seed + rank}), "
                     f"G={G:g} along x, tau={TAU:g}, walls in y"),
        "nx": a.nx, "ny": a.ny, "storage": a.storage,
        "lb_steps_per_step": a.chunk,
        "l2": "no flush: 1.2 GB of distributions per step >> 129 MB L2",
    }


def make_medium(a, rank=0):
    import media
    eps, K, _ = media.two_phase_medium(a.nx, a.ny, om_fraction=a.om_fraction,
                                       corr_len=a.corr_len, seed=a.seed + rank)
    return eps, K


# -- distributed plumbing --------------------------------------------------

def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# -- clocks ---------------------------------------------------------------

class Clocks:
    FIELDS = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 10:
                    continue
                if self.uuid and parts[1] != self.uuid:
                    continue
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[6:10]) if v == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows),
                "power_w_max": max((float(r[4]) for r in rows
                                    if r[4].replace(".", "").isdigit()), default=None)}


def gpu_uuid():
    try:
        import torch
        u = torch.cuda.get_device_properties(torch.cuda.current_device()).uuid
        return "GPU-" + str(u)
    except Exception:
        return None


# -- roofline evidence ----------------------------------------------------

def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def source_hash():
    """Hash of the step kernel's source (csrc/glbm_kernels.cuh): a committed
    ncu traffic figure is used only while the kernel it measured is unchanged."""
    h = hashlib.sha256()
    h.update(open(os.path.join(ROOT, "paper_1601_00704_gb300", "csrc", "glbm_kernels.cuh"), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(storage, nx, ny):
    """DRAM bytes per launch of the step kernel from the committed ncu summary,
    scaled to this lattice; None if absent or taken from other source code."""
    path = os.path.join(ROOT, "profiles", f"k_step_{storage}.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m_src = re.search(r"source_sha256_16:\s*([0-9a-f]{16})", text)
    m_b = re.search(r"dram_bytes_per_node_update:\s*([0-9.eE+-]+)", text)
    if not (m_src and m_b) or m_src.group(1) != source_hash():
        return None
    return float(m_b.group(1)) * nx * ny


# -- CPU oracle timing ------------------------------------------------------

def oracle_sample(a, eps, K, seconds, nsteps=None):
    """Time the FP64 oracle (OpenMP build, all host cores) on the same
    medium for a bounded number of time steps; returns (GLUPS, cores, steps, s)."""
    import oracle
    oracle.build()
    o = oracle.Oracle(a.nx, a.ny, tau=TAU, threads=os.cpu_count())
    cores = oracle._lib(True).orc_threads(0)
    o.set_medium(eps, K)
    o.set_force(G)
    if nsteps is None:
        t0 = time.perf_counter()
        o.step(1)
        t1 = time.perf_counter() - t0
        nsteps = max(1, min(500, int(seconds / max(t1, 1e-6))))
    t0 = time.perf_counter()
    o.step(nsteps)
    dt = time.perf_counter() - t0
    return a.nx * a.ny * nsteps / dt / 1e9, cores, nsteps, dt


def cpu_desc():
    model = ""
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    return model


# -- time to a converged permeability -------------------------------------------

# The solver's own stopping rule (one a user can apply): the relative change
# of U_x per TTC_CHECK steps at most TTC_TOL on TTC_PATIENCE consecutive
# checks.  The reference run continues the FP32 run to TTC_REF_TOL.
TTC_TOL, TTC_CHECK, TTC_PATIENCE = 1e-5, 1000, 3
TTC_REF_TOL = 1e-6
TTC_MAX = 2_000_000


def format_throughput(a, eps, K, steps=300):
    """GLUPS of each storage format on the benchmark lattice (HBM-bound),
    timed with CUDA events over `steps` steps after 100 warm-up steps."""
    import torch

    import paper_1601_00704_gb300 as pkg
    out = {}
    stream = torch.cuda.Stream()
    for st in ("f32", "f16", "bf16"):
        s = pkg.Solver(a.nx, a.ny, tau=TAU, storage=st, stream=stream)
        s.set_medium(eps, K)
        s.set_force(G)
        s.step(100)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(steps)
        e1.record(stream)
        e1.synchronize()
        us = e0.elapsed_time(e1) * 1e3 / steps
        bpu = 18 * ELEM[st] + COEF[st]
        out[st] = {"glups": a.nx * a.ny / us / 1e3, "us_per_step": us,
                   "bytes_per_node_update": bpu,
                   "frac_of_measured_hbm": bpu * a.nx * a.ny / us / 1e3 / peaks()[0]}
        s.close()
    return out


def time_to_converged(a, variants=("f32", "f16", "bf16")):
    """Per storage format, from rest on an n x n medium with the widened K
    spread (log-uniform [1e-6, 1e-2] in both phases, seed --seed): steps and
    CUDA-event seconds until the solver's own convergence test stops the run,
    and the error of K_app at that stop against K_ref.  K_ref continues the
    FP32 run to a tenfold tighter tolerance (its own remaining error is
    about a tenth of the stopped runs')."""
    import torch

    import media
    import paper_1601_00704_gb300 as pkg
    n = a.ttc_n
    eps, K, _ = media.two_phase_medium(n, n, om_fraction=a.om_fraction, corr_len=a.corr_len,
                                       seed=a.seed, k_iom=(1e-6, 1e-2), k_om=(1e-6, 1e-2))
    stream = torch.cuda.Stream()
    runs, k_ref, ref = {}, None, None
    for v in variants:
        s = pkg.Solver(n, n, tau=TAU, storage=v, stream=stream)
        s.set_medium(eps, K)
        s.set_force(G)
        s.set_convergence(TTC_PATIENCE)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        steps, conv = s.step(TTC_MAX, tol=TTC_TOL, check_every=TTC_CHECK)
        k = s.permeability()
        e1.record(stream)
        e1.synchronize()
        runs[v] = {"steps": steps, "seconds": e0.elapsed_time(e1) * 1e-3, "converged": conv, "k_app": k}
        if v == "f32":
            more, rconv = s.step(TTC_MAX, tol=TTC_REF_TOL, check_every=TTC_CHECK)
            k_ref = s.permeability()
            ref = {"steps": steps + more, "converged": rconv}
        s.close()
    for r in runs.values():
        r["rel_err"] = r["k_app"] / k_ref - 1
    base = runs["f32"]["seconds"]
    return {
        "workload": (f"{n}x{n} two-phase medium (OM fraction {a.om_fraction}, correlation length "
                     f"{a.corr_len:g}, seed {a.seed}), K log-uniform [1e-6,1e-2] in both phases (the "
                     "widened spread of the precision workload), from rest"),
        "stop_rule": f"relative change of U_x <= {TTC_TOL:g} per {TTC_CHECK} steps on {TTC_PATIENCE} "
                     "consecutive checks (the solver's own test)",
        "k_ref": k_ref,
        "k_ref_from": (f"the FP32 run continued to <= {TTC_REF_TOL:g} per {TTC_CHECK} steps on "
                       f"{TTC_PATIENCE} checks ({ref['steps']} steps, converged={ref['converged']})"),
        "runs": runs,
        "speedup_vs_f32": {v: base / r["seconds"] for v, r in runs.items() if v != "f32" and r["converged"]},
        "max_abs_rel_err": max(abs(r["rel_err"]) for r in runs.values()),
    }


# -- batched media: DGM/GMS sweep -------------------------------------------

DX = 7.8125e-9          # lattice spacing (m): 1024 nodes span 8 micrometres
T_GAS, ETA, TORT = 350.0, 18.231e-6, 2.0
DS = 1e-8               # surface diffusivity (m^2/s) of the paper's shale inputs
RHO_KEROGEN, EPS_KEROGEN = 1.65e3, 0.2   # Eq. 38 kerogen density, porosity
RHO_CH4 = 0.717         # kg/m^3, methane at standard conditions
MDARCY = 9.869233e-16   # m^2


BATCH_TOL, BATCH_CHECK, BATCH_PATIENCE, BATCH_MAX = 1e-5, 1000, 3, 300_000


def batch_bench(a):
    """Many media of uneven size with per-node K from the DGM/GMS model,
    advanced together: the autotuned schedule (threads per block, tile
    order, one launch per step from captured graphs or one persistent
    cooperative launch per chunk), fixed-length throughput of both launch
    modes, a run of the whole batch until every medium has converged, and
    the same media stepped one lattice at a time."""
    import numpy as np
    import torch

    import media
    import paper_1601_00704_gb300 as pkg
    t0 = time.perf_counter()
    specs = media.shale_batch(a.batch_count, seed=a.seed)
    gen_s = time.perf_counter() - t0
    shapes = [(m["n"], m["n"]) for m in specs]
    stream = torch.cuda.Stream()
    b = pkg.Batch(shapes, tau=TAU, storage="f32", stream=stream)
    t0 = time.perf_counter()
    kfields = []
    for i, m in enumerate(specs):
        qsat = pkg.qsat_from_langmuir_volume(m["V_L"], RHO_KEROGEN, EPS_KEROGEN,
                                             max(m["toc"], 1e-9), RHO_CH4)
        K = pkg.kapp_field(m["r"], m["organic"], m["eps"], m["P"], T_GAS, ETA, TORT,
                           qsat, 1.0 / m["P_L"], DS, DX)
        b.set_medium(i, m["eps"], K)
        kfields.append((float(K.min()), float(K.max())))
    setup_s = time.perf_counter() - t0
    b.set_force(G)
    b.set_convergence(BATCH_PATIENCE)
    threads, order = b.autotune(trial_steps=10)
    persistent = b.persistent
    nodes = b.info()["nodes"]

    def timed(n, **kw):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        l0 = b.info()["launches"]
        e0.record(stream)
        out = b.step(n, **kw)
        e1.record(stream)
        e1.synchronize()
        return out, e0.elapsed_time(e1) * 1e-3, b.info()["launches"] - l0

    modes = {}
    for pers in (False, True):
        b.set_persistent(pers)
        b.reset()
        b.step(100, check_every=100)  # warm-up (captures the chunk graph)
        _, sec, launches = timed(a.batch_steps, check_every=100)
        modes["persistent" if pers else "graph_per_step"] = {
            "glups": nodes * a.batch_steps / sec / 1e9, "seconds": sec, "launches": launches}
    b.set_persistent(persistent)
    b.reset()
    (done, left), conv_s, conv_launches = timed(BATCH_MAX, tol=BATCH_TOL, check_every=BATCH_CHECK)
    res = b.results()
    b.close()
    steps = res["steps"]
    sizes = np.array([ny * nx for ny, nx in shapes], dtype=np.float64)
    kphys = res["kxx"] * DX * DX / MDARCY
    edges = [0, 2000, 4000, 8000, 16000, 32000, 64000, 128000, BATCH_MAX]
    hist, _ = np.histogram(steps, bins=edges)
    # the same media, one lattice at a time, for a shorter run
    seq_steps = max(10, a.batch_steps // 10)
    t_seq = 0.0
    for i, m in enumerate(specs):
        n = m["n"]
        qsat = pkg.qsat_from_langmuir_volume(m["V_L"], RHO_KEROGEN, EPS_KEROGEN,
                                             max(m["toc"], 1e-9), RHO_CH4)
        K = pkg.kapp_field(m["r"], m["organic"], m["eps"], m["P"], T_GAS, ETA, TORT,
                           qsat, 1.0 / m["P_L"], DS, DX)
        s = pkg.Solver(n, n, tau=TAU)
        s.set_medium(m["eps"], K)
        s.set_force(G)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        s.step(seq_steps)
        s.mean_velocity()
        t_seq += time.perf_counter() - t1
        s.close()
    best = max(modes.values(), key=lambda r: r["glups"])
    return {
        "workload": (f"{len(specs)} media, square sides uniform in 64..1024 (step 64), "
                     f"{nodes} nodes; OM fraction 0.2 (correlation length 8); pore radius "
                     f"lognormal (median 5 nm OM / 20 nm IOM, sigma_ln 0.5); P 0.5-30 MPa, "
                     f"P_L 2-10 MPa, V_L 0.002-0.01 m^3/kg; methane at 350 K, D_s 1e-8 m^2/s; "
                     f"dx {DX:g} m; per-node K from Eqs. 18-19; FP32, walls in y"),
        "nodes": nodes, "steps": a.batch_steps,
        "glups": best["glups"],
        "launch_modes": modes,
        "schedule": {"threads": threads, "order": order, "persistent": persistent, "autotuned": True},
        "converged_run": {
            "stop_rule": f"per medium: relative change of U_x <= {BATCH_TOL:g} per {BATCH_CHECK} steps on "
                         f"{BATCH_PATIENCE} consecutive checks; the medium then leaves the batch",
            "seconds": conv_s, "batch_steps": done, "media_left": left,
            "converged": int(res["converged"].sum()), "launches": conv_launches,
            "node_updates": float((sizes * steps).sum()),
            "glups": float((sizes * steps).sum()) / conv_s / 1e9,
            "exit_steps": {"min": int(steps.min()), "median": float(np.median(steps)),
                           "max": int(steps.max()),
                           "histogram": {f"{lo}-{hi}": int(c) for lo, hi, c in zip(edges[:-1], edges[1:], hist)}},
            "k_app_mD": {"min": float(kphys.min()), "median": float(np.median(kphys)),
                         "max": float(kphys.max())},
        },
        "one_at_a_time_glups": nodes * seq_steps / t_seq / 1e9,
        "k_lattice_range": [min(k[0] for k in kfields), max(k[1] for k in kfields)],
        "generate_s": gen_s, "setup_s": setup_s,
    }


# -- learned warm start ---------------------------------------------------------

SWEEP_OM = (0.05, 0.10, 0.20, 0.30, 0.40)
SWEEP_CORR = (4, 8, 16, 32, 64)


def sweep(a):
    """The two-phase workload over OM fraction x correlation length: per
    cell the kernel throughput (CUDA events over the whole run) and K_app
    after at most a.sweep steps or convergence (relative change of U_x
    below 1e-10 per 1000 steps)."""
    import torch

    import media
    import paper_1601_00704_gb300 as pkg
    stream = torch.cuda.Stream()
    cells = []
    bytes_per = ELEM[a.storage] * 18 + 2 * (8 if a.storage == "f64" else 4)
    peak = peaks()[0]
    for om in SWEEP_OM:
        for cl in SWEEP_CORR:
            eps, K, _ = media.two_phase_medium(a.nx, a.ny, om_fraction=om, corr_len=cl, seed=a.seed)
            s = pkg.Solver(a.nx, a.ny, tau=TAU, storage=a.storage, stream=stream)
            s.set_medium(eps, K)
            s.set_force(G)
            s.step(100)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            done, conv = s.step(a.sweep, tol=1e-10, check_every=1000)
            e1.record(stream)
            e1.synchronize()
            sec = e0.elapsed_time(e1) * 1e-3
            glups = a.nx * a.ny * done / sec / 1e9
            cells.append({"om_fraction": om, "corr_len": cl, "steps": done, "converged": bool(conv),
                          "glups": glups, "frac_of_measured_hbm": glups * bytes_per / peak,
                          "k_app": s.permeability()})
            s.close()
    g = [c["glups"] for c in cells]
    return {"workload": f"{a.nx}x{a.ny} two-phase media, OM fraction {list(SWEEP_OM)} x correlation length "
                        f"{list(SWEEP_CORR)}, seed {a.seed}, storage {a.storage}, up to {a.sweep} steps or "
                        f"relative change of U_x < 1e-10 per 1000 steps",
            "glups_min": min(g), "glups_max": max(g), "cells": cells}


def warm_start(a):
    """Cold vs surrogate-initialised runs (FP32 and BF16) on three unseen
    2048^2 media of the surrogate's training recipe, with the committed
    weights."""
    from paper_1601_00704_gb300 import surrogate
    from paper_1601_00704_gb300 import train_surrogate as T
    path = T.DEFAULT_WEIGHTS
    if not os.path.exists(path):
        return {"unavailable": f"no trained weights at {os.path.relpath(path, ROOT)}"}
    meta = json.load(open(os.path.splitext(path)[0] + ".json"))
    net = surrogate.UNet(base=meta["base"], levels=meta["levels"], max_ch=meta.get("max_ch"))
    net.load(path)
    out = T.warm_start_study(net, log=lambda *_: None)
    out["network"] = {"levels": meta["levels"], "base": meta["base"], "max_ch": meta.get("max_ch"),
                      "params": meta["params"], "weights": os.path.relpath(path, ROOT)}
    return out


# -- arms ---------------------------------------------------------------------

def run_reference(a, world, rank):
    if rank != 0:
        return 0
    eps, K = make_medium(a)
    # each benchmark step: a bounded sample of the same workload (full lattice,
    # a few time steps), sized so warm-up + timed steps stay within minutes
    per = max(5.0, min(30.0, 150.0 / max(1, a.steps + a.warmup)))
    g1, cores, n, dt = oracle_sample(a, eps, K, per)
    times = []
    for i in range(a.warmup + a.steps):
        g, cores, _, dt = oracle_sample(a, eps, K, per, nsteps=n)
        if i >= a.warmup:
            times.append(dt)
    tot = sum(times)
    val = a.nx * a.ny * n * a.steps / tot / 1e9
    cfg = workload(a)
    cfg["lb_steps_per_step"] = n
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT,
        "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": 1e3 * tot / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded Gaussian-random-field two-phase medium)",
        "config": cfg,
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{n} time steps of the full {a.nx}x{a.ny} lattice per "
                                   f"step, FP64 oracle, OpenMP over rows on {cpu_desc()}"},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    emit(line, a)
    return 0


def emit(line, a):
    """The one JSON result line on stdout and, with --jsonl, appended to that file."""
    text = json.dumps(line)
    print(text, flush=True)
    if a.jsonl:
        with open(a.jsonl, "a") as fh:
            fh.write(text + "\n")


def run_ours(a, world, rank, local):
    import numpy as np
    import torch

    import paper_1601_00704_gb300 as pkg
    from paper_1601_00704_gb300 import build as pbuild
    if not torch.cuda.is_available():
        raise SystemExit("bench.py: a CUDA device is required")
    torch.cuda.set_device(local)
    pbuild.build()
    eps, K = make_medium(a, rank)
    N = a.nx * a.ny
    stream = torch.cuda.Stream()
    s = pkg.Solver(a.nx, a.ny, tau=TAU, storage=a.storage, walls=True, stream=stream)
    s.set_medium(eps, K)
    s.set_force(G, 0.0)
    for _ in range(a.warmup):
        s.step(a.chunk)
    torch.cuda.synchronize()
    barrier(world)
    _, l0 = s.counters()
    clocks = Clocks(gpu_uuid())
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    clocks.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(a.steps):
        s.step(a.chunk)
    ev1.record(stream)
    ev1.synchronize()
    clk = clocks.stop()
    torch.cuda.synchronize()
    barrier(world)
    _, l1 = s.counters()
    ms = max_over_ranks(ev0.elapsed_time(ev1), world)
    kapp = s.permeability()
    updates = N * a.chunk * a.steps
    value = world * updates / (ms * 1e-3) / 1e9
    # dominant kernel: the fused step, chunk launches per benchmark step
    # (the finalize kernel adds ~3 us per chunk, included here)
    bpu = 18 * ELEM[a.storage] + COEF[a.storage]
    per_launch_s = ms * 1e-3 / (a.chunk * a.steps)
    achieved = bpu * N / per_launch_s / 1e9
    peak, peak_kind = peaks()
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": ncu_traffic(a.storage, a.nx, a.ny),
            "peak_kind": peak_kind, "bytes_per_node_update": bpu,
            "kernel": f"k_step<{a.storage}> (fused pull-stream + collide)",
            "launch_us": per_launch_s * 1e6,
            "nominal": {"peak": NOMINAL_HBM_GBS, "frac": achieved / NOMINAL_HBM_GBS,
                        "what": "GB300 HBM3e nominal bandwidth"}}

    e2e = None
    if not a.no_e2e:
        # the same metric through the public API from pinned host buffers:
        # set_medium (H2D of eps, K) + chunk steps + K_app read-back per step
        pe = torch.from_numpy(eps).pin_memory()
        pk = torch.from_numpy(K).pin_memory()
        he, hk = pe.numpy(), pk.numpy()
        for _ in range(1):
            s.set_medium(he, hk)
            s.step(a.chunk)
            s.permeability()
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(a.steps):
            s.set_medium(he, hk)
            s.step(a.chunk)
            s.permeability()
        torch.cuda.synchronize()
        dt = max_over_ranks(time.perf_counter() - t0, world)
        e2e = {"value": world * updates / dt / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": 2 * 8 * N, "d2h_bytes_per_step": 40}

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        g, cores, n, dt = oracle_sample(a, eps, K, a.cpu_seconds)
        cpu = {"value": g, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{n} time steps of the full {a.nx}x{a.ny} lattice ({dt:.1f} s), "
                         f"FP64 oracle, OpenMP over rows on {cpu_desc()}"}
    s.close()
    # single-GPU studies (skipped under torchrun, where only the scaling
    # measurement above is wanted)
    ttc = batch = formats = warm = swp = None
    if world == 1:
        formats = format_throughput(a, eps, K)
        if not a.no_ttc:
            ttc = time_to_converged(a)
        if not a.no_warm:
            warm = warm_start(a)
        if not a.no_batch:
            batch = batch_bench(a)
        if a.sweep > 0:
            swp = sweep(a)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": a.storage,
            "data": "synthetic (seeded Gaussian-random-field two-phase medium)",
            "config": workload(a),
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
            "gpu_launches": l1 - l0, "k_app": kapp,
            "storage_formats": formats,
            "time_to_converged": ttc,
            "warm_start": warm,
            "batch": batch,
        }
        if swp is not None:
            line["sweep"] = swp
        emit(line, a)
    return 0


def main():
    a = args_()
    world, rank, local = dist_setup()
    if a.impl == "reference":
        rc = run_reference(a, world, rank)
    else:
        rc = run_ours(a, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
