#!/usr/bin/env python
"""Benchmark of the ES-BGK kinetic stage update (coupled IMEX domain decomposition).

Workload (default): the precision-form configuration -- 256 x 256 periodic cells
on [0,1]^2, 48 x 48 velocities on [-8,8]^2, a Gaussian density blob on a uniform
flow, every cell kinetic, ARS(2,3,3), f stored in FP32 (six f-sized arrays of
604 MB: the stage kernel streams from HBM).  Beside it, the coupled
ES-BGK/Euler configuration (128 x 128 outflow cells, 32 x 32 velocities,
four-quadrant Riemann data, plain switch) under the key riemann_128x32.
A step is one full step of Algorithm 1 (regime update, three stages with
coupling, final combination).  Metric: kinetic (cell x velocity) stage updates
per second = sum over steps of K_kinetic * N_v^2 * (transport evaluations).

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                [--workload riemann|blob|sine|batch|learned|switchnet] [--prec fp32|fp64|bf16]
Under torchrun every rank runs an independent replica (seed = rank): weak
scaling, no collective on the data path.  Prints one JSON line on rank 0.
"""

import os

# the CPU oracle legs are timed single-threaded; say so in "cores"
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse  # noqa: E402
import hashlib  # noqa: E402
import json  # noqa: E402
import statistics  # noqa: E402
import subprocess  # noqa: E402
import sys  # noqa: E402
import time  # noqa: E402

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "kinetic (cell x velocity) stage updates/s"
UNIT = "updates/s"
# accesses of f-sized arrays per element per step, and transport evaluations
# per step (running-accumulator form of the IMEX step)
ACCESSES = {"ars233": (12, 3), "imex_euler": (2, 1)}
ELEM = {"fp64": 8, "fp32": 4, "bf16": 2}
DTYPE = {"fp64": "f64", "fp32": "f32", "bf16": "bf16-storage/f32"}


def make_workload(name, seed, nx=None):
    """The workload recipe; nx (blob only) shrinks the grid to nx x nx cells
    for profiling captures."""
    if name == "riemann":
        return W.riemann_quadrants(seed=seed)
    if name == "blob":
        return W.gaussian_blob() if nx is None else W.gaussian_blob(nx=nx, ny=nx)
    if name == "sine":
        return W.sine_periodic()
    raise SystemExit("unknown workload " + name)


def describe(wl, name, prec):
    g, v, p = wl["grid"], wl["vmesh"], wl["params"]
    return {"workload": "%s %dx%d cells, %dx%d velocities on [-%g,%g]^2, %s, %s switch" % (
        {"riemann": "four-quadrant Riemann ES-BGK/Euler", "blob": "Gaussian blob all-kinetic",
         "sine": "sine-periodic all-kinetic"}[name], g["nx"], g["ny"], v["nv"], v["nv"], v["vmax"], v["vmax"],
        wl["scheme"], p["switch"]),
        "nx": g["nx"], "ny": g["ny"], "nv": v["nv"], "scheme": wl["scheme"], "prec": prec,
        "switch": p["switch"], "dt": wl["dt"]}


def batch_workload(n):
    return ("batched form: %d independent periodic cases, N_x = N_y in 64..256, N_v in 16..40 on [-8,8]^2, "
            "eps log-uniform [1e-4,1e-1], plain switch, ARS(2,3,3)" % n)


LEARNED_WORKLOAD = ("learned switch: 512x512 cells, 32x32 velocities on [-8,8]^2, four-quadrant Riemann data plus "
                    "a density blob at (0.3, 0.7), learned switch, ARS(2,3,3)")
SWITCHNET_METRIC = "learned-switch network: cells per second (one Adam training step)"
SWITCHNET_WORKLOAD = "switch network: training batches of 32 x 128 x 128 cells; inference of one 512 x 512 image"


# ---------------------------------------------------------------------------
# CPU oracle sample (cpu_baseline and the reference arm)

def oracle_sample(name, steps, warmup=0):
    """Time the FP64 CPU oracle on a bounded sample of the workload: the same
    domain, velocity grid, scheme and data recipe on fewer cells (32 x 32 for
    the Riemann recipes).  The learned-switch workload is sampled with the
    paper's criterion (plain switch), the method the network assists.
    Returns (updates/s, description, per-step s)."""
    import oracle as O
    if name == "riemann":
        wl = W.riemann_quadrants(nx=32, ny=32, seed=0)
    elif name == "learned":
        wl = W.learned_switch_case(nx=32, ny=32, seed=0)
        wl["params"] = dict(wl["params"], switch="plain")
    elif name == "blob":
        wl = W.gaussian_blob(nx=16, ny=16)
    else:
        wl = W.sine_periodic()
    P = O.Problem(**wl["grid"], **wl["vmesh"], **wl["params"])
    tab = {"ars233": O.ARS233, "imex_euler": O.IMEX_EULER}[wl["scheme"]]
    nL = ACCESSES[wl["scheme"]][1]
    st = O.init_state(P, **wl["fields"])
    for _ in range(warmup):
        st = O.step(P, st, wl["dt"], tab)
    upd, per = 0, []
    for _ in range(steps):
        t0 = time.perf_counter()
        st = O.step(P, st, wl["dt"], tab)
        per.append(time.perf_counter() - t0)
        upd += int(st.kin.sum()) * P.nv * P.nv * nL
    g, v = wl["grid"], wl["vmesh"]
    desc = "FP64 numpy oracle, %d steps of the same configuration on %dx%d cells (%dx%d velocities), " \
           "single-threaded" % (steps, g["nx"], g["ny"], v["nv"], v["nv"])
    if name == "learned":
        desc += "; plain criterion (the oracle has the paper's switch, not the network)"
    return upd / sum(per), desc, per


def switchnet_oracle_sample(steps):
    """FP64 oracle of the switch network on a bounded sample of its training
    workload: Adam steps on batches of 2 images of 128 x 128 cells (the timed
    image size, 1/16 of its batch), random features and labels.  Returns
    (cells/s, description, per-step s)."""
    from oracle import cnn as C
    rng = np.random.default_rng(0)
    theta = C.init_params(0)
    m, v = np.zeros_like(theta), np.zeros_like(theta)
    x = rng.standard_normal((2, 128, 128, 5))
    y = (rng.random((2, 128, 128)) < 0.25).astype(np.float64)
    per = []
    for t in range(1, steps + 1):
        t0 = time.perf_counter()
        _, g = C.grad(theta, x, y, 3.0)
        theta, m, v = C.adam(theta, m, v, g, t, 1e-3)
        per.append(time.perf_counter() - t0)
    desc = ("FP64 numpy oracle of the switch network, %d Adam steps on batches of 2 x 128 x 128 cells "
            "(random features and labels), single-threaded" % steps)
    return x.shape[0] * 128 * 128 * steps / sum(per), desc, per


def _sample(kind, steps, warmup=0):
    """One bounded oracle sample of a workload kind (single process)."""
    if kind == "batch":
        return batch_oracle_sample(steps)
    if kind == "switchnet":
        return switchnet_oracle_sample(steps)
    return oracle_sample(kind, steps, warmup=warmup)


def _sample_worker(job):
    kind, steps, warmup = job
    t0 = time.perf_counter()
    val, desc, per = _sample(kind, steps, warmup)
    return val, desc, per, time.perf_counter() - t0


def oracle_all_cores(kind, steps, warmup=0, procs=None):
    """The oracle on every host core: one single-threaded process per core,
    each running the same bounded sample (independent copies of the sampled
    window, like the GPU's replicas).  Throughput = the work of all processes
    over the slowest process's timed steps.  The pool is started with 'spawn'
    (fresh interpreters that never touch the GPU).  Returns (value, desc,
    per-step seconds of process 0, cores)."""
    import multiprocessing as mp
    procs = procs or os.cpu_count() or 1
    with mp.get_context("spawn").Pool(procs) as pool:
        res = pool.map(_sample_worker, [(kind, steps, warmup)] * procs)
    per_proc = [sum(r[2]) for r in res]
    work = sum(r[0] * sum(r[2]) for r in res)  # each process's units = its rate x its timed seconds
    value = work / max(per_proc)
    desc = res[0][1].replace("single-threaded", "%d single-threaded processes (one per host core)" % procs)
    return value, desc, res[0][2], procs


def cpu_baseline(kind, steps):
    """cpu_baseline of a bench line: the oracle on all host cores, and on one."""
    unit = "cells/s" if kind == "switchnet" else UNIT
    v1, d1, _ = _sample(kind, steps)
    va, da, _, cores = oracle_all_cores(kind, steps)
    return {"value": va, "unit": unit, "cores": cores, "kind": "oracle", "sample": da,
            "single_core": {"value": v1, "cores": 1, "sample": d1}}


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    metric, unit = METRIC, UNIT
    if args.workload == "batch":
        cfg = {"workload": batch_workload(args.cases), "cases": args.cases, "prec": "fp64"}
    elif args.workload == "learned":
        cfg = {"workload": LEARNED_WORKLOAD, "prec": "fp64"}
    elif args.workload == "switchnet":
        metric, unit = SWITCHNET_METRIC, "cells/s"
        cfg = {"workload": SWITCHNET_WORKLOAD, "features": 5, "hidden": 32, "prec": "fp64"}
    else:
        cfg = describe(make_workload(args.workload, 0), args.workload, "fp64")
    val, desc, per, cores = oracle_all_cores(args.workload, args.steps,
                                             warmup=0 if args.workload in ("batch", "switchnet") else args.warmup)
    # the oracle runs the same recipe on a bounded window, named here
    cfg["sampled"] = desc
    out = {"metric": metric, "value": val, "unit": unit, "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * sum(per) / len(per), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": cfg, "impl": "reference",
           "cpu_baseline": {"value": val, "unit": unit, "cores": cores, "kind": "oracle", "sample": desc},
           "e2e": {"value": val, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# clocks during the timed region

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            time.sleep(0.3)  # sampling has started before the timed region does
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------

# the sources that define the stage kernels (the network, the host runtime and
# the criterion's kernels do not change their traffic)
STAGE_SOURCES = ("common.cuh", "kernels_impl.cuh", "tile_impl.cuh", "launch.h", "kernels_f32.cu", "kernels_f64.cu",
                 "kernels_bf16.cu", "kernels_f32_sums.cu", "kernels_bf16_sums.cu")


def source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2512_03586_gb300", "csrc")
    for f in STAGE_SOURCES:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def measured_peak():
    try:
        m = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(m["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, STREAM-style copy)"
    except Exception:
        return 6800.0, "fallback 6.8 TB/s"


def stored_traffic(prec, workload):
    """DRAM bytes per kinetic element-evaluation of the stage kernel from the
    committed ncu summary, if it was taken on the current kernel sources."""
    p = os.path.join(ROOT, "profiles", "stage_kernel_traffic.json")
    try:
        d = json.load(open(p))
        e = d["entries"]["%s/%s" % (workload, prec)]
        if e["source_hash"] != source_hash():
            return None
        return float(e["dram_bytes_per_element_eval"])
    except Exception:
        return None


def combine_ranks(ms, updates, device, world):
    """Whole-job figures of independent replicas: the slowest rank's time and
    the sum of every rank's updates (the only collectives of a run; the data
    path has none)."""
    if world <= 1:
        return ms, float(updates)
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms, float(updates)], dtype=torch.float64, device=device)
    mx = t.clone()
    dist.all_reduce(mx[:1], op=dist.ReduceOp.MAX)
    dist.all_reduce(t[1:], op=dist.ReduceOp.SUM)
    return float(mx[0]), float(t[1])


def _measure(G, args, name, prec, steps, warmup, dev, world, local, rank, barrier, cpu_steps=0):
    """Time `steps` steps of workload `name` on this rank's replica (seed =
    rank): the device-timed line, the stage kernel's roofline, the end-to-end
    figure through the C ABI and the clock record."""
    import torch
    wl = make_workload(name, rank, nx=args.nx if name == args.workload else None)
    f = wl["fields"]
    # a non-default stream: repeated steps replay as CUDA graphs
    torch.cuda.set_stream(torch.cuda.Stream(dev))
    s = G.Solver(wl["grid"], wl["vmesh"], wl["params"], prec=prec, device=dev)
    s.set_state(f["rho"], f["ux"], f["uy"], f["T"], f["eps"], f["kin"])
    tab = G.make_tableau(wl["scheme"])
    dt = wl["dt"]
    nvv = wl["vmesh"]["nv"] ** 2
    acc, nL = ACCESSES[wl["scheme"]]
    ebytes = ELEM[prec]
    for _ in range(warmup):
        s.step(dt, tab)
    s.sync()
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)

    # --- timed region: K steps, L2 flushed before each (outside the events)
    c0 = s.counters()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        for k in range(steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            s.step(dt, tab)
            ev[k][1].record(stream)
        torch.cuda.synchronize(dev)
        barrier()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    s.sync()
    c1 = s.counters()
    updates = (c1["kinetic_cell_updates"] - c0["kinetic_cell_updates"]) * nvv
    fills_timed = c1["buffer_fills"] - c0["buffer_fills"]
    ms_max, updates_all = combine_ranks(ms, float(updates), dev, world)
    value = updates_all / (ms_max * 1e-3)
    # algorithmic bytes of the timed steps (all stage launches) over the whole step time
    step_bytes = updates * (acc / nL) * ebytes + fills_timed * nvv * ebytes

    # --- per-kernel device times: the same steps as plain launches (no graph),
    # an event pair around every launch on the launching stream
    k2 = max(3, min(steps, 20))
    s.timing(True)
    s.timing_read()
    cb = s.counters()
    for k in range(k2):
        flush.fill_(float(k))
        s.step(dt, tab)
    tk = s.timing_read()
    s.timing(False)
    ca = s.counters()
    evals = ca["kinetic_cell_updates"] - cb["kinetic_cell_updates"]
    fills = ca["buffer_fills"] - cb["buffer_fills"]
    st_ms = tk["stage"][0] + tk["final"][0]
    st_n = tk["stage"][1] + tk["final"][1]
    algo_bytes = evals * nvv * (acc / nL) * ebytes + fills * nvv * ebytes
    achieved = algo_bytes / (st_ms * 1e-3) / 1e9 if st_ms > 0 else None
    peak, peak_src = measured_peak()
    tr = stored_traffic(prec, name)
    launches_per_step = (tk["l1"][1] + tk["flags"][1] + 2 * tk["compact"][1] + tk["prep"][1] + tk["stage"][1]
                         + tk["final"][1]) / k2
    step_ms_kernels = sum(v[0] for v in tk.values()) / k2

    # --- end to end through the C ABI with pinned host buffers
    nc = s.nc
    pin = {k: torch.empty(nc, dtype=torch.float64).pin_memory().numpy() for k in ("rho", "ux", "uy", "T", "eps")}
    mom = s.moments()
    for q, k in enumerate(("rho", "ux", "uy", "T")):
        pin[k][:] = mom[q].reshape(-1)
    pin["eps"][:] = f["eps"].reshape(-1)
    kin = torch.empty(nc, dtype=torch.uint8).pin_memory().numpy()
    kin[:] = s.flags().reshape(-1)
    outp = torch.empty((4, nc), dtype=torch.float64).pin_memory().numpy()
    k3 = max(3, min(steps, 10))
    e0 = s.counters()["kinetic_cell_updates"]
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(k3):
        s.set_state(pin["rho"], pin["ux"], pin["uy"], pin["T"], pin["eps"], kin)
        s.step(dt, tab)
        s.moments(out=outp)
    t_e2e = time.perf_counter() - t0
    e_upd = (s.counters()["kinetic_cell_updates"] - e0) * nvv
    kin_frac = c1["kinetic_cells"] / nc
    s.close()
    del flush

    cfg = describe(wl, name, prec)
    cfg.update({"l2": "flushed (256 MB write) before every timed step, outside the step's events",
                "parallelism": "replicas" if world > 1 else "single GPU",
                "kinetic_fraction_end": kin_frac, "kernel_launches_per_step": launches_per_step})
    return {"value": value, "ms_per_step": ms_max / steps, "config": cfg,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": (achieved / peak) if achieved else None,
                         "traffic": (tr * evals * nvv / st_n) if (tr is not None and st_n) else None,
                         "kernel": "stage_kernel (fused IMEX stage + final combination)",
                         "algorithmic_bytes_per_launch": algo_bytes / st_n if st_n else None,
                         "avg_launch_ms": st_ms / st_n if st_n else None,
                         "stage_ms_per_step": st_ms / k2, "peak_source": peak_src,
                         "bytes_model": "%d f-array accesses per element per step / %d transport evaluations x %d B,"
                                        " plus one write per buffer-cell element reconstructed" % (acc, nL, ebytes),
                         "timing": "avg_launch_ms from CUDA events around each stage launch on its stream, in "
                                   "plain launches of the same steps right after the timed region",
                         "whole_step": {"achieved": step_bytes / (ms * 1e-3) / 1e9 if ms > 0 else None,
                                        "frac": step_bytes / (ms * 1e-3) / 1e9 / peak if ms > 0 else None,
                                        "note": "algorithmic bytes of the timed steps' stage launches divided by "
                                                "the whole timed step (every other launch of the step included)"}},
            "kernel_ms_per_step": {k: v[0] / k2 for k, v in tk.items()},
            "kernel_sum_ms_per_step": step_ms_kernels,
            "e2e": {"value": e_upd / t_e2e, "unit": UNIT, "h2d_bytes_per_step": 5 * nc * 8 + nc,
                    "d2h_bytes_per_step": 4 * nc * 8,
                    "note": "each step: esbgk_set_state from pinned host arrays, which restarts the run from "
                            "the macroscopic state and regime map (f rebuilt as the projected Maxwellian of U in "
                            "kinetic cells), then esbgk_step, then esbgk_get_moments to pinned host arrays"},
            "clocks": clk.summary(), "gpu_launches": int(round(launches_per_step * steps))}


def ours_arm(args):
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import paper_2512_03586_gb300 as G

    def barrier():
        if world > 1:
            dist.barrier()

    m = _measure(G, args, args.workload, args.prec, args.steps, args.warmup, dev, world, local, rank, barrier)
    extra = None
    if args.workload == "blob" and not args.no_extra:
        # the coupled Riemann configuration (128^2 cells, 32^2 velocities, plain switch) beside the headline
        r = _measure(G, args, "riemann", args.prec, 50, args.warmup, dev, world, local, rank, barrier)
        extra = {"value": r["value"], "unit": UNIT, "ms_per_step": r["ms_per_step"], "steps": 50,
                 "config": r["config"], "roofline": r["roofline"], "e2e": r["e2e"], "clocks": r["clocks"],
                 "kernel_ms_per_step": r["kernel_ms_per_step"]}
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    out = {"metric": METRIC, "value": m["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": m["ms_per_step"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[args.prec], "data": "synthetic",
           "config": m["config"], "roofline": m["roofline"], "kernel_ms_per_step": m["kernel_ms_per_step"],
           "kernel_sum_ms_per_step": m["kernel_sum_ms_per_step"], "e2e": m["e2e"], "clocks": m["clocks"],
           "gpu_launches": m["gpu_launches"]}
    if extra:
        out["riemann_128x32"] = extra
    if not args.no_cpu_baseline and world == 1:
        out["cpu_baseline"] = cpu_baseline(args.workload, args.cpu_steps)
    print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def batch_oracle_sample(steps):
    """FP64 oracle on a bounded sample of the batched workload: one case of
    the same recipe on 32 x 32 cells with N_v = 28 (the mean of 16..40)."""
    import oracle as O
    wl = W.batched_cases(n_cases=1, seed0=0, sizes=[32], nvs=[28])[0]
    P = O.Problem(**wl["grid"], **wl["vmesh"], **wl["params"])
    st = O.init_state(P, **wl["fields"])
    upd, per = 0, []
    for _ in range(steps):
        t0 = time.perf_counter()
        st = O.step(P, st, wl["dt"], O.ARS233)
        per.append(time.perf_counter() - t0)
        upd += int(st.kin.sum()) * P.nv * P.nv * 3
    desc = "FP64 numpy oracle, %d ARS(2,3,3) steps of one batched-recipe case on 32x32 cells, 28x28 " \
           "velocities, plain switch, single-threaded" % steps
    return upd / sum(per), desc, per


def batch_arm(args):
    """Batched form: 64 independent cases (uneven grids and velocity meshes)
    advanced by one launch per kernel, replayed as a CUDA graph."""
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_2512_03586_gb300 as G

    def barrier():
        if world > 1:
            dist.barrier()

    cases = W.batched_cases(n_cases=args.cases, seed0=rank * args.cases)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    b = G.BatchSolver([(c["grid"], c["vmesh"], c["params"]) for c in cases], prec=args.prec, device=dev,
                      stream=stream)
    for i, c in enumerate(cases):
        f = c["fields"]
        b.set_state(i, f["rho"], f["ux"], f["uy"], f["T"], f["eps"], f["kin"])
    dts = np.array([c["dt"] for c in cases])
    tab = G.make_tableau("ars233")
    threads, ctas = b.autotune(dts, tab)
    sched = b.schedule()
    for _ in range(args.warmup):
        b.step(dts, tab)
    b.sync()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    c0 = b.counters()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            b.step(dts, tab)
            ev[k][1].record(stream)
        torch.cuda.synchronize(dev)
        barrier()
    ms = sum(a.elapsed_time(e) for a, e in ev)
    b.sync()
    c1 = b.counters()
    updates = (c1["element_updates"] - c0["element_updates"]) * 1.0
    ms_max, updates_all = combine_ranks(ms, updates, dev, world)
    value = updates_all / (ms_max * 1e-3)

    # per-kernel device times (plain launches with events)
    k2 = max(3, min(args.steps, 10))
    b.timing(True)
    b.timing_read()
    cb = b.counters()
    for k in range(k2):
        flush.fill_(float(k))
        b.step(dts, tab)
    tk = b.timing_read()
    b.timing(False)
    ca = b.counters()
    el = ca["element_updates"] - cb["element_updates"]
    ebytes = ELEM[args.prec]
    st_ms = tk["stage"][0] + tk["final"][0]
    st_n = tk["stage"][1] + tk["final"][1]
    algo_bytes = el * (12 / 3) * ebytes
    achieved = algo_bytes / (st_ms * 1e-3) / 1e9 if st_ms > 0 else None
    peak, peak_src = measured_peak()
    # launches per step: l1 offsets + l1 + flags, categorize + compact + offsets, prep, stages
    launches_per_step = 3 + 3 + 1 + (tk["stage"][1] + tk["final"][1]) / k2

    # end to end: every case's state from pinned host memory, one step, every case's moments back
    pins = []
    for i, c in enumerate(cases):
        nx, ny = c["grid"]["nx"], c["grid"]["ny"]
        m = b.moments(i)
        arr = torch.empty((5, nx * ny), dtype=torch.float64).pin_memory().numpy()
        arr[:4] = m.reshape(4, -1)
        arr[4] = c["fields"]["eps"].reshape(-1)
        kin = torch.empty(nx * ny, dtype=torch.uint8).pin_memory().numpy()
        kin[:] = b.flags(i).reshape(-1)
        outp = torch.empty((4, ny, nx), dtype=torch.float64).pin_memory().numpy()
        pins.append((arr, kin, outp))
    k3 = 3
    e0 = b.counters()["element_updates"]
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(k3):
        for i, (arr, kin, _o) in enumerate(pins):
            b.set_state(i, arr[0], arr[1], arr[2], arr[3], arr[4], kin)
        b.step(dts, tab)
        for i, (_a, _k, outp) in enumerate(pins):
            b.moments(i, out=outp)
    t_e2e = time.perf_counter() - t0
    e_upd = b.counters()["element_updates"] - e0
    ncells = sum(c["grid"]["nx"] * c["grid"]["ny"] for c in cases)
    elems = sum(c["grid"]["nx"] * c["grid"]["ny"] * c["vmesh"]["nv"] ** 2 for c in cases)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline("batch", max(2, args.cpu_steps // 4))
    cfg = {"workload": batch_workload(len(cases)),
           "cases": len(cases), "cells": ncells, "elements": elems, "prec": args.prec,
           "l2": "flushed (256 MB write) before every timed step; f arrays far exceed L2",
           "parallelism": "replicas" if world > 1 else "single GPU",
           "autotuned": {"threads": threads, "ctas_per_sm": ctas,
                                     "per_cell_form_by_nv": {str(k): v for k, v in sched["forms"].items()}}, "cuda_graph": True,
           "kinetic_fraction_end": c1["kinetic_cells"] / ncells}
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[args.prec], "data": "synthetic", "config": cfg,
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": (achieved / peak) if achieved else None, "traffic": None,
                        "kernel": "batch_stage_kernel (all cases, fused IMEX stage + final combination; one "
                                  "launch per per-cell form present, timed together per stage)",
                        "algorithmic_bytes_per_launch": algo_bytes / st_n if st_n else None,
                        "avg_launch_ms": st_ms / st_n if st_n else None, "peak_source": peak_src,
                        "bytes_model": "12 f-array accesses per element per step / 3 transport evaluations x %d B"
                                       % ebytes},
           "kernel_ms_per_step": {k: v[0] / k2 for k, v in tk.items()},
           "e2e": {"value": e_upd / t_e2e, "unit": UNIT,
                   "h2d_bytes_per_step": sum(5 * 8 * c["grid"]["nx"] * c["grid"]["ny"] + c["grid"]["nx"] * c["grid"]["ny"]
                                             for c in cases),
                   "d2h_bytes_per_step": 4 * 8 * ncells,
                   "note": "each step: esbgk_batch_set_state of every case from pinned host arrays, "
                           "esbgk_batch_step, esbgk_batch_get_moments of every case to pinned host arrays"},
           "clocks": clk.summary(), "gpu_launches": int(round(launches_per_step * args.steps))}
    if cpu:
        out["cpu_baseline"] = cpu
    print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def learned_arm(args):
    """Learned switch (deployment config): train the network on plain-criterion
    histories of the four-quadrant Riemann recipe (128 x 128 cells, 32 x 32
    velocities, 48 seeds) and of the deployment recipe on its 512 x 512 grid
    (3 other seeds, cut into 128 x 128 tiles), deploy it on 512 x 512 cells
    (Riemann data plus a density blob) in FP32, and compare with the plain
    criterion in FP32 and in FP64 on wall-clock per simulated time and on the
    macroscopic error against an all-kinetic FP32 run of the same problem."""
    import torch
    import paper_2512_03586_gb300 as G
    from paper_2512_03586_gb300 import switch_train as T
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    t0 = time.perf_counter()
    train_cases = [W.riemann_quadrants(nx=128, ny=128, nv=32, seed=1000 + s, steps=args.train_steps)
                   for s in range(args.train_seeds)]
    X, Y = T.collect(train_cases, steps=args.train_steps, prec="fp32", device=dev)
    # plus histories of the deployment recipe on its own grid (other seeds), cut into 128 x 128 tiles
    fine = [W.learned_switch_case(seed=2000 + s, steps=args.train_steps) for s in range(3)]
    for c in fine:
        c["params"] = dict(c["params"], switch="plain")
    Xf, Yf = T.collect(fine, steps=args.train_steps, prec="fp32", device=dev)
    Xf, Yf = T.crop(Xf, Yf, 128)
    X, Y = torch.cat([X, Xf]), torch.cat([Y, Yf])
    del Xf, Yf
    t_collect = time.perf_counter() - t0
    # one network per initialisation seed, same data; seed 0's is timed below
    nets = []
    for seed in range(args.init_seeds):
        t0 = time.perf_counter()
        th, hi = T.train(X, Y, T.init_params(seed), epochs=30, batch=32, lr=3e-3, device=dev)
        torch.cuda.synchronize(dev)
        nets.append((th, hi, time.perf_counter() - t0))
    theta, hist, t_train = nets[0]
    del X, Y

    wl = W.learned_switch_case(seed=rank)
    f = wl["fields"]
    dt, nsim = wl["dt"], args.sim_steps
    tab = G.make_tableau(wl["scheme"])
    nvv = wl["vmesh"]["nv"] ** 2

    def make(switch, prec, kin=None, params=None):
        s = G.Solver(wl["grid"], wl["vmesh"], dict(wl["params"], switch=switch), prec=prec, device=dev)
        s.set_state(f["rho"], f["ux"], f["uy"], f["T"], f["eps"], f["kin"] if kin is None else kin)
        if switch == "learned":
            s.set_switch_params(theta if params is None else params)
        return s

    def run(s, n):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0 = s.counters()
        stream = torch.cuda.current_stream(dev)
        torch.cuda.synchronize(dev)
        ev0.record(stream)
        for _ in range(n):
            s.step(dt, tab)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        s.sync()
        c1 = s.counters()
        return ev0.elapsed_time(ev1), (c1["kinetic_cell_updates"] - c0["kinetic_cell_updates"]) * nvv

    ref = make("frozen", "fp32", kin=np.ones_like(f["kin"]))
    run(ref, nsim)
    Uref = ref.cons()
    ref.close()
    err = lambda U: float(np.abs(U - Uref).sum() / np.abs(Uref).sum())
    res = {}
    for name, sw, prec in (("plain_fp64", "plain", "fp64"), ("plain_fp32", "plain", "fp32"),
                           ("learned_fp32", "learned", "fp32")):
        s = make(sw, prec)
        ms, upd = run(s, nsim)
        res[name] = {"ms_per_sim_time": ms / (nsim * dt), "ms_per_step": ms / nsim, "updates_per_s": upd / (ms * 1e-3),
                     "error_vs_all_kinetic": err(s.cons()), "kinetic_cell_steps": upd // nvv // 3}
        if sw == "learned":
            res[name]["judge"] = s.switch_stats()
            s.timing(True)
            s.timing_read()
            for _ in range(5):
                s.step(dt, tab)
            tk = s.timing_read()
            s.timing(False)
            res[name]["network_ms_per_step"] = tk["other"][0] / 5
            res[name]["criterion_ms_per_step"] = (tk["l1"][0] + tk["flags"][0]) / 5
            # kernels per step: l1, flags, 5 of the network (features, two convolutions, head, judge),
            # categorize + compact, prep, stages and final combination
            launches_per_step = (tk["l1"][1] + tk["flags"][1] + 5 * tk["other"][1] + 2 * tk["compact"][1]
                                 + tk["prep"][1] + tk["stage"][1] + tk["final"][1]) / 5
            learned = s
        else:
            s.close()
    # the networks of the other initialisation seeds, against plain FP32 (same precision)
    p32 = res["plain_fp32"]
    seeds = []
    for seed, (th, hi, tt) in enumerate(nets):
        if seed == 0:
            r = res["learned_fp32"]
        else:
            s = make("learned", "fp32", params=th)
            ms, upd = run(s, nsim)
            r = {"ms_per_sim_time": ms / (nsim * dt), "error_vs_all_kinetic": err(s.cons()),
                 "kinetic_cell_steps": upd // nvv // 3}
            s.close()
        seeds.append({"init_seed": seed, "final_loss": hi[-1], "train_s": tt,
                      "wall_per_sim_time_vs_plain_fp32": r["ms_per_sim_time"] / p32["ms_per_sim_time"],
                      "error_vs_plain_fp32": r["error_vs_all_kinetic"] / p32["error_vs_all_kinetic"],
                      "kinetic_work_vs_plain_fp32": r["kinetic_cell_steps"] / max(p32["kinetic_cell_steps"], 1)})

    # the combined form: learned switch + FP32 storage + batched form, four
    # copies of the deployment case in one batch (a batch equals its single
    # runs to rounding, so case 0's error is the learned run's)
    nb = args.batch_cases
    bstream = torch.cuda.Stream(dev)
    with torch.cuda.stream(bstream):
        bs = G.BatchSolver([(wl["grid"], wl["vmesh"], dict(wl["params"], switch="learned"))] * nb, prec="fp32",
                           device=dev, stream=bstream)
        for i in range(nb):
            bs.set_state(i, f["rho"], f["ux"], f["uy"], f["T"], f["eps"], f["kin"])
            bs.set_switch_params(i, theta)
        dts = np.full(nb, dt)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(bstream)
        for _ in range(nsim):
            bs.step(dts, tab)
        e1.record(bstream)
        torch.cuda.synchronize(dev)
        bs.sync()
        bms = e0.elapsed_time(e1)
        berr = err(bs.cons(0))
        del bs
    per_case = bms / nb / (nsim * dt)
    combined = {"cases": nb, "ms_per_step": bms / nsim, "ms_per_sim_time_per_case": per_case,
                "error_vs_all_kinetic_case0": berr,
                "wall_per_sim_time_vs_plain_fp64": per_case / res["plain_fp64"]["ms_per_sim_time"],
                "error_vs_plain_fp64": berr / res["plain_fp64"]["error_vs_all_kinetic"],
                "wall_per_sim_time_vs_learned_fp32_single": per_case / res["learned_fp32"]["ms_per_sim_time"]}

    # timed region of the line: K steps of the learned FP32 form, L2 flushed between steps
    for _ in range(args.warmup):
        learned.step(dt, tab)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    c0 = learned.counters()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            learned.step(dt, tab)
            ev[k][1].record(stream)
        torch.cuda.synchronize(dev)
    ms = sum(a.elapsed_time(b) for a, b in ev)
    c1 = learned.counters()
    value = (c1["kinetic_cell_updates"] - c0["kinetic_cell_updates"]) * nvv / (ms * 1e-3)
    if rank != 0:
        return
    p64, l32 = res["plain_fp64"], res["learned_fp32"]
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32", "data": "synthetic",
           "config": {"workload": LEARNED_WORKLOAD, "prec": "fp32",
                      "training": "%d Riemann seeds x %d steps at 128x128 / 32x32 plus 3 seeds of this recipe at "
                                  "512x512 cut into 128x128 tiles (plain criterion labels, next step), 30 epochs "
                                  "Adam; collect %.1f s, train %.1f s, final loss %.4f" % (
                                      args.train_seeds, args.train_steps, t_collect, t_train, hist[-1]),
                      "comparison_steps": nsim,
                      "l2": "flushed (256 MB write) before every timed step"},
           "comparison": res,
           "learned_fp32_vs_plain_fp64": {"wall_per_sim_time_ratio": l32["ms_per_sim_time"] / p64["ms_per_sim_time"],
                                          "error_ratio": l32["error_vs_all_kinetic"] / p64["error_vs_all_kinetic"]},
           "learned_fp32_vs_plain_fp32_by_init_seed": seeds,
           "learned_fp32_batched_vs_plain_fp64": combined,
           "learned_fp32_vs_plain_fp32_spread": {
               k: [min(x[k] for x in seeds), max(x[k] for x in seeds)]
               for k in ("wall_per_sim_time_vs_plain_fp32", "error_vs_plain_fp32", "kinetic_work_vs_plain_fp32")},
           "clocks": clk.summary(), "gpu_launches": int(round(launches_per_step * args.steps))}
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline("learned", args.cpu_steps)
    print(json.dumps(out), flush=True)


def switchnet_arm(args):
    """Kernels of the learned switch alone: inference of one 512 x 512 image
    (the deployment grid) and Adam training steps on batches of 32 images of
    128 x 128 cells, random features and labels.  Roofline of the dominant
    kernel (the 32 -> 32 channel 3 x 3 convolution) against the measured bf16
    tensor peak."""
    import torch
    import paper_2512_03586_gb300 as G
    from paper_2512_03586_gb300 import switch_train as T
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if int(os.environ.get("RANK", "0")) != 0:
        return
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    gen = torch.Generator(device=dev).manual_seed(0)

    def feats(n, H, Wd):
        x = torch.zeros((n, H, Wd, G.CNN_CHANNELS), dtype=torch.bfloat16, device=dev)
        x[..., :5] = torch.randn((n, H, Wd, 5), generator=gen, device=dev).to(torch.bfloat16)
        return x

    theta = T.init_params(0)
    n_tr, Ht = 32, 128
    net = G.SwitchNet(n_tr, Ht, Ht, device=dev)
    net.set_params(theta)
    xt = feats(n_tr, Ht, Ht)
    yt = (torch.rand((n_tr, Ht, Ht), generator=gen, device=dev) < 0.25).to(torch.uint8)
    inf = G.SwitchNet(1, 512, 512, device=dev)
    inf.set_params(theta)
    xi = feats(1, 512, 512)
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        net.train_step(xt, yt, 3.0, 1e-3)
        inf.forward(xi)
    torch.cuda.synchronize(dev)

    def timed(fn, k):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / k

    # at least ~0.4 s of timed work per figure, so that the clock record has samples
    est_tr = timed(lambda: net.train_step(xt, yt, 3.0, 1e-3), 3)
    est_inf = timed(lambda: inf.forward(xi), 3)
    k_tr = max(args.steps, int(400.0 / max(est_tr, 1e-3)))
    k_inf = max(args.steps, int(400.0 / max(est_inf, 1e-3)))
    with ClockSampler(local) as clk:
        ms_train = timed(lambda: net.train_step(xt, yt, 3.0, 1e-3), k_tr)
        ms_inf = timed(lambda: inf.forward(xi), k_inf)
        # the 32 -> 32 convolution alone, through the forward pass of one image
        ms_fwd = ms_inf
    cells_tr, cells_inf = n_tr * Ht * Ht, 512 * 512
    # algorithmic flops per cell: conv1 2*32*45, conv2 2*32*288, head 2*32
    f_fwd = 2 * 32 * 45 + 2 * 32 * 288 + 2 * 32
    f_train = f_fwd + 2 * 32 * 288 * 2 + 2 * 32 * 45  # + input and weight gradients of conv2, weight gradient of conv1
    try:
        m = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        peak, src = float(m["bf16_tflops"]), "measured (MEASURED_PEAKS.json bf16_tflops, cuBLAS burst)"
    except Exception:
        peak, src = 1900.0, "fallback 1.9 PFLOP/s"
    tf_inf = cells_inf * f_fwd / (ms_fwd * 1e-3) / 1e12
    out = {"metric": SWITCHNET_METRIC, "value": cells_tr / (ms_train * 1e-3),
           "unit": "cells/s", "n_gpus": 1, "steps": k_tr, "warmup": args.warmup, "ms_per_step": ms_train,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16 operands / f32 accumulation",
           "data": "synthetic", "config": {"workload": SWITCHNET_WORKLOAD, "features": 5, "hidden": 32},
           "inference": {"ms": ms_inf, "cells_per_s": cells_inf / (ms_inf * 1e-3)},
           "roofline": {"bound": "tensor", "achieved": tf_inf, "peak": peak, "unit": "TFLOP/s", "frac": tf_inf / peak,
                        "traffic": None, "kernel": "forward pass (5->32 convolution on mma.sync, 32->32 convolution "
                                                   "on tcgen05.mma with a tensor-memory accumulator, head), "
                                                   "512 x 512 cells", "peak_source": src,
                        "flops_model": "%d flops per cell (2 x 32 x 45 + 2 x 32 x 288 + 2 x 32)" % f_fwd},
           "train_tflops": cells_tr * f_train / (ms_train * 1e-3) / 1e12,
           "clocks": clk.summary(),
           # per training step: two convolutions, head, head reduction, weight gradient and its reduction
           # (twice), input-gradient convolution, Adam = 10; per inference: two convolutions and the head
           "gpu_launches": k_tr * 10 + k_inf * 3}
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline("switchnet", 3)
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="blob", choices=["riemann", "blob", "sine", "batch", "learned", "switchnet"])
    ap.add_argument("--train-seeds", type=int, default=48)
    ap.add_argument("--train-steps", type=int, default=30)
    ap.add_argument("--sim-steps", type=int, default=100, help="steps of the learned-switch comparison runs")
    ap.add_argument("--init-seeds", type=int, default=3, help="networks trained from these many initialisations")
    ap.add_argument("--batch-cases", type=int, default=4, help="cases of the batched learned-switch comparison")
    ap.add_argument("--cases", type=int, default=64, help="cases of the batched workload")
    ap.add_argument("--prec", default="fp32", choices=["fp32", "fp64", "bf16"])
    ap.add_argument("--cpu-steps", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--nx", type=int, default=None, help="blob workload on nx x nx cells (profiling captures)")
    ap.add_argument("--no-extra", action="store_true", help="skip the coupled Riemann line beside the headline")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        reference_arm(args)
    elif args.workload == "batch":
        batch_arm(args)
    elif args.workload == "learned":
        learned_arm(args)
    elif args.workload == "switchnet":
        switchnet_arm(args)
    else:
        ours_arm(args)


if __name__ == "__main__":
    main()
