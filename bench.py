#!/usr/bin/env python3
"""Benchmark of the SC-LBM hot path on GB300.

Headline workload: the large synthetic urban ensemble (512x256x128 cells, 96
seeded buildings, three uncertain inputs -- speed error, power-law exponent,
wind angle -- on the level-4 Clenshaw-Curtis Smolyak grid, 69 nodes,
BGK + Smagorinsky, FP32 shifted populations, 88 GB of populations).  One
benchmark step = `--lbm-steps` (default 100) stream-collide time steps of all
69 nodes followed by the FP64 quadrature reduction to mean / std / gPC fields
and the 95% profile bands; the full 10000-step run is 100 benchmark steps
(`full_run_s` extrapolates it from the timed steps).

value      ensemble GLUPS = cells x nodes x time steps / seconds (device time,
           inputs resident), whole job over all ranks.
e2e        the same metric through the C ABI with host buffers over the same
           number of steps: per step sc_lbm_init from pinned host geometry
           (H2D), the time steps, and sc_lbm_moments into pinned host outputs
           (D2H).
roofline   the stream-collide kernels: algorithmic bytes (152 B per fluid
           cell update in FP32, 19 reads + 19 writes) per time step over the
           average time-step duration (CUDA events on the library's stream),
           against the measured HBM copy bandwidth.
Extra keys: the plain one-node-at-a-time FP64 GPU path on the same domain,
the 256x128x64 13-node LES ensemble and the three-domain batched ensemble
(FP32 and BF16 storage, autotuned) with the error of their mean / std fields
against the FP64 path, BF16 / FP16 storage, the paper's collision, an hourly
inflow series, the paper's case at full size, the adjoint, and the FP64 CPU
oracle on the host cores (cpu_baseline: all cores and one thread).

Under torchrun the collocation nodes are sharded over the ranks (contiguous
node ranges); each benchmark step ends with the all-reduce of the FP64
moment sums and the finishing kernel (`parallelism: "nodes"`).

`--impl reference` times the FP64 CPU oracle on a bounded sample of the same
workload instead (the method has no other reference implementation).
"""
import argparse
import hashlib
import json
import os
import platform
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ensemble GLUPS & %HBM roofline, batched FP32 vs plain FP64; adjoint s/gradient"
HEADLINE = "urban_large_512x256x128_cc4"
BYTES_PER_LUP = {1: 152, 2: 76, 3: 76, 0: 304}
DTYPE = {1: "f32", 2: "bf16-storage/f32", 3: "f16-storage/f32", 0: "f64"}
DEFAULT_LBM_STEPS = {HEADLINE: 100, "urban_les_256x128x64_cc3": 500, "urban_batched_3domains": 200}
LEGS = "plain,cpu,e2e,les,batched,storage,rr,series,paper,adjoint,tune"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--lbm-steps", type=int, default=0,
                    help="time steps per benchmark step (0: 100 for the headline workload)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16", "fp16"])
    ap.add_argument("--workload", default=HEADLINE,
                    choices=[HEADLINE, "urban_les_256x128x64_cc3", "urban_batched_3domains",
                             "urban_les_rr_256x128x64_cc3", "urban_gh121_256x128x64_rr",
                             "urban_disk_540x540x40_gh121"],
                    help="the benchmark workload; the extra legs run with the headline workload only")
    ap.add_argument("--nodes", type=int, default=0,
                    help="profiling case: a coarser Smolyak level (fewer nodes), same domain (0 = as defined)")
    ap.add_argument("--skip", default="", help="comma list of extra legs to skip: " + LEGS)
    ap.add_argument("--tuning", default="",
                    help="fixed launch shape block_x,block_y,slab_z,tile_order,exec_mode,graph_steps,variant "
                         "instead of the autotuner")
    ap.add_argument("--leg", default="",
                    help="run only this extra leg (plain, les, batched, rr, series, paper, adjoint) and print its "
                         "result (profiling runs)")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash():
    """Hash of the stream-collide kernels' code (comments and whitespace
    removed, so that a recorded traffic figure follows the code only)."""
    import re
    h = hashlib.sha256()
    for f in ("lbm_kernels.cu", "lbm_device.cuh", "sclbm_internal.h"):
        with open(os.path.join(ROOT, "paper_2508_18202_gb300", "csrc", f)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def tuning_key(t):
    return ",".join(str(t[k]) for k in ("block_x", "block_y", "slab_z", "tile_order", "exec_mode",
                                        "graph_steps", "variant"))


def recorded_traffic(kernel_hash, workload, tuning):
    """DRAM bytes per time step from the committed ncu summary, if it was taken
    on the current kernel source in the same launch shape."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        e = d.get(workload)
        if e and e.get("kernel_hash") == kernel_hash and e.get("tuning") == tuning_key(tuning):
            return float(e["dram_bytes_per_time_step"])
    except Exception:
        pass
    return None


def host_info():
    model = platform.machine()
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"nproc": os.cpu_count(), "cpu": model, "arch": platform.machine()}


class Clocks:
    """nvidia-smi samples of the SM clock and throttle reasons during the
    timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def workload_named(name):
    from paper_2508_18202_gb300 import workloads as W
    return dict({w["name"]: w for w in W.ALL}[name])


def workload_for(args):
    from paper_2508_18202_gb300 import workloads as W
    wl = workload_named(args.workload)
    wl["precision"] = {"fp32": W.FP32_SHIFT, "bf16": W.BF16_STORE, "fp16": W.FP16_STORE}[args.precision]
    if args.nodes:
        # profiling case: a coarser sparse grid (fewer nodes), same domain
        wl["domains"] = [dict(wl["domains"][0], quad_level=args.nodes)]
    return wl


# ------------------------------------------------------------------ CPU oracle
class OracleNode:
    """One collocation node of a workload on the FP64 oracle, set up once
    (geometry, inflow table, equilibrium start); run(k) advances it k time
    steps and returns the seconds taken."""

    def __init__(self, wl, threads=None):
        from oracle import oracle as O
        self.O = O
        self.threads = O.set_threads(threads or os.cpu_count() or 1)
        D = wl["domains"][0]
        self.cells = D["nx"] * D["ny"] * D["nz"]
        self.p = O.params(D["nx"], D["ny"], D["nz"], D["bc"], wl["tau0"], wl["c_smag"], wl["ramp_steps"],
                          collision=wl.get("collision", 0))
        self.flags = O.geometry(D["nx"], D["ny"], D["nz"], D.get("seed", 0), D.get("n_buildings", 0),
                                *D.get("fp", (1, 1)), *D.get("h", (1, 1)), boxes=D.get("boxes"),
                                disk_radius=D.get("disk_radius", 0.0))
        Z, a = O.quadrature(wl["quad_rule"], len(wl["inputs"]), D["quad_level"], wl["lo"], wl["hi"])
        xi, al, th = O.node_inflow_params(Z[0], wl["inputs"], wl["u_ref"], wl["alpha"], wl.get("angle_deg", 0.0))
        self.uin = O.inflow(D["nz"], wl["u_ref"], xi, al, D["nz"], th)
        self.f = O.init_equilibrium(self.p, self.flags)
        self.n = 0

    def run(self, k):
        t0 = time.perf_counter()
        self.O.run(self.p, self.flags, self.uin, self.f, self.n, k)
        self.n += k
        return time.perf_counter() - t0


def time_oracle(wl, budget_s, threads=None):
    """FP64 oracle on one node of the workload for about budget_s seconds of
    time steps.  Returns (GLUPS, threads, steps, seconds)."""
    node = OracleNode(wl, threads)
    one = node.run(1)
    steps = max(1, min(200, int(budget_s / max(one, 1e-6))))
    dt = node.run(steps)
    return node.cells * steps / dt / 1e9, node.threads, steps, dt


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    wl = workload_for(args)
    D = wl["domains"][0]
    node = OracleNode(wl)
    one = node.run(1)
    k = max(1, int(3.0 / max(one, 1e-6)))   # about 3 s of CPU work per benchmark step
    vals = []
    for i in range(args.warmup + args.steps):
        dt = node.run(k)
        if i >= args.warmup:
            vals.append(dt)
    ms = 1000.0 * sum(vals) / len(vals)
    glups = node.cells * k / (ms * 1e-3) / 1e9
    hi = host_info()
    sample = ("FP64 oracle on %d threads, one collocation node of %dx%dx%d, %d time steps per benchmark step"
              % (node.threads, D["nx"], D["ny"], D["nz"], k))
    line = {
        "impl": "reference", "metric": METRIC, "value": round(glups, 6), "unit": "GLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": wl["name"], "cells": node.cells, "time_steps_per_step": k,
                   "l2": "inputs larger than L2", "host": hi},
        "cpu_baseline": {"value": round(glups, 6), "unit": "GLUPS", "cores": node.threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(glups, 6), "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU legs
class Ctx:
    """Shared state of the GPU arm: modules, the tuning of the headline run,
    the peak bandwidth."""

    def __init__(self, S, W, torch, np, peak, tuning):
        self.S, self.W, self.torch, self.np, self.peak, self.tuning = S, W, torch, np, peak, tuning
        self.shapes = {}   # FP32 launch shape per workload, from the legs that tuned it

    def release(self, ens):
        ens.close()
        del ens
        self.torch.cuda.empty_cache()

    def timed_steps(self, ens, n):
        """Device time (ms) of n time steps on the handle's stream."""
        e0, e1 = (self.torch.cuda.Event(enable_timing=True) for _ in range(2))
        e0.record(ens.stream)
        self.S.sc_lbm_step(ens.h, n)
        e1.record(ens.stream)
        ens.stream.synchronize()
        ens.sync()
        return e0.elapsed_time(e1)


def sizes(S, cfg, ens):
    nd = cfg.c.n_domains
    cells = [cfg.domains[d]["nx"] * cfg.domains[d]["ny"] * cfg.domains[d]["nz"] for d in range(nd)]
    fluid = [int((S.sc_lbm_geometry(cfg, d) == 0).sum()) for d in range(nd)]
    nodes = list(ens.n_nodes)
    return cells, fluid, nodes


def field_errors(cx, wl, precisions, steps, ramp):
    """Relative L2 error (fluid cells) of the mean and std fields of every
    domain after `steps` time steps, for each precision, against the FP64
    plain path on the same inputs; the start-up ramp is shortened to `ramp`
    steps so that the flow is driven at full strength when compared.
    Computed outside any timed region."""
    S, W, np, torch = cx.S, cx.W, cx.np, cx.torch
    base = dict(wl, ramp_steps=ramp)
    cfg = S.make_config(base)
    nd = cfg.c.n_domains
    masks = [S.sc_lbm_geometry(cfg, d) == 0 for d in range(nd)]

    def fields(prec):
        e = S.Ensemble(S.make_config(dict(base, precision=prec)))
        e.step(steps)
        out = []
        for d in range(nd):
            m = e.moments(d)
            out.append((m["mean"].cpu().numpy(), m["std"].cpu().numpy()))
        e.sync()
        cx.release(e)
        return out

    def rel(a, b):
        return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))

    ref = fields(W.FP64_PLAIN)
    res = {}
    for name, prec in precisions:
        got = fields(prec)
        res[name] = {"err_mean": [round(rel(g[0][m], r[0][m]), 8) for g, r, m in zip(got, ref, masks)],
                     "err_std": [round(rel(g[1][m], r[1][m]), 8) for g, r, m in zip(got, ref, masks)]}
        if nd == 1:
            res[name] = {k: v[0] for k, v in res[name].items()}
    res["against"] = "FP64 plain GPU path, %d time steps, %d-step ramp, relative L2 over fluid cells" % (steps, ramp)
    return res


def leg_plain(cx, wl, glups):
    """Plain FP64, one node per launch, on the headline domain: two nodes of
    the rule (the path runs nodes one after another, so GLUPS per node is the
    ensemble's)."""
    S, W = cx.S, cx.W
    nodes = 2
    pw = dict(wl, precision=W.FP64_PLAIN, node_begin=0, node_count=nodes)
    pe = S.Ensemble(S.make_config(pw))
    S.sc_lbm_step(pe.h, 2)
    pe.sync()
    n = 10
    pms = cx.timed_steps(pe, n)
    cells, fluid, _ = sizes(S, S.make_config(pw), pe)
    cx.release(pe)
    g = cells[0] * nodes * n / (pms * 1e-3) / 1e9
    return {"value": round(g, 4), "unit": "GLUPS", "nodes_timed": nodes, "time_steps": n,
            "ms_per_time_step_per_node": round(pms / (n * nodes), 3),
            "hbm_frac": round(304 * fluid[0] * g / cells[0] / cx.peak, 4),
            "speedup_batched_fp32": round(glups / g, 2)}


def tuned_ensemble(cx, wl, tuning=None):
    """An ensemble in the given launch shape (a tuning dict), else autotuned."""
    S = cx.S
    ens = S.Ensemble(S.make_config(wl))
    if tuning is not None:
        S.sc_lbm_set_tuning(ens.h, **tuning)
    else:
        S.sc_lbm_autotune(ens.h, os.path.join(ROOT, "paper_2508_18202_gb300", "_build", "tuning_cache.json"))
    return ens


def leg_ensemble(cx, name, n_time, precisions, err_steps, err_ramp):
    """GLUPS and HBM fraction of a workload (autotuned per precision) in each
    precision, plus the error of its mean / std fields against FP64.  The
    FP32 launch shape is kept in cx.shapes for the legs on the same domain."""
    S, W = cx.S, cx.W
    wl = workload_named(name)
    out = {"workload": name}
    for pname, prec in precisions:
        w = dict(wl, precision=prec)
        ens = tuned_ensemble(cx, w)
        cells, fluid, nodes = sizes(S, S.make_config(w), ens)
        S.sc_lbm_step(ens.h, 4)
        ens.sync()
        ms = cx.timed_steps(ens, n_time)
        tun = S.sc_lbm_get_tuning(ens.h)
        if prec == W.FP32_SHIFT:
            cx.shapes[name] = tun
        cx.release(ens)
        lups = sum(c * n for c, n in zip(cells, nodes))
        flups = sum(f * n for f, n in zip(fluid, nodes))
        out[pname] = {"value": round(lups * n_time / (ms * 1e-3) / 1e9, 3), "unit": "GLUPS",
                      "hbm_frac": round(BYTES_PER_LUP[prec] * flups / (ms / n_time * 1e-3) / 1e9 / cx.peak, 4),
                      "time_steps": n_time, "tuning": tuning_key(tun)}
    out["errors"] = field_errors(cx, wl, precisions, err_steps, err_ramp)
    return out


def leg_rr(cx):
    S, W = cx.S, cx.W
    rwl = dict(W.URBAN_LES_RR)
    ens = tuned_ensemble(cx, rwl, cx.shapes.get(W.URBAN_LES["name"]))
    cells, fluid, nodes = sizes(S, S.make_config(rwl), ens)
    S.sc_lbm_step(ens.h, 4)
    ens.sync()
    ms = cx.timed_steps(ens, 400)
    cx.release(ens)
    g = cells[0] * nodes[0] * 400 / (ms * 1e-3) / 1e9
    return {"value": round(g, 3), "unit": "GLUPS", "workload": rwl["name"],
            "hbm_frac": round(152 * fluid[0] * nodes[0] / (ms / 400 * 1e-3) / 1e9 / cx.peak, 4)}


def leg_series(cx):
    """Hourly inflow series on the LES ensemble: targets every 100 levels,
    25-level moves between them (synthetic speed factors and a random walk of
    directions)."""
    S, W, np = cx.S, cx.W, cx.np
    wl = dict(W.URBAN_LES)
    per, interp, n_t, n_time = 100, 25, 12, 400
    rng = np.random.default_rng(2024)
    speed = np.clip(1.0 + 0.15 * rng.standard_normal(n_t), 0.5, 1.5)
    dirs = np.cumsum(20.0 * rng.standard_normal(n_t))
    ie = tuned_ensemble(cx, wl, cx.shapes.get(wl["name"]))
    cells, fluid, nodes = sizes(S, S.make_config(wl), ie)
    ie.set_inflow_series(speed, dirs, per, interp)
    S.sc_lbm_step(ie.h, wl["ramp_steps"] + 4)   # past the start-up ramp, untimed
    ie.sync()
    _, c0 = S.sc_lbm_counters(ie.h)
    ms = cx.timed_steps(ie, n_time)
    _, c1 = S.sc_lbm_counters(ie.h)
    cx.release(ie)
    g = cells[0] * nodes[0] * n_time / (ms * 1e-3) / 1e9
    return {"value": round(g, 3), "unit": "GLUPS", "targets": n_t, "steps_per_target": per,
            "interp_steps": interp, "levels": [wl["ramp_steps"] + 4, wl["ramp_steps"] + 4 + n_time],
            "kernel_launches": int(c1 - c0),
            "hbm_frac": round(152 * fluid[0] * nodes[0] / (ms / n_time * 1e-3) / 1e9 / cx.peak, 4)}


def leg_paper(cx):
    """The paper's case at full size: disk of radius 270 and height 40, 121
    Gauss-Hermite nodes, regularized collision (default launch shape), plus
    one moment and degree-5 Hermite gPC reduction of all 121 nodes."""
    S, W, torch = cx.S, cx.W, cx.torch
    pw = W.URBAN_DISK_PAPER
    pcfg = S.make_config(pw)
    pe = S.Ensemble(pcfg)
    cells, fluid, nodes = sizes(S, pcfg, pe)
    S.sc_lbm_step(pe.h, 4)
    pe.sync()
    n_time = 40
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record(pe.stream)
    S.sc_lbm_step(pe.h, n_time)
    e1.record(pe.stream)
    pe.moments(0, gpc=True)
    e2.record(pe.stream)
    pe.stream.synchronize()
    pe.sync()
    pms = e0.elapsed_time(e1)
    rc_chk, nbad = S.sc_lbm_check(pe.h)
    cx.release(pe)
    return {"value": round(cells[0] * nodes[0] * n_time / (pms * 1e-3) / 1e9, 3), "unit": "GLUPS",
            "workload": pw["name"], "nodes": nodes[0], "fluid_cells": fluid[0],
            "fluid_glups": round(fluid[0] * nodes[0] * n_time / (pms * 1e-3) / 1e9, 3),
            "hbm_frac": round(152 * fluid[0] * nodes[0] / (pms / n_time * 1e-3) / 1e9 / cx.peak, 4),
            "ms_per_time_step": round(pms / n_time, 3),
            "moments_gpc_ms": round(e1.elapsed_time(e2), 3),
            "populations_gb": round(cells[0] * nodes[0] * 19 * 4 / 1e9, 1),
            "state_ok": rc_chk == S.SC_OK and nbad == 0}


def leg_adjoint(cx):
    """Seconds per gradient on the 128x64x48 urban domain, 2000 steps, 16
    probes, 45 checkpoints, and the ratio to one forward run."""
    S, W, np, torch = cx.S, cx.W, cx.np, cx.torch
    aw = W.URBAN_ADJOINT
    acfg = S.make_config(aw)
    probes = S.sc_lbm_probe_points(acfg, 0, aw["n_probes"])
    ae = S.Ensemble(acfg)
    S.sc_lbm_set_inflow(ae.h, *aw["truth"], 0.0)
    ae.step(aw["steps"])
    ua = ae.velocity(0, 0).double().cpu().numpy()
    AD = aw["domains"][0]
    target = np.array([ua[:, x + AD["nx"] * (y + AD["ny"] * z)] for x, y, z in probes])
    assim = S.Assimilation(ae, probes, target, aw["steps"])
    assim.loss_and_grad(*aw["guess"])  # warm-up
    torch.cuda.synchronize()
    reps = 3
    t0 = time.perf_counter()
    for _ in range(reps):
        Jg, gg, _ = assim.loss_and_grad(*aw["guess"])
    s_grad = (time.perf_counter() - t0) / reps
    S.sc_lbm_reset(ae.h)
    S.sc_lbm_set_inflow(ae.h, *aw["guess"], 0.0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ae.step(aw["steps"])
    ae.sync()
    s_fwd = time.perf_counter() - t0
    _, kl = S.sc_lbm_counters(ae.h)
    cx.release(ae)
    del assim
    acells = AD["nx"] * AD["ny"] * AD["nz"]
    return {"value": round(s_grad, 4), "unit": "s/gradient", "workload": aw["name"], "time_steps": aw["steps"],
            "checkpoints": int(np.ceil(np.sqrt(aw["steps"]))), "forward_s": round(s_fwd, 4),
            "ratio_to_forward": round(s_grad / s_fwd, 2),
            "sweeps_glups": round(3 * acells * aw["steps"] / s_grad / 1e9, 3),
            "loss": Jg, "grad": [float(gg[0]), float(gg[1])]}


def leg_e2e(cx, wl, cfg, columns, L, n_steps, world, n_nodes_all):
    """End to end through the C ABI with host buffers: per benchmark step
    sc_lbm_init from pinned host geometry (H2D), L time steps, and the moments
    into pinned host memory (D2H).  Under torchrun each rank initialises its
    own node range, and the moments come from the FP64 moment sums
    all-reduced over the ranks and finished by the library (the one exchange
    of the sharded path); the value counts every rank's lattice updates over
    the slowest rank's time."""
    S, torch, np = cx.S, cx.torch, cx.np
    D = wl["domains"][0]
    cells = D["nx"] * D["ny"] * D["nz"]
    flags = S.sc_lbm_geometry(cfg, 0)
    ws = torch.empty(S.sc_lbm_workspace_size(cfg), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()
    flags_pinned = torch.from_numpy(flags).pin_memory()
    mean_h = torch.empty(cells, dtype=torch.float64).pin_memory()
    std_h = torch.empty(cells, dtype=torch.float64).pin_memory()
    prof_h = torch.empty(len(columns) * D["nz"] * 4, dtype=torch.float64).pin_memory()
    fh = (S.C.c_void_p * 1)(flags_pinned.data_ptr())
    if world > 1:
        dist = torch.distributed
        s1, s2 = (torch.empty(cells, dtype=torch.float64, device="cuda") for _ in range(2))
        mean_d, std_d = (torch.empty(cells, dtype=torch.float64, device="cuda") for _ in range(2))
        wt = torch.empty(1, dtype=torch.float64, device="cuda")
        cur = torch.cuda.current_stream()
    t = cx.tuning
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(n_steps):
        hh = S.C.c_void_p()
        S._call("sc_lbm_init", cfg.ref, S.C.c_void_p(ws.data_ptr()), ws.numel(),
                S.C.c_void_p(stream.cuda_stream), fh, S.C.byref(hh))
        S._call("sc_lbm_set_tuning", hh, S.C.byref(S.sc_lbm_tuning(
            t["block_x"], t["block_y"], t["slab_z"], t["tile_order"], t["exec_mode"], t["graph_steps"],
            t["variant"])), handle=hh)
        S.sc_lbm_step(hh, L)
        if world > 1:
            S.sc_lbm_moment_sums(hh, 0, s1, s2, None)
            wt.fill_(S.sc_lbm_weight_sum(hh, 0))
            cur.wait_stream(stream)
            for x in (s1, s2, wt):
                dist.all_reduce(x, op=dist.ReduceOp.SUM)
            stream.wait_stream(cur)
            S.sc_lbm_moments_from_sums(hh, 0, s1, s2, float(wt.item()), mean_d, std_d)
            cur.wait_stream(stream)
            mean_h.copy_(mean_d, non_blocking=True)
            std_h.copy_(std_d, non_blocking=True)
            cur.synchronize()
        else:
            S.sc_lbm_moments(hh, 0, mean_h, std_h, columns, prof_h, None, None, out_host=True)
        S.sc_lbm_destroy(hh)
    dt = time.perf_counter() - t0
    if world > 1:
        tt = torch.tensor([dt], device="cuda")
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        dt = float(tt.item())
    del ws
    torch.cuda.empty_cache()
    # geometry flags, link words, class bytes; listed (outlet) cells with
    # their 256-byte rule records (each rank holds the geometry); inflow
    # tables; node weights x gPC basis (the ramp travels in the launch
    # parameters)
    n_listed = int((flags.reshape(D["nz"], D["ny"], D["nx"])[:, :, -1] == 0).sum())
    P = 1
    if wl.get("gpc_degree", -1) >= 0:
        from math import comb
        P = comb(wl["gpc_degree"] + len(wl["inputs"]), len(wl["inputs"])) + 1
    h2d = world * (cells * (1 + 8 + 1) + n_listed * (4 + 256)) + n_nodes_all * (D["nz"] * (16 + 24) + 8 * P)
    if world > 1:
        d2h = world * 2 * 8 * cells
        note = ("per step and rank: sc_lbm_init of its node range from pinned host geometry, %d time steps, "
                "FP64 moment sums all-reduced, mean and std to pinned host; bytes summed over the ranks" % L)
    else:
        d2h = 2 * 8 * cells + len(columns) * D["nz"] * 4 * 8
        note = "per step: sc_lbm_init from pinned host geometry, %d time steps, moments to pinned host" % L
    return {"value": round(float(cells) * n_nodes_all * L * n_steps / dt / 1e9, 4), "unit": "GLUPS",
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "steps": n_steps, "note": note}


def leg_cpu(wl_head):
    """The FP64 oracle on the host cores: all threads on one node of the
    headline domain (about 15 s), one thread on one node of the 256x128x64
    LES domain (about 10 s), with the full runs they extrapolate to."""
    g, thr, steps, dt = time_oracle(wl_head, budget_s=15.0)
    D = wl_head["domains"][0]
    cells = D["nx"] * D["ny"] * D["nz"]
    les = workload_named("urban_les_256x128x64_cc3")
    g1, thr1, steps1, dt1 = time_oracle(les, budget_s=10.0, threads=1)
    L = les["domains"][0]
    lcells = L["nx"] * L["ny"] * L["nz"]
    return {"value": round(g, 6), "unit": "GLUPS", "cores": thr, "kind": "oracle",
            "sample": "FP64 oracle, one node of %dx%dx%d for %d time steps (%.1f s) on %d threads"
                      % (D["nx"], D["ny"], D["nz"], steps, dt, thr),
            "full_run_extrapolated_h": round(cells * 69 * wl_head.get("steps", 10000) / (g * 1e9) / 3600.0, 1),
            "single_thread": {"value": round(g1, 6), "unit": "GLUPS", "cores": thr1,
                              "sample": "one node of %dx%dx%d for %d time steps (%.1f s)"
                                        % (L["nx"], L["ny"], L["nz"], steps1, dt1),
                              "les_ensemble_extrapolated_h": round(lcells * 13 * les["steps"] / (g1 * 1e9) / 3600.0,
                                                                   1)},
            "host": host_info()}


def one_leg(args, S, W, torch, np):
    """A single extra leg, alone (for profiling its kernels)."""
    peak, _ = peaks()
    cx = Ctx(S, W, torch, np, peak, None)
    prec = {"fp32": W.FP32_SHIFT, "bf16": W.BF16_STORE, "fp16": W.FP16_STORE}[args.precision]
    name = args.leg
    if name == "plain":
        r = leg_plain(cx, workload_for(args), float("nan"))
    elif name == "les":
        r = leg_ensemble(cx, "urban_les_256x128x64_cc3", 20, [(args.precision, prec)], 20, 10)
    elif name == "batched":
        r = leg_ensemble(cx, "urban_batched_3domains", 20, [(args.precision, prec)], 20, 10)
    elif name == "rr":
        r = leg_rr(cx)
    elif name == "series":
        r = leg_series(cx)
    elif name == "paper":
        r = leg_paper(cx)
    elif name == "adjoint":
        r = leg_adjoint(cx)
    else:
        raise SystemExit("unknown leg " + name)
    print(json.dumps({"leg": name, "result": r}), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm
def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2508_18202_gb300 import sclbm as S
    from paper_2508_18202_gb300 import workloads as W

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if args.leg:
        return one_leg(args, S, W, torch, np)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    skip = set(s for s in args.skip.split(",") if s)
    if args.workload != HEADLINE or args.nodes:
        skip |= set(LEGS.split(",")) - {"tune"}
    if world > 1:
        # the extra legs are single-GPU measurements; e2e runs on every rank
        skip |= set(LEGS.split(",")) - {"tune", "e2e"}

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    wl = workload_for(args)
    L = args.lbm_steps or DEFAULT_LBM_STEPS.get(args.workload, 100)
    ndom = len(wl["domains"])
    full_cfg = S.make_config(wl)
    _, a_full = S.sc_lbm_quadrature(full_cfg, 0)
    if world > 1:
        if ndom != 1:
            raise SystemExit("node sharding covers single-domain workloads")
        b, c = S.shard_nodes(len(a_full), world, rank)
        cfg = S.make_config(wl, node_begin=b, node_count=c)
    else:
        cfg = full_cfg
    ens = S.Ensemble(cfg)
    h = ens.h
    cells_d, fluid_d, nodes_d = sizes(S, cfg, ens)
    lup_step = sum(c * n for c, n in zip(cells_d, nodes_d))
    flup_step = sum(f * n for f, n in zip(fluid_d, nodes_d))
    columns = [S.sc_lbm_probe_columns(cfg, d, wl.get("n_columns", 4)) for d in range(ndom)]
    if args.tuning:
        bx, by, bz, order, mode, gsteps, variant = (int(v) for v in args.tuning.split(","))
        S.sc_lbm_set_tuning(h, bx, by, bz, order, mode, gsteps, variant)
    elif "tune" not in skip:
        S.sc_lbm_autotune(h, os.path.join(ROOT, "paper_2508_18202_gb300", "_build", "tuning_cache.json"))
    tuning = S.sc_lbm_get_tuning(h)
    S.sc_lbm_reset(h)
    P = ens.cfg.c.gpc_degree
    wsum = S.sc_lbm_rule_weight_sum(full_cfg, 0)

    def bench_step(ev=None):
        if ev is not None:
            ev[0].record(ens.stream)
        S.sc_lbm_step(h, L)
        if ev is not None:
            ev[1].record(ens.stream)
        if world > 1:
            # node shards: moment sums, all-reduce, finish (the one exchange)
            out = ens.sharded_moments(0, gpc=P >= 0)
            return [out]
        return [ens.moments(d, probes=columns[d], gpc=P >= 0) for d in range(ndom)]

    for _ in range(args.warmup):
        bench_step()
    ens.sync()
    barrier()
    _, k0 = S.sc_lbm_counters(h)
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        t_start.record(ens.stream)
        for k in range(args.steps):
            bench_step(kev[k])
        t_end.record(ens.stream)
        ens.stream.synchronize()
        barrier()
    _, k1 = S.sc_lbm_counters(h)
    ens.sync()
    ms_total = t_start.elapsed_time(t_end)
    ms_kernel = sum(a.elapsed_time(b) for a, b in kev)
    if world > 1:
        t = torch.tensor([ms_total], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_total = float(t.item())
    # every rank advanced its own nodes: the whole job's lattice updates
    lups_all = float(sum(c * len(a_full) for c in cells_d)) if world > 1 else float(lup_step)
    glups = lups_all * L * args.steps / (ms_total * 1e-3) / 1e9
    step_ms = ms_kernel / (args.steps * L)
    alg_bytes = BYTES_PER_LUP[wl["precision"]] * flup_step
    achieved = alg_bytes / (step_ms * 1e-3) / 1e9
    peak, peak_kind = peaks()
    khash = kernel_source_hash()
    traffic = recorded_traffic(khash, wl["name"] + ("" if not args.nodes else "_L%d" % args.nodes), tuning)
    if traffic is not None and world > 1:
        # the recorded figure covers every node of the rule; this rank's
        # launches run its node range (traffic is proportional to nodes)
        traffic = traffic * sum(nodes_d) / len(a_full)
    extra = {}
    out = ens.moments(0, probes=columns[0], gpc=P >= 0)
    fl = torch.from_numpy(S.sc_lbm_geometry(cfg, 0) == 0).cuda()
    extra["mean_u_fluid"] = float(out["mean"][fl].mean().item())
    ens.close()
    del ens, out
    torch.cuda.empty_cache()

    cx = Ctx(S, W, torch, np, peak, tuning)
    legs = {}

    def run_leg(name, fn, *a):
        if name in skip or rank != 0:
            return None
        t0 = time.perf_counter()
        r = fn(*a)
        if isinstance(r, dict):
            r["leg_s"] = round(time.perf_counter() - t0, 1)
        return r

    legs["plain_fp64"] = run_leg("plain", leg_plain, cx, wl, glups)
    # the 13-node LES ensemble in FP32 and in BF16 / FP16 storage (the
    # storage key), each against the FP64 path
    les_prec = [("fp32", W.FP32_SHIFT)]
    if "storage" not in skip:
        les_prec += [("bf16", W.BF16_STORE), ("fp16", W.FP16_STORE)]
    les = run_leg("les", leg_ensemble, cx, "urban_les_256x128x64_cc3", 500, les_prec, 300, 100)
    legs["les_256x128x64"] = les
    if les and "bf16" in les:
        legs["storage"] = {k: dict(les[k], err_mean=les["errors"][k]["err_mean"],
                                   err_std=les["errors"][k]["err_std"]) for k in ("bf16", "fp16")}
        legs["storage"]["against"] = les["errors"]["against"]
    legs["batched_3domains"] = run_leg("batched", leg_ensemble, cx, "urban_batched_3domains", 200,
                                       [("fp32", W.FP32_SHIFT), ("bf16", W.BF16_STORE)], 300, 100)
    legs["regularized"] = run_leg("rr", leg_rr, cx)
    legs["inflow_series"] = run_leg("series", leg_series, cx)
    legs["paper_case"] = run_leg("paper", leg_paper, cx)
    legs["adjoint"] = run_leg("adjoint", leg_adjoint, cx)
    e2e = None
    if "e2e" not in skip:
        e2e = leg_e2e(cx, wl, cfg, columns[0], L, args.steps, world, len(a_full))
    cpu = None
    if "cpu" not in skip and rank == 0 and world == 1:
        cpu = leg_cpu(wl)

    if rank == 0:
        steps_full = wl.get("steps", 0)
        line = {
            "metric": METRIC, "value": round(glups, 4), "unit": "GLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_total / args.steps, 3),
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
            "dtype": DTYPE[wl["precision"]], "data": "synthetic",
            "config": {"workload": wl["name"],
                       "cells": cells_d[0] if ndom == 1 else cells_d,
                       "fluid_cells": fluid_d[0] if ndom == 1 else fluid_d,
                       "nodes": len(a_full) if ndom == 1 else nodes_d,
                       "time_steps_per_step": L,
                       "full_run_time_steps": steps_full,
                       "full_run_s": round(ms_total / args.steps * steps_full / L / 1e3, 2) if steps_full else None,
                       "full_run_note": "the full run is %d benchmark steps; full_run_s extrapolates the timed "
                                        "steps (%d time steps)" % (steps_full // L if steps_full else 0,
                                                                   L * args.steps),
                       "parallelism": ("nodes: %d contiguous node ranges, FP64 moment sums all-reduced per "
                                       "benchmark step" % world) if world > 1 else "single",
                       "l2": "inputs larger than L2 (%.1f GB of populations)"
                             % (lup_step * 19 * BYTES_PER_LUP[wl["precision"]] / 152 * 4 / 1e9),
                       "tuning": tuning},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "traffic": traffic,
                         "peak_kind": peak_kind,
                         "kernel": "one time step: aa_even or aa_odd_bulk (+ listed cells), averaged per level",
                         "bytes_per_fluid_lup": BYTES_PER_LUP[wl["precision"]],
                         "algorithmic_bytes_per_time_step": int(alg_bytes),
                         "avg_time_step_ms": round(step_ms, 5), "kernel_hash": khash},
            "fluid_glups": round(glups * flup_step / lup_step, 4),
            **legs,
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(k1 - k0),
            "clocks": clk.summary(), "extra": extra,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
