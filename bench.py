#!/usr/bin/env python3
"""Benchmark of the SC-LBM hot path on GB300.

One benchmark step = one output interval of the synthetic urban LES ensemble
(256x128x64 cells, 24 seeded buildings, 13 Clenshaw-Curtis Smolyak nodes,
BGK + Smagorinsky, FP32 shifted populations): `--lbm-steps` (default 500)
stream-collide time steps of every node, followed by the FP64 quadrature
reduction to mean / std / gPC fields and the 95% profile bands.  Ten steps
are the full 5000-step run.

value      ensemble GLUPS = cells x nodes x time steps / seconds (device time,
           inputs resident), whole job over all ranks.
e2e        the same metric through the C ABI with host buffers: per step
           sc_lbm_init from pinned host geometry (H2D), the time steps, and
           sc_lbm_moments into pinned host outputs (D2H).
roofline   the stream-collide kernel: algorithmic bytes (152 B per fluid
           cell update in FP32, 19 reads + 19 writes) per launch over the
           average launch duration, against the measured HBM copy bandwidth.
Also reported: the plain one-node-at-a-time FP64 GPU path, BF16 / FP16
storage, and the FP64 CPU oracle on the host cores (cpu_baseline).

`--impl reference` times the FP64 CPU oracle on a bounded sample of the same
workload instead (the method has no other reference implementation).
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ensemble GLUPS & %HBM roofline, batched FP32 vs plain FP64; adjoint s/gradient"
BYTES_PER_LUP = {1: 152, 2: 76, 3: 76, 0: 304}
DTYPE = {1: "f32", 2: "bf16-storage/f32", 3: "f16-storage/f32", 0: "f64"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--lbm-steps", type=int, default=500, help="time steps per benchmark step")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16", "fp16"])
    ap.add_argument("--workload", default="urban_les_256x128x64_cc3",
                    choices=["urban_les_256x128x64_cc3", "urban_batched_3domains", "urban_large_512x256x128_cc4",
                             "urban_les_rr_256x128x64_cc3", "urban_gh121_256x128x64_rr",
                             "urban_disk_540x540x40_gh121"],
                    help="the benchmark workload; the other two are measured without the extra legs")
    ap.add_argument("--nodes", type=int, default=0,
                    help="profiling case: keep only this many Smolyak levels' worth of nodes (0 = all)")
    ap.add_argument("--skip", default="",
                    help="comma list of extra legs to skip: plain,storage,rr,series,paper,cpu,e2e,tune,adjoint")
    ap.add_argument("--tuning", default="",
                    help="fixed launch shape block_x,block_y,slab_z,tile_order,exec_mode,graph_steps,variant "
                         "instead of the autotuner")
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
    h = hashlib.sha256()
    for f in ("lbm_kernels.cu", "lbm_device.cuh", "sclbm_internal.h"):
        with open(os.path.join(ROOT, "paper_2508_18202_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel_hash, workload):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        e = d.get(workload)
        if e and e.get("kernel_hash") == kernel_hash:
            return float(e["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


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


def workload_for(args):
    from paper_2508_18202_gb300 import workloads as W
    wl = dict({w["name"]: w for w in W.ALL}[args.workload])
    wl["precision"] = {"fp32": W.FP32_SHIFT, "bf16": W.BF16_STORE, "fp16": W.FP16_STORE}[args.precision]
    if args.nodes:
        # profiling case: a coarser sparse grid (fewer nodes), same domain
        wl["domains"] = [dict(wl["domains"][0], quad_level=args.nodes)]
    return wl


# ------------------------------------------------------------------ CPU oracle
def time_oracle(wl, budget_s=15.0, threads=None):
    """FP64 oracle on one collocation node of the workload: time steps sized to
    roughly budget_s seconds.  Returns (GLUPS, threads, steps, seconds)."""
    from oracle import oracle as O
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    nthreads = O.set_threads(threads or os.cpu_count() or 1)
    D = wl["domains"][0]
    p = O.params(D["nx"], D["ny"], D["nz"], D["bc"], wl["tau0"], wl["c_smag"], wl["ramp_steps"],
                 collision=wl.get("collision", 0))
    flags = O.geometry(D["nx"], D["ny"], D["nz"], D.get("seed", 0), D.get("n_buildings", 0),
                       *D.get("fp", (1, 1)), *D.get("h", (1, 1)), boxes=D.get("boxes"),
                       disk_radius=D.get("disk_radius", 0.0))
    Z, a = O.quadrature(wl["quad_rule"], len(wl["inputs"]), D["quad_level"], wl["lo"], wl["hi"])
    xi, al, th = O.node_inflow_params(Z[0], wl["inputs"], wl["u_ref"], wl["alpha"], wl.get("angle_deg", 0.0))
    uin = O.inflow(D["nz"], wl["u_ref"], xi, al, D["nz"], th)
    f = O.init_equilibrium(p, flags)
    t0 = time.perf_counter()
    O.run(p, flags, uin, f, 0, 1)
    one = time.perf_counter() - t0
    steps = max(1, min(200, int(budget_s / max(one, 1e-6))))
    t0 = time.perf_counter()
    O.run(p, flags, uin, f, 1, steps)
    dt = time.perf_counter() - t0
    cells = D["nx"] * D["ny"] * D["nz"]
    return cells * steps / dt / 1e9, nthreads, steps, dt


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    wl = workload_for(args)
    D = wl["domains"][0]
    vals = []
    info = None
    for k in range(args.warmup + args.steps):
        g, thr, steps, dt = time_oracle(wl, budget_s=4.0)
        if k >= args.warmup:
            vals.append((g, steps, dt))
        info = (thr, steps)
    glups = sum(v[0] for v in vals) / len(vals)
    ms = 1000.0 * sum(v[2] for v in vals) / len(vals)
    sample = ("FP64 oracle, one collocation node of %dx%dx%d, %d time steps per benchmark step"
              % (D["nx"], D["ny"], D["nz"], info[1]))
    line = {
        "impl": "reference", "metric": METRIC, "value": round(glups, 6), "unit": "GLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": wl["name"], "cells": D["nx"] * D["ny"] * D["nz"], "nodes": 13,
                   "l2": "inputs larger than L2"},
        "cpu_baseline": {"value": round(glups, 6), "unit": "GLUPS", "cores": info[0], "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(glups, 6), "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
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
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    skip = set(s for s in args.skip.split(",") if s)
    if args.workload != "urban_les_256x128x64_cc3":
        skip |= {"plain", "storage", "rr", "series", "paper", "e2e", "adjoint", "cpu"}  # legs of the default workload

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    wl = workload_for(args)
    D = wl["domains"][0]
    cfg = S.make_config(wl)
    ens = S.Ensemble(cfg)
    h = ens.h
    ndom = len(wl["domains"])
    cells_d = [d["nx"] * d["ny"] * d["nz"] for d in wl["domains"]]
    nodes_d = [ens.n_nodes[d] for d in range(ndom)]
    fluid_d = [int((S.sc_lbm_geometry(cfg, d) == 0).sum()) for d in range(ndom)]
    # lattice updates and fluid updates of all (domain, node) pairs per time step
    lup_step = sum(c * n for c, n in zip(cells_d, nodes_d))
    flup_step = sum(f * n for f, n in zip(fluid_d, nodes_d))
    cells, nodes, fluid = cells_d[0], nodes_d[0], fluid_d[0]
    flags = S.sc_lbm_geometry(cfg, 0)
    columns = [S.sc_lbm_probe_columns(cfg, d, wl.get("n_columns", 4)) for d in range(ndom)]
    if args.tuning:
        bx, by, bz, order, mode, gsteps, variant = (int(v) for v in args.tuning.split(","))
        S.sc_lbm_set_tuning(h, bx, by, bz, order, mode, gsteps, variant)
    elif "tune" not in skip:
        S.sc_lbm_autotune(h, os.path.join(ROOT, "paper_2508_18202_gb300", "_build", "tuning_cache.json"))
    tuning = S.sc_lbm_get_tuning(h)
    S.sc_lbm_reset(h)
    L = args.lbm_steps
    P = ens.cfg.c.gpc_degree

    def bench_step(ev=None):
        if ev is not None:
            ev[0].record(ens.stream)
        S.sc_lbm_step(h, L)
        if ev is not None:
            ev[1].record(ens.stream)
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
    lups = float(lup_step) * L * args.steps * world
    glups = lups / (ms_total * 1e-3) / 1e9
    launch_ms = ms_kernel / (args.steps * L)
    alg_bytes = BYTES_PER_LUP[wl["precision"]] * flup_step
    achieved = alg_bytes / (launch_ms * 1e-3) / 1e9
    peak, peak_kind = peaks()
    khash = kernel_source_hash()
    traffic = recorded_traffic(khash, wl["name"] + ("" if not args.nodes else "_L%d" % args.nodes))
    extra = {}
    # fields sanity (not timed)
    out = ens.moments(0, probes=columns[0], gpc=P >= 0)
    mean = out["mean"]
    extra["mean_u_fluid"] = float(mean[torch.from_numpy(flags == 0).cuda()].mean().item())
    ens.close()
    del ens
    torch.cuda.empty_cache()

    # ---- plain FP64, one node at a time, one launch per step
    plain = None
    if "plain" not in skip and rank == 0:
        pw = dict(wl, precision=W.FP64_PLAIN)
        pe = S.Ensemble(S.make_config(pw))
        n_plain_steps = 20
        S.sc_lbm_step(pe.h, 2)
        pe.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(pe.stream)
        S.sc_lbm_step(pe.h, n_plain_steps)
        e1.record(pe.stream)
        pe.stream.synchronize()
        pe.sync()
        pms = e0.elapsed_time(e1)
        plain_glups = cells * nodes * n_plain_steps / (pms * 1e-3) / 1e9
        plain = {"value": round(plain_glups, 4), "unit": "GLUPS",
                 "ms_per_time_step_per_node": round(pms / (n_plain_steps * nodes), 4),
                 "hbm_frac": round(304 * fluid * plain_glups / cells / peak, 4),
                 "speedup_batched_fp32": round(glups / world / plain_glups, 2)}
        pe.close()
        del pe
        torch.cuda.empty_cache()

    # ---- reduced storage
    storage = {}
    if "storage" not in skip and rank == 0 and args.precision == "fp32":
        for name, prec in (("bf16", W.BF16_STORE), ("fp16", W.FP16_STORE)):
            se = S.Ensemble(S.make_config(dict(wl, precision=prec)))
            S.sc_lbm_set_tuning(se.h, **{k: tuning[k] for k in ("block_x", "block_y", "slab_z", "tile_order")},
                                exec_mode=tuning["exec_mode"], graph_steps=tuning["graph_steps"])
            S.sc_lbm_step(se.h, 4)
            se.sync()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(se.stream)
            S.sc_lbm_step(se.h, 200)
            e1.record(se.stream)
            se.stream.synchronize()
            se.sync()
            sms = e0.elapsed_time(e1)
            g = cells * nodes * 200 / (sms * 1e-3) / 1e9
            storage[name] = {"value": round(g, 3), "unit": "GLUPS",
                             "hbm_frac": round(76 * fluid * nodes / (sms / 200 * 1e-3) / 1e9 / peak, 4)}
            se.close()
            del se
            torch.cuda.empty_cache()

    # ---- the paper's collision (recursive regularized, third-order equilibrium)
    regularized = None
    if "rr" not in skip and rank == 0 and args.precision == "fp32":
        rwl = dict(W.URBAN_LES_RR, precision=wl["precision"])
        re_ = S.Ensemble(S.make_config(rwl))
        S.sc_lbm_set_tuning(re_.h, **{k: tuning[k] for k in ("block_x", "block_y", "slab_z", "tile_order")},
                            exec_mode=tuning["exec_mode"], graph_steps=tuning["graph_steps"],
                            variant=tuning["variant"])
        S.sc_lbm_step(re_.h, 4)
        re_.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(re_.stream)
        S.sc_lbm_step(re_.h, 400)
        e1.record(re_.stream)
        re_.stream.synchronize()
        re_.sync()
        rms = e0.elapsed_time(e1)
        g = cells * nodes * 400 / (rms * 1e-3) / 1e9
        regularized = {"value": round(g, 3), "unit": "GLUPS", "workload": rwl["name"],
                       "hbm_frac": round(152 * fluid * nodes / (rms / 400 * 1e-3) / 1e9 / peak, 4)}
        re_.close()
        del re_
        torch.cuda.empty_cache()

    # ---- hourly inflow series: targets every 100 levels, 25-level moves
    # between them (synthetic speed factors and a random walk of directions)
    inflow_series = None
    if "series" not in skip and rank == 0 and args.precision == "fp32":
        per, interp, n_t, n_time = 100, 25, 12, 400
        rng = np.random.default_rng(2024)
        speed = np.clip(1.0 + 0.15 * rng.standard_normal(n_t), 0.5, 1.5)
        dirs = np.cumsum(20.0 * rng.standard_normal(n_t))
        ie = S.Ensemble(S.make_config(wl))
        S.sc_lbm_set_tuning(ie.h, **{k: tuning[k] for k in ("block_x", "block_y", "slab_z", "tile_order")},
                            exec_mode=tuning["exec_mode"], graph_steps=tuning["graph_steps"],
                            variant=tuning["variant"])
        ie.set_inflow_series(speed, dirs, per, interp)
        S.sc_lbm_step(ie.h, wl["ramp_steps"] + 4)   # past the start-up ramp, untimed
        ie.sync()
        _, c0 = S.sc_lbm_counters(ie.h)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ie.stream)
        S.sc_lbm_step(ie.h, n_time)
        e1.record(ie.stream)
        ie.stream.synchronize()
        ie.sync()
        _, c1 = S.sc_lbm_counters(ie.h)
        ims = e0.elapsed_time(e1)
        g = lup_step * n_time / (ims * 1e-3) / 1e9
        inflow_series = {"value": round(g, 3), "unit": "GLUPS", "targets": n_t, "steps_per_target": per,
                         "interp_steps": interp, "levels": [wl["ramp_steps"] + 4, wl["ramp_steps"] + 4 + n_time],
                         "kernel_launches": int(c1 - c0),
                         "hbm_frac": round(BYTES_PER_LUP[wl["precision"]] * flup_step / (ims / n_time * 1e-3) / 1e9
                                           / peak, 4)}
        ie.close()
        del ie
        torch.cuda.empty_cache()

    # ---- the paper's case at full size: disk of radius 270 and height 40,
    # 121 Gauss-Hermite nodes, regularized collision (default launch shape)
    paper_case = None
    if "paper" not in skip and rank == 0 and args.precision == "fp32":
        pw = W.URBAN_DISK_PAPER
        pcfg = S.make_config(pw)
        pe = S.Ensemble(pcfg)
        pcells = pw["domains"][0]["nx"] * pw["domains"][0]["ny"] * pw["domains"][0]["nz"]
        pfluid = int((S.sc_lbm_geometry(pcfg, 0) == 0).sum())
        pnodes = pe.n_nodes[0]
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
        paper_case = {"value": round(pcells * pnodes * n_time / (pms * 1e-3) / 1e9, 3), "unit": "GLUPS",
                      "workload": pw["name"], "nodes": pnodes, "fluid_cells": pfluid,
                      "fluid_glups": round(pfluid * pnodes * n_time / (pms * 1e-3) / 1e9, 3),
                      "hbm_frac": round(152 * pfluid * pnodes / (pms / n_time * 1e-3) / 1e9 / peak, 4),
                      "ms_per_time_step": round(pms / n_time, 3),
                      "moments_gpc_ms": round(e1.elapsed_time(e2), 3),
                      "populations_gb": round(pcells * pnodes * 19 * 4 / 1e9, 1),
                      "state_ok": rc_chk == S.SC_OK and nbad == 0}
        pe.close()
        del pe
        torch.cuda.empty_cache()

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if "e2e" not in skip:
        ws = torch.empty(S.sc_lbm_workspace_size(cfg), dtype=torch.uint8, device="cuda")
        stream = torch.cuda.Stream()
        flags_pinned = torch.from_numpy(flags).pin_memory()
        mean_h = torch.empty(cells, dtype=torch.float64).pin_memory()
        std_h = torch.empty(cells, dtype=torch.float64).pin_memory()
        prof_h = torch.empty(len(columns[0]) * D["nz"] * 4, dtype=torch.float64).pin_memory()
        fh = (S.C.c_void_p * 1)(flags_pinned.data_ptr())
        n_e2e = max(2, min(args.steps, 3))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            hh = S.C.c_void_p()
            S._call("sc_lbm_init", cfg.ref, S.C.c_void_p(ws.data_ptr()), ws.numel(),
                    S.C.c_void_p(stream.cuda_stream), fh, S.C.byref(hh))
            S._call("sc_lbm_set_tuning", hh, S.C.byref(S.sc_lbm_tuning(
                tuning["block_x"], tuning["block_y"], tuning["slab_z"], tuning["tile_order"],
                tuning["exec_mode"], tuning["graph_steps"])), handle=hh)
            S.sc_lbm_step(hh, L)
            S.sc_lbm_moments(hh, 0, mean_h, std_h, columns[0], prof_h, None, None, out_host=True)
            S.sc_lbm_destroy(hh)
        dt = time.perf_counter() - t0
        if world > 1:
            t = torch.tensor([dt], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            dt = float(t.item())
        # geometry flags, link words, class bytes; listed (outlet) cells with their
        # 256-byte rule records; inflow tables; node weights x gPC basis (the ramp
        # travels in the launch parameters)
        n_listed = int((flags.reshape(D["nz"], D["ny"], D["nx"])[:, :, -1] == 0).sum())
        h2d = (cells * (1 + 8 + 1) + n_listed * (4 + 256) + nodes * D["nz"] * (16 + 24)
               + nodes * 8 * (1 + 6))
        d2h = 2 * 8 * cells + len(columns[0]) * D["nz"] * 4 * 8
        e2e = {"value": round(float(cells) * nodes * L * n_e2e * world / dt / 1e9, 4), "unit": "GLUPS",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "note": "per step: sc_lbm_init from pinned host geometry, %d time steps, moments to pinned host" % L}
        del ws

    # ---- adjoint seconds per gradient (128x64x48 urban domain, 2000 steps, 16 probes)
    adjoint = None
    if "adjoint" not in skip and rank == 0:
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
        acells = AD["nx"] * AD["ny"] * AD["nz"]
        adjoint = {"value": round(s_grad, 4), "unit": "s/gradient",
                   "workload": aw["name"], "time_steps": aw["steps"],
                   "checkpoints": int(np.ceil(np.sqrt(aw["steps"]))),
                   "forward_s": round(s_fwd, 4), "ratio_to_forward": round(s_grad / s_fwd, 2),
                   "sweeps_glups": round(3 * acells * aw["steps"] / s_grad / 1e9, 3),
                   "loss": Jg, "grad": [float(gg[0]), float(gg[1])]}
        ae.close()
        del ae, assim
        torch.cuda.empty_cache()

    # ---- CPU oracle baseline (rank 0, N = 1 only)
    cpu = None
    if "cpu" not in skip and rank == 0 and world == 1:
        g, thr, steps, dt = time_oracle(wl, budget_s=15.0)
        cpu = {"value": round(g, 6), "unit": "GLUPS", "cores": thr, "kind": "oracle",
               "sample": "FP64 oracle, one node of %dx%dx%d for %d time steps (%.1f s)"
                         % (D["nx"], D["ny"], D["nz"], steps, dt)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(glups, 4), "unit": "GLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_total / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[wl["precision"]], "data": "synthetic",
            "config": {"workload": wl["name"],
                       "cells": cells if ndom == 1 else cells_d,
                       "fluid_cells": fluid if ndom == 1 else fluid_d,
                       "nodes": nodes if ndom == 1 else nodes_d,
                       "time_steps_per_step": L, "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs larger than L2 (%.2f GB of populations)"
                             % (lup_step * 19 * BYTES_PER_LUP[wl["precision"]] / 152 * 4 / 1e9),
                       "tuning": tuning},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "traffic": traffic,
                         "peak_kind": peak_kind,
                         "kernel": "one time step: aa_even + (aa_odd_bulk + aa_odd_boundary), averaged per level",
                         "bytes_per_fluid_lup": BYTES_PER_LUP[wl["precision"]],
                         "avg_launch_ms": round(launch_ms, 5), "kernel_hash": khash},
            "fluid_glups": round(glups * flup_step / lup_step, 4),
            "plain_fp64": plain, "storage": storage or None, "regularized": regularized,
            "inflow_series": inflow_series, "paper_case": paper_case,
            "adjoint": adjoint,
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(k1 - k0),
            "clocks": clk.summary(), "extra": extra,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
