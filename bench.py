#!/usr/bin/env python
"""Benchmark of the SRM hot path on GB300 (one JSON line on stdout).

A step is one complete generation: Algorithm 1 iterated from the RSA start
to the target volume fraction, followed by the binary64 certification of the
final state (time-to-target).  The workload is the 1e6-sphere polydisperse
clustered RVE (log-normal radii, 200 Gaussian clusters, RSA at 0.1, target
0.40) in the FP32 cell-relative form with FP64 certification.

value    particle-updates/s = N x sweeps / device time of the K timed steps
         (inputs resident on the device, CUDA events on the handle's stream),
         summed over ranks (each rank runs its own RVE: weak scaling).
e2e      the same metric through the public API from host buffers: srm_init
         from host arrays (host-to-device copies), the run, the certification
         and srm_positions (device-to-host copy of the result) all inside the
         timed region.
roofline the dominant kernel, from CUDA events recorded between the launches
         of each super-step in a separate timing pass over a whole generation;
         the overlap check (Algorithm 6) gets its own entry.

--impl reference times the FP64 CPU reference on the host cores, each step a
bounded sample (one sweep of Algorithm 3 over all particles at the start of
the run).  The GPU arm's cpu_baseline times the reference at three states of
the GPU run and extrapolates its time to the target.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-updates/s & time-to-target phi, 1e6 3D spheres; FP32 vs FP64; % HBM peak"
FP32_LANES_PER_SM = 128
N_SM = 152
SM_MAX_MHZ = 2070.0


def workload_desc(w, precision):
    return {
        "workload": (f"{w.name}: {w.dim}D, N={w.n}, box {w.box[0]:.4g}^{w.dim}, target phi "
                     f"{w.target_phi}, RSA start at f0=0.1"
                     + (", log-normal radii (mean 1, sd 0.2, truncated [0.5, 2]), 200 Gaussian "
                        "clusters (sigma = 5 mean radii)" if w.name == "poly_1m" else ", monodisperse")),
        "n": w.n, "dim": w.dim, "target_phi": w.target_phi,
        "c_w": w.c_w, "c_m": round(w.c_m, 8), "N_k": w.N_k, "N_l": w.N_l, "N_shake": w.N_shake,
        "precision": ("fp32 cell-relative offsets, fp64 scale/phi bookkeeping and certification"
                      if precision == 32 else "fp64 absolute positions (bit-exact with the reference)"),
        "l2": "256 MiB buffer written between timed steps (L2 flushed)",
    }


def hbm_side(w, precision, ms, pk):
    """The sweep against HBM: its algorithmic bytes per launch are one read
    and one write of every particle's position and radius and one moved
    flag (FP32 form: 16 + 16 + 1 bytes; FP64 form: 32 + 32 + 1)."""
    per = 33 if precision == 32 else 65
    gbs = per * w.n / (ms * 1e-3) / 1e9
    return {"bytes_per_launch": per * w.n, "achieved_gbs": gbs, "peak_gbs": pk["hbm_gbs"],
            "frac": gbs / pk["hbm_gbs"]}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": SM_MAX_MHZ}, "fallback"


class ClockSampler:
    """nvidia-smi clock and throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.p = None
        # samples of the timed region; SRM_CLOCKS_DIR keeps them where a caller wants them
        base = os.environ.get("SRM_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(base, f"clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-i", str(self.dev), "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
            self.f.close()

    def summary(self):
        if not self.p:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def source_sha(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


KERNEL_SOURCES = ["paper_2605_18254_gb300/csrc/k_sweep.cu", "paper_2605_18254_gb300/csrc/k_check.cu",
                  "paper_2605_18254_gb300/csrc/srm_dev.cuh", "paper_2605_18254_gb300/csrc/srm_stencil.cuh"]


def committed_traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)
    except Exception:
        return None
    e = t.get(kernel)
    if not e or e.get("source_sha") != source_sha(KERNEL_SOURCES):
        return None
    return e.get("dram_bytes_per_launch_full")


def cpu_sample(w, sweeps=1):
    """The FP64 reference on the host: sweeps of Algorithm 3 over all particles
    at the first swollen scale.  Returns (particle-updates/s, seconds)."""
    import oracle
    s = oracle.System(w.dim, w.box, w.x, w.radii, lam=1.0, target_phi=w.target_phi, c_w=w.c_w,
                      c_m=w.c_m, N_k=w.N_k, N_l=w.N_l, N_shake=w.N_shake, seed=w.seed)
    s.lam = 1.0 * (1.0 + w.c_w)
    t0 = time.perf_counter()
    for _ in range(sweeps):
        s.sweep()
    dt = time.perf_counter() - t0
    return w.n * sweeps / dt, dt


def cpu_samples(w, states):
    """The FP64 reference on the host, one sweep of Algorithm 3 over all
    particles from each of the given states (label, positions, scale): the
    swept scale is the state's scale swollen by one step (a sweep of the N_k
    loop).  Returns {label: seconds}."""
    import oracle
    out = {}
    for label, x, lam in states:
        s = oracle.System(w.dim, w.box, x, w.radii, lam=lam * (1.0 + w.c_w), target_phi=w.target_phi, c_w=w.c_w,
                          c_m=w.c_m, N_k=w.N_k, N_l=w.N_l, N_shake=w.N_shake, seed=w.seed)
        t0 = time.perf_counter()
        s.sweep()
        out[label] = time.perf_counter() - t0
    return out


def weighted_oracle_time(samples, record):
    """Extrapolated reference time of a whole generation: the run's sweeps
    (record: (scale, sweeps so far) after each chunk of iterations) each
    timed at the reference's per-sweep time for that scale, interpolated
    linearly in the scale between the sampled states ((scale, seconds))."""
    pts = sorted(samples)

    def t_at(lam):
        if lam <= pts[0][0]:
            return pts[0][1]
        for (l0, t0), (l1, t1) in zip(pts, pts[1:]):
            if lam <= l1:
                return t1 if l1 <= l0 else t0 + (t1 - t0) * (lam - l0) / (l1 - l0)
        return pts[-1][1]
    total, prev_lam, prev_sw = 0.0, record[0][0], record[0][1]
    for lam, sw in record[1:]:
        total += (sw - prev_sw) * t_at(0.5 * (lam + prev_lam))
        prev_lam, prev_sw = lam, sw
    return total


def make_workload(name):
    import srm_inputs
    return srm_inputs.RECIPES[name]()


def run_reference(args, rank, world):
    if rank != 0:
        return
    t0 = time.time()
    w = make_workload(args.workload)
    for _ in range(args.warmup):
        cpu_sample(w, 1)
    tot, dt_all = 0.0, []
    for _ in range(args.steps):
        ups, dt = cpu_sample(w, 1)
        dt_all.append(dt)
    value = w.n * args.steps / sum(dt_all)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "particle-updates/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(dt_all) / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_desc(w, 64),
        "cpu_baseline": {"value": value, "unit": "particle-updates/s", "cores": 1, "kind": "oracle",
                         "sample": f"each step: 1 sweep of Algorithm 3 over all {w.n} particles at the "
                                   "first swollen scale (the start of the run, where sweeps are cheapest; the "
                                   "other states of the run need the GPU to reach), single-threaded FP64 "
                                   "reference"},
        "e2e": {"value": value, "unit": "particle-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "wall_s": time.time() - t0,
    }
    print(json.dumps(line), flush=True)


def _oracle_member(args):
    """One RVE of the ensemble run to target by the reference (worker
    process); returns (particle updates, seconds)."""
    import oracle
    import srm_inputs
    i, seed0 = args
    w = srm_inputs.ensemble_member(i, 256, seed0)
    s = oracle.System(w.dim, w.box, w.x, w.radii, lam=1.0, target_phi=w.target_phi, c_w=w.c_w, c_m=w.c_m,
                      N_k=w.N_k, N_l=w.N_l, N_shake=w.N_shake, seed=w.seed)
    t0 = time.perf_counter()
    s.run()
    dt = time.perf_counter() - t0
    return w.n * s.counters()["sweeps"], dt


def run_oracle_timing(args, rank, world):
    """The reference on the host cores: C1 run in full; C2 and C3 one sweep,
    extrapolated to the sweeps of a full run (labelled); ensemble throughput
    of one reference process per core on the first members of C4."""
    if rank != 0:
        return
    import multiprocessing as mp
    import platform
    import oracle
    import srm_inputs
    out = {"host": {"machine": platform.machine(), "cores": os.cpu_count()}}
    w = srm_inputs.disks_1k()
    s = oracle.System(w.dim, w.box, w.x, w.radii, lam=1.0, target_phi=w.target_phi, c_w=w.c_w, c_m=w.c_m,
                      N_k=w.N_k, N_l=w.N_l, N_shake=w.N_shake, seed=w.seed)
    t0 = time.perf_counter()
    s.run()
    dt = time.perf_counter() - t0
    sw = s.counters()["sweeps"]
    out["disks_1k_full_run"] = {"seconds": dt, "sweeps": sw, "particle_updates_per_s": w.n * sw / dt,
                                "cores": 1}
    for name, sweeps_full in (("spheres_100k", args.c2_sweeps), ("poly_1m", args.c3_sweeps)):
        wl = srm_inputs.RECIPES[name]()
        ups, dts = cpu_sample(wl, 1)
        out[name] = {"one_sweep_s": dts, "particle_updates_per_s": ups, "cores": 1,
                     "extrapolated_time_to_target_s": dts * sweeps_full,
                     "note": f"one sweep timed, times {sweeps_full} sweeps of the GPU run to target (extrapolated)"}
    nproc = os.cpu_count() or 1
    members = [(i, 0) for i in range(min(args.oracle_members, 256))]
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(nproc) as pool:
        res = pool.map(_oracle_member, members)
    wall = time.perf_counter() - t0
    out["ensemble_members"] = {"members": len(members), "processes": nproc, "wall_s": wall,
                               "particle_updates_per_s": sum(u for u, _ in res) / wall,
                               "note": "first members of the 256-RVE ensemble (2D disks), each run to target"}
    line = {"impl": "reference", "metric": "reference throughput on the host cores", "value":
            out["ensemble_members"]["particle_updates_per_s"], "unit": "particle-updates/s", "n_gpus": 0,
            "steps": 1, "warmup": 0, "ms_per_step": 1e3 * wall, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "oracle timing: C1 in full, C2/C3 one sweep extrapolated, C4 members on "
                                   f"{nproc} processes"}, "oracle": out}
    print(json.dumps(line), flush=True)


def combine_ranks(dev_s, e2e_s, updates, dist=None, device="cpu"):
    """Whole-job numbers of replicas: the slowest rank's times, the sum of
    the particle updates of all ranks (host-side reduction only; the ranks
    exchange no simulation data)."""
    if dist is None:
        return dev_s, e2e_s, updates
    import torch
    t = torch.tensor([dev_s, e2e_s], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([updates], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t[0]), float(t[1]), float(u[0])


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    import paper_2605_18254_gb300 as srm

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
    w = make_workload(args.workload)
    if rank:
        # every rank generates its own RVE (weak scaling, no data exchange)
        import srm_inputs
        w = srm_inputs.RECIPES[args.workload](seed=w.seed + 1000 * rank)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    x_host = torch.from_numpy(np.ascontiguousarray(w.x)).pin_memory()
    r_host = torch.from_numpy(np.ascontiguousarray(w.radii)).pin_memory()
    kw = dict(c_m=w.c_m, c_w=w.c_w, N_k=w.N_k, N_l=w.N_l, N_shake=w.N_shake,
              precision=args.precision, init="explicit", stream=stream.cuda_stream)

    def new_rve():
        return srm.Rve(w.dim, w.box, r_host.numpy(), w.target_phi, w.seed, positions=x_host.numpy(), **kw)

    def one_step(timed):
        flush.fill_(1)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        torch.cuda.synchronize()
        t_wall = time.perf_counter()
        ev[0].record(stream)
        g = new_rve()                       # host -> device copies of the inputs
        ev[1].record(stream)
        info = g.run_to_target()
        pairs, gap, phi = g.certify()
        ev[2].record(stream)
        xo, ro = g.positions()               # device -> host copy of the result
        ev[3].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t_wall
        st = g.state()
        g.close()
        return dict(info=info, pairs=pairs, gap=gap, phi=phi, launches=st["kernel_launches"],
                    dev_s=ev[1].elapsed_time(ev[2]) / 1e3, e2e_s=ev[0].elapsed_time(ev[3]) / 1e3,
                    wall_s=wall, sweeps=info["sweeps"])

    for _ in range(args.warmup):
        one_step(False)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    res = []
    with ClockSampler(local_rank) as clk:
        for _ in range(args.steps):
            res.append(one_step(True))
    torch.cuda.synchronize()
    dev_s = sum(r["dev_s"] for r in res)
    e2e_s = sum(r["e2e_s"] for r in res)
    sweeps = sum(r["sweeps"] for r in res)
    updates = float(w.n) * sweeps
    dev_max, e2e_max, updates_all = combine_ranks(dev_s, e2e_s, updates, dist, dev)
    if rank != 0:
        return
    ok = all(r["pairs"] == 0 and r["info"]["converged"] and abs(r["phi"] - w.target_phi) < 1e-9
             for r in res)

    # ---- roofline of the dominant kernel: a timing pass over the same
    # generation to target (CUDA events between the stages of every
    # super-step, on the handle's stream)
    g = new_rve()
    g.set_timing(True)
    st0 = g.state()
    record = [(st0["lambda"], 0)]
    states = [("start", np.ascontiguousarray(w.x), st0["lambda"])]
    mid_phi = 0.5 * (w.target_phi + 0.1)
    while True:
        info = g.run_to_target(25) if not g.state()["done"] else None
        st = g.state()
        record.append((st["lambda"], st["sweeps"]))
        if len(states) == 1 and st["phi"] >= mid_phi:
            states.append((f"phi={st['phi']:.3f}", g.positions()[0], st["lambda"]))
        if st["done"]:
            break
    states.append((f"phi={st['phi']:.3f}", g.positions()[0], st["lambda"]))
    tm = g.timings()
    st1 = g.state()
    tun = g.tuning()
    g.close()
    f32 = int(args.precision == 32)
    staged = int(tun["sweep_path"] == 2)
    kname = {"sweep": f"k_draw + k_sweep_df<{w.dim},{f32},{staged}> ({'staged' if staged else 'general'} path)",
             "check": f"{'k_check_cells' if st1['check_kernel'] else 'k_check'}<{f32}>"}
    # the check's floor: the first iterations, where almost every particle
    # moves and the check only reads the moved flags
    g = new_rve()
    g.set_timing(True)
    g.run_to_target(3)
    tm0 = g.timings()
    g.close()
    per_launch = {
        "sweep": tm["ms_sweep"] / max(1, tm["sweep_launches"]),
        "check": tm["ms_check"] / max(1, tm["check_launches"]),
        "bin": tm["ms_bin"] / max(1, tm["supersteps"]),
    }
    totals = {"sweep": tm["ms_sweep"], "check": tm["ms_check"], "bin": tm["ms_bin"], "control": tm["ms_control"]}
    dom = max(("sweep", "check", "bin"), key=lambda k: totals[k])
    pk, pk_kind = peaks()
    flops_per_pair = 11.0 if w.dim == 3 else 8.0
    if dom in ("sweep", "check"):
        # algorithmic work: the pairs Algorithm 5 examines (every trial
        # against the particles of the 3^d cells around the home cell) for
        # the sweep; the pairs the check tests for Algorithm 6
        pairs = (st1["pairs_alg5"] - st0["pairs_alg5"]) if dom == "sweep" else (st1["pairs_check"] - st0["pairs_check"])
        tested = (st1["pairs_sweep"] - st0["pairs_sweep"]) if dom == "sweep" else pairs
        launches = tm["sweep_launches"] if dom == "sweep" else tm["check_launches"]
        flops = flops_per_pair * pairs / max(1, launches)
        achieved = flops / (per_launch[dom] * 1e-3) / 1e12
        peak = N_SM * FP32_LANES_PER_SM * 2 * pk.get("sm_max_mhz", SM_MAX_MHZ) * 1e6 / 1e12
        if args.precision == 64:
            peak = peak / 64.0
        roof = {"kernel": kname[dom], "bound": "alu", "achieved": achieved,
                "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": committed_traffic(f"k_{dom}{args.precision}"),
                "per_launch_ms": per_launch[dom],
                "work": (f"{flops_per_pair:.0f} flops per pair x {pairs / max(1, launches):.4g} pairs per launch: "
                         + ("every trial of Algorithm 3 against the particles of the 3^d cells around its home cell "
                            f"(Algorithm 5's candidate set; {(st1['trials'] - st0['trials']) / max(1, launches):.4g} "
                            f"trials per launch); after culling the kernel tests {tested / max(1, launches):.4g} pairs"
                            if dom == "sweep" else "pairs tested by the check")),
                "hbm_side": hbm_side(w, args.precision, per_launch[dom], pk) if dom == "sweep" else None,
                "peak_basis": (f"FP32 lanes: {N_SM} SMs x {FP32_LANES_PER_SM} x 2 flops x "
                               f"{pk.get('sm_max_mhz', SM_MAX_MHZ):.0f} MHz" + (" / 64 (FP64 rate)" if args.precision == 64 else "")),
                "stage_ms_total": totals, "supersteps": tm["supersteps"],
                "rates": {"trials_per_s": (st1["trials"] - st0["trials"]) / max(1e-9, tm["ms_sweep"] * 1e-3),
                          "check_particles_per_s": w.n * tm["check_launches"] / max(1e-9, tm["ms_check"] * 1e-3),
                          "note": "trial moves of Algorithm 3 per second of sweep stage; particles checked by "
                                  "Algorithm 6 per second of check stage (every particle of a checked sweep)"}}
    else:
        bytes_per = w.n * (64 if args.precision == 32 else 96)
        achieved = bytes_per / (per_launch["bin"] * 1e-3) / 1e9
        roof = {"kernel": "binning", "bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"],
                "unit": "GB/s", "frac": achieved / pk["hbm_gbs"], "traffic": None,
                "stage_ms_total": totals}
    roof["peak_source"] = f"{pk_kind}" + (" (HBM from MEASURED_PEAKS.json)" if pk_kind == "measured" else "")
    # the overlap check (Algorithm 6) against HBM: its algorithmic bytes per
    # launch are the moved flag, the position and the cell index of every
    # particle plus the cell starts (FP32 form, 3D: 1 + 16 + 4 + 4 / 1.5)
    cb = (1 + (16 if args.precision == 32 else 32) + 4) + 4.0 / 1.5
    ck_ms = per_launch["check"]
    floor_ms = tm0["ms_check"] / max(1, tm0["check_launches"])
    roof["check"] = {
        "kernel": kname["check"], "bound": "hbm", "per_launch_ms": ck_ms,
        "bytes_per_launch": cb * w.n, "achieved": cb * w.n / (ck_ms * 1e-3) / 1e9, "peak": pk["hbm_gbs"],
        "unit": "GB/s", "frac": cb * w.n / (ck_ms * 1e-3) / 1e9 / pk["hbm_gbs"],
        "floor_ms": floor_ms, "floor_frac": cb * w.n / (floor_ms * 1e-3) / 1e9 / pk["hbm_gbs"],
        "traffic": committed_traffic(f"k_check{args.precision}"),
        "launches": tm["check_launches"],
        "note": ("per_launch_ms over the whole generation; floor_ms over the checks of the first 3 iterations, "
                 "where almost every particle moved and the check only reads flags (launch and read floor); "
                 "the time above the floor is the stencil walks of the particles that did not move"),
    }

    # ---- FP64 form on the same sample (first sweeps), for the precision comparison
    cmp = {}
    if args.compare_fp64 and args.precision == 32:
        for prec in (32, 64):
            kw2 = dict(kw)
            kw2["precision"] = prec
            g = srm.Rve(w.dim, w.box, r_host.numpy(), w.target_phi, w.seed, positions=x_host.numpy(), **kw2)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            inf = g.run_to_target(args.compare_iters)
            e1.record(stream)
            torch.cuda.synchronize()
            cmp[f"fp{prec}"] = {"particle_updates_per_s": w.n * inf["sweeps"] / (e0.elapsed_time(e1) / 1e3),
                                "sweeps": inf["sweeps"], "iterations": inf["iterations"]}
            g.close()
        cmp["sample"] = f"first {args.compare_iters} iterations of Algorithm 1 from the RSA start"
        cmp["fp32_over_fp64"] = cmp["fp32"]["particle_updates_per_s"] / cmp["fp64"]["particle_updates_per_s"]

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        import platform
        secs = cpu_samples(w, states)
        lam_of = {label: lam for label, _, lam in states}
        t_ref = weighted_oracle_time([(lam_of[k] * (1.0 + w.c_w), v) for k, v in secs.items()], record)
        sw_run = record[-1][1]
        cpu = {"value": w.n * sw_run / t_ref, "unit": "particle-updates/s", "cores": 1, "kind": "oracle",
               "sample": (f"1 sweep of Algorithm 3 over all {w.n} particles from each of {len(states)} states of the "
                          f"GPU run ({', '.join(f'{k}: {v:.2f} s' for k, v in secs.items())}; single-threaded FP64 "
                          f"reference; host {platform.machine()}, {os.cpu_count()} cores), weighted by the run's "
                          f"{sw_run} sweeps over the scale"),
               "extrapolated_time_to_target_s": t_ref,
               "gpu_time_to_target_s": dev_max / args.steps,
               "note": "extrapolated: per-sweep times interpolated between the sampled states, times the sweeps of "
                       "the GPU run; the reference runs the same method in the same order (FP64)"}

    h2d = int(x_host.numel() * 8 + r_host.numel() * 8)
    d2h = int(w.n * w.dim * 8 + w.n * 8)
    line = {
        "metric": METRIC, "value": updates_all / dev_max, "unit": "particle-updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dev_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if args.precision == 32 else "f64", "data": "synthetic",
        "config": workload_desc(w, args.precision) | {"parallelism": f"replicas x{world}"},
        "time_to_target_s": dev_max / args.steps,
        "sweeps_per_step": sweeps / args.steps,
        "certified": ok,
        "e2e": {"value": updates_all / e2e_max, "unit": "particle-updates/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "time_to_target_s": e2e_max / args.steps},
        "roofline": roof,
        "cpu_baseline": cpu,
        "precision_compare": cmp or None,
        "gpu_launches": int(sum(r["launches"] for r in res)),
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# batched ensemble: many RVEs of uneven size and dimension in one batch
# ---------------------------------------------------------------------------
def _place_worker(args):
    import srm_inputs
    dim, n, r0, seed = args
    import numpy as np
    return srm_inputs.rsa(dim, (1.0,) * dim, np.full(n, r0), seed)


def run_ensemble(args, rank, world, local_rank):
    """256 RVEs (half disks, half spheres, N log-uniform 1e3..1e5, targets
    uniform 0.30..0.55, seeds 0..255) advanced by the same launches; a step
    runs the whole batch to its targets and certifies every member."""
    import multiprocessing as mp
    import numpy as np
    import srm_inputs
    count = args.ensemble_count
    ws = srm_inputs.ensemble(count=count, seed0=1000 * rank)
    import torch
    import paper_2605_18254_gb300 as srm
    torch.cuda.set_device(local_rank)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    jobs = [srm.make_job(w.dim, w.box, w.radii, w.target_phi, w.seed, c_m=w.c_m, c_w=w.c_w,
                         precision=args.precision, init="explicit", positions=w.x) for w in ws]
    n_total = sum(w.n for w in ws)

    tuned = {}

    def one_step(tune=False):
        flush.fill_(1)
        torch.cuda.synchronize()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(stream)
        b = srm.Batch(jobs, stream=stream.cuda_stream)
        if tuned:
            b.set_tuning(tuned["sweep_blocks_per_sm"], tuned["stage_capacity"], tuned["sweep_path"])
        e[1].record(stream)
        if tune:
            tuned.update(b.autotune(8))
        ok = b.run()
        cert = [b.certify(i) for i in range(len(ws))]
        e[2].record(stream)
        torch.cuda.synchronize()
        sweeps = [b.state(i)["sweeps"] for i in range(len(ws))]
        launches = b.state(0)["kernel_launches"]
        b.close()
        upd = float(sum(w.n * s for w, s in zip(ws, sweeps)))
        return dict(dev_s=e[1].elapsed_time(e[2]) / 1e3, e2e_s=e[0].elapsed_time(e[2]) / 1e3, upd=upd,
                    ok=ok and all(c[0] == 0 and abs(c[2] - w.target_phi) < 1e-9 for c, w in zip(cert, ws)),
                    launches=launches, max_sweeps=max(sweeps))

    dist = None
    if world > 1:
        import torch.distributed as dist
    for k in range(args.warmup):
        one_step(tune=k == 0)
    res = []
    if dist:
        dist.barrier()
    with ClockSampler(local_rank) as clk:
        for _ in range(args.steps):
            res.append(one_step())
    dev = sum(r["dev_s"] for r in res)
    e2e = sum(r["e2e_s"] for r in res)
    upd = sum(r["upd"] for r in res)
    # replicas: the slowest rank's times, the updates of all ranks
    dev, e2e, upd = combine_ranks(dev, e2e, upd, dist, torch.device("cuda", local_rank))
    if rank != 0:
        return
    line = {
        "metric": "particle-updates/s, batched ensemble of RVEs", "value": upd / dev, "unit": "particle-updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dev / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == 32 else "f64", "data": "synthetic",
        "config": {"workload": f"ensemble: {count} RVEs, first half 2D disks, second half 3D spheres, N "
                               f"log-uniform in [1e3, 1e5] (total {n_total}), targets uniform in [0.30, 0.55], "
                               "monodisperse, RSA start at 0.1, seeds 0..255, one batch (every kernel serves "
                               "all RVEs), captured graph",
                   "rves": count, "particles": n_total,
                   "tuning": {"sweep_blocks_per_sm": tuned.get("sweep_blocks_per_sm"),
                              "stage_capacity": tuned.get("stage_capacity"),
                              "sweep_path": tuned.get("sweep_path"),
                              "how": "srm_batch_autotune during the first warm-up step (candidate sweep "
                                     "grids and staging capacities timed on the running batch; the sweep "
                                     "kernel stays the default), applied to every later batch"},
                   "l2": "256 MiB buffer written between timed steps (L2 flushed)"},
        "time_to_target_s": dev / args.steps, "certified": all(r["ok"] for r in res),
        "e2e": {"value": upd / e2e, "unit": "particle-updates/s",
                "h2d_bytes_per_step": int(sum(w.n * (w.dim + 1) * 8 for w in ws)),
                "d2h_bytes_per_step": 24 * len(ws)},
        "gpu_launches": int(sum(r["launches"] for r in res)),
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# serving: one 1e7-sphere job beside a Poisson stream of smaller jobs
# ---------------------------------------------------------------------------
def run_serve(args, rank, world, local_rank):
    """The 1e7-sphere RVE (unit cube, target 0.30) submitted to the serving
    loop beside a Poisson stream of 2D/3D jobs (N log-uniform 1e4..1e6,
    targets 0.30..0.50), arrival rate about 70% of the measured capacity of
    the small-job pool; p50/p99 time-to-target and throughput."""
    import math
    import multiprocessing as mp
    import numpy as np
    import srm_inputs
    n_jobs = args.serve_jobs
    rng = np.random.default_rng(5 + 1000 * rank)
    specs = []
    for i in range(n_jobs):
        dim = 2 if rng.random() < 0.5 else 3
        n = int(math.floor(1e4 * 100.0 ** rng.random()))
        phi = 0.30 + 0.20 * rng.random()
        r_t = math.sqrt(phi / (n * math.pi)) if dim == 2 else (phi * 3.0 / (4.0 * math.pi * n)) ** (1 / 3)
        specs.append((dim, n, phi, r_t, r_t * (0.1 / phi) ** (1.0 / dim), 2000 + i))
    big_n = args.serve_big
    big_rt = (0.30 * 3.0 / (4.0 * math.pi * big_n)) ** (1 / 3)
    big_r0 = big_rt * (0.1 / 0.30) ** (1 / 3)
    # starting configurations are placed ahead of time, in parallel on the host
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(16, os.cpu_count() or 4)) as pool:
        xs = pool.map(_place_worker, [(d, n, r0, sd) for d, n, _, _, r0, sd in specs] + [(3, big_n, big_r0, 5)])
    import torch
    import paper_2605_18254_gb300 as srm
    from paper_2605_18254_gb300 import serve
    torch.cuda.set_device(local_rank)

    def job(i):
        d, n, phi, r_t, r0, sd = specs[i]
        return srm.make_job(d, (1.0, 1.0, 1.0), np.full(n, r0), phi, sd, c_m=0.1 * r_t, c_w=0.01,
                            precision=args.precision, init="explicit", positions=xs[i])

    big_job = srm.make_job(3, (1.0, 1.0, 1.0), np.full(big_n, big_r0), 0.30, 5, c_m=0.1 * big_rt, c_w=0.01,
                           precision=args.precision, init="explicit", positions=xs[-1])
    big_cells = srm.srm_job_footprint(big_job[0])[1]
    small_cells = 0
    for i in range(n_jobs):
        j = job(i)  # keep the arrays the job points to alive while it is used
        small_cells = max(small_cells, srm.srm_job_footprint(j[0])[1])
    # small jobs in a 2D and a 3D pool (one sweep launch per super-step each,
    # the pools overlap on their streams), the big job in a pool of its own
    half = max(1, args.serve_slots // 2)
    pools = [serve.PoolSpec(slots=half, max_particles=1_000_000, max_cells=small_cells, dim=2),
             serve.PoolSpec(slots=half, max_particles=1_000_000, max_cells=small_cells, dim=3),
             serve.PoolSpec(slots=1, max_particles=big_n, max_cells=big_cells, dim=3)]
    server = serve.Server(pools, precision=args.precision, advance=16)
    # capacity of the small-job pools: a burst of jobs all arriving at t = 0
    calib = [serve.Request(rid=i, arrival=0.0, job=job(i)) for i in range(min(16, n_jobs))]
    done, wall = server.run(calib)
    rate = 0.7 * len(done) / wall
    reqs = serve.poisson_stream(n_jobs, rate, 5, lambda i, r: job(i))
    reqs.append(serve.Request(rid=n_jobs, arrival=0.0, job=big_job))
    with ClockSampler(local_rank) as clk:
        done, wall = server.run(reqs)
    server.close()
    summ = serve.summarize(done, wall)
    big = [r for r in done if r.rid == n_jobs][0]
    # replicas: every rank serves its own stream; the slowest rank's wall
    # time, the updates of all ranks
    dist = None
    if world > 1:
        import torch.distributed as dist
    wall_max, _, upd_all = combine_ranks(wall, wall, summ["particle_updates_per_s"] * wall, dist,
                                         torch.device("cuda", local_rank))
    if rank != 0:
        return
    line = {
        "metric": "p50/p99 time-to-target and particle-updates/s under continuous batching",
        "value": upd_all / wall_max, "unit": "particle-updates/s", "n_gpus": world, "steps": 1,
        "warmup": 1, "ms_per_step": 1e3 * wall, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == 32 else "f64", "data": "synthetic",
        "config": {"workload": f"serving: 1 RVE of {big_n} 3D spheres (unit cube, target 0.30) submitted at t=0 "
                               f"beside {n_jobs} jobs (2D/3D, N log-uniform 1e4..1e6, targets 0.30..0.50) "
                               f"arriving as a Poisson stream at {rate:.2f} jobs/s (70% of the measured "
                               "capacity of the small-job pools); pools: "
                               f"{half} 2D slots and {half} 3D slots of 1e6 particles + 1 slot of {big_n}, each pool "
                               "one batch on its own stream"},
        "serving": summ, "big_job_time_to_target_s": big.finished - big.arrival,
        "big_job_sweeps": big.sweeps, "arrival_rate_jobs_per_s": rate,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def regime_run(srm, dim, n, phi_t, seed, c_w, c_m_rel, precision, wall_cap, voxels):
    """One generation from an RSA start at 0.1 (monodisperse, unit box) with
    the given swelling rate and migration length (relative to the target
    radius); stops at the target or after wall_cap seconds.  Returns the
    reached fraction, time, counters and the descriptors of Section 3.2."""
    import numpy as np
    import torch
    r_t = math.sqrt(phi_t / (n * math.pi)) if dim == 2 else (phi_t * 3.0 / (4.0 * math.pi * n)) ** (1.0 / 3.0)
    g = srm.Rve(dim, (1.0,) * dim, ("mono", r_t * (0.1 / phi_t) ** (1.0 / dim)), phi_t, seed, n=n,
                c_m=c_m_rel * r_t, c_w=c_w, precision=precision, init="rsa", f0=0.1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    info = {}
    while time.perf_counter() - t0 < wall_cap:
        info = g.run_to_target(200)
        if info["converged"]:
            break
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    st = g.state()
    pairs, gap_min, phi = g.certify()
    d, _, gap = g.nearest()
    cnt, lvf = g.voronoi_lvf((voxels,) * dim)
    g.close()
    R = r_t * (phi / phi_t) ** (1.0 / dim)
    return {"dim": dim, "n": n, "target_phi": phi_t, "c_w": c_w, "c_m_over_r": c_m_rel,
            "reached_phi": phi, "converged": bool(info.get("converged", False)), "seconds": wall,
            "iterations": st["iterations"], "accepted": st["accepted"], "shaken": st["shaken"],
            "sweeps": st["sweeps"], "certified_pairs": pairs,
            "nn_dist_over_d": {"mean": float(np.mean(d) / (2 * R)), "std": float(np.std(d) / (2 * R))},
            "nn_gap_over_d": {"mean": float(np.mean(gap) / (2 * R)), "std": float(np.std(gap) / (2 * R)),
                              "p05": float(np.percentile(gap, 5) / (2 * R))},
            "lvf": {"mean": float(np.mean(lvf)), "std": float(np.std(lvf)),
                    "p05": float(np.percentile(lvf, 5)), "p95": float(np.percentile(lvf, 95))},
            "voxels_per_axis": voxels}


def run_regimes(args, rank, world, local_rank):
    """Equilibrium-like and clustered configurations (Section 3.2: 2D disks
    and 3D spheres at 0.5) and the dense limits (Section 2: random close
    packing for disks, about 0.60 for spheres), with the nearest-neighbour
    and local-volume-fraction statistics that tell them apart."""
    import torch
    import paper_2605_18254_gb300 as srm
    torch.cuda.set_device(local_rank)
    cap = args.regime_seconds
    # (dim, N, target, seed, c_w, c_m / target radius): slow swelling with
    # long migration relaxes toward equilibrium; fast swelling with migration
    # just long enough to clear the overlaps of one swell step leaves clusters
    runs = {
        "2d_equilibrium_0.5": (2, 5000, 0.5, 11, 0.002, 0.5),
        "2d_clustered_0.5": (2, 5000, 0.5, 11, 0.01, 0.03),
        "3d_equilibrium_0.5": (3, 5000, 0.5, 12, 0.002, 0.1),
        "3d_clustered_0.5": (3, 5000, 0.5, 12, 0.01, 0.03),
        "2d_dense_0.87": (2, 5000, 0.87, 13, 0.0003, 0.01),
        "3d_dense_0.60": (3, 10000, 0.60, 14, 0.0005, 0.05),
    }
    out = {}
    t0 = time.perf_counter()
    for name, (dim, n, phi, seed, c_w, cm) in runs.items():
        # the dense runs get ten times the cap: 0.87 takes about a minute
        out[name] = regime_run(srm, dim, n, phi, seed, c_w, cm, args.precision, cap * (10 if "dense" in name else 1),
                               400 if dim == 2 else 64)
    wall = time.perf_counter() - t0
    line = {"metric": "reached volume fraction and structure descriptors per regime", "value": wall,
            "unit": "s", "n_gpus": world, "steps": 1, "warmup": 0, "ms_per_step": 1e3 * wall,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == 32 else "f64", "data": "synthetic",
            "config": {"workload": "regimes: monodisperse RSA starts at 0.1 in a unit box; equilibrium-like "
                                   "(slow swelling, long migration) vs clustered (fast swelling, short migration) at "
                                   "0.5 (2D 5000 disks, 3D 5000 spheres), dense runs toward 0.87 (2D) and 0.60 (3D) "
                                   f"capped at {cap:.0f} s ({10 * cap:.0f} s for the dense ones); descriptors in "
                                   "binary64 on the GPU"},
            "regimes": out}
    if rank == 0:
        print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# platelets (Section 3.3): house of cards to rho = 5, then relaxation
# ---------------------------------------------------------------------------
def platelet_cpu_baseline(w, states, record, relaxed, relax, D):
    """The binary64 reference on one host core, one sweep from each sampled
    state of the GPU run (generation states at their next swollen scale, and
    the relaxed state with the relaxation parameters), extrapolated to the
    run: generation sweeps at the per-sweep time interpolated in the scale
    between the sampled states, plus the relaxation sweeps at the relaxed
    state's time."""
    import oracle
    samples, times = [], {}
    for label, x, u, lam in states:
        lam_s = min(lam * (1.0 + w.c_w), 1.0)
        o = oracle.PlateletSystem(w.box, x, u, w.a0, w.t0, lam=lam_s, lam_t=1.0, c_w=w.c_w, c_m=w.c_m,
                                  c_r=w.c_r, seed=w.seed)
        t0 = time.perf_counter()
        o.sweep()
        times[label] = time.perf_counter() - t0
        samples.append((lam, times[label]))
    o = oracle.PlateletSystem(w.box, relaxed[0], relaxed[1], w.a0, w.t0, lam=1.0, lam_t=1.0, c_w=0.0,
                              c_m=0.1 * D, c_r=0.1, seed=w.seed)
    t0 = time.perf_counter()
    o.sweep()
    t_rel = time.perf_counter() - t0
    t_gen = weighted_oracle_time(samples, record)
    sweeps = record[-1][1] + relax
    total = t_gen + relax * t_rel
    return {"value": w.n * sweeps / total, "unit": "particle-updates/s", "cores": 1, "kind": "oracle",
            "sample": "one sweep of the single-threaded binary64 reference from each of "
                      + ", ".join(f"{k}: {v:.2f} s" for k, v in times.items())
                      + f" (states of the GPU generation) and from the relaxed state: {t_rel:.2f} s",
            "extrapolated_time_to_target_s": t_gen, "extrapolated_relaxation_s": relax * t_rel,
            "note": "extrapolated: generation sweeps at per-sweep times interpolated in the scale between the "
                    "sampled states, plus the relaxation sweeps at the relaxed state's time"}


def run_platelets(args, rank, world, local_rank):
    """20000 spherodisks of aspect ratio 100 from a bounding-sphere RSA start
    to number density 5 (Eq. 1) with house-of-cards parameters, then
    relaxation sweeps with zero swelling and longer steps; one step = both
    phases from the same start.  value: platelet updates per second of
    device time from the uploaded start to the end of the relaxation; e2e
    adds the upload of the start and the read-back of the final state."""
    import numpy as np
    import torch
    import srm_inputs
    import paper_2605_18254_gb300 as srm
    torch.cuda.set_device(local_rank)
    stream = torch.cuda.current_stream()
    w = srm_inputs.platelets(seed=7 + 1000 * rank)
    D = w.extra["D"]
    relax = args.plt_relax
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    x_host = torch.from_numpy(np.ascontiguousarray(w.x)).pin_memory()
    u_host = torch.from_numpy(np.ascontiguousarray(w.u)).pin_memory()
    last = {}

    def alignment(x, u):
        """Mean |n_i . n_j| over pairs of centres closer than D (1/2 for
        independent uniform orientations): the local order that relaxation
        grows (Section 3.3, Fig. 8)."""
        from scipy.spatial import cKDTree
        p = cKDTree(x, boxsize=np.asarray(w.box)).query_pairs(D, output_type="ndarray")
        return float(np.mean(np.abs(np.sum(u[p[:, 0]] * u[p[:, 1]], axis=1))))

    def one_step():
        flush.fill_(1)
        torch.cuda.synchronize()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        e[0].record(stream)
        g = srm.Platelets(w.box, x_host.numpy(), u_host.numpy(), w.a0, w.t0, w.lambda0, 1.0, w.seed, c_w=w.c_w,
                          c_m=w.c_m, c_r=w.c_r, stream=stream.cuda_stream)
        e[1].record(stream)
        info = g.run_to_target(4000)
        e[2].record(stream)
        g.set_params(c_w=0.0, c_m=0.1 * D, c_r=0.1)
        acc = g.sweeps(relax)
        e[3].record(stream)
        x, u, st = g.state()
        cnt, _ = g.check()
        e[4].record(stream)
        torch.cuda.synchronize()
        g.close()
        last["relaxed"] = (x, u)
        sweeps = info["sweeps"] + relax
        checks = info["sweeps"] - info["shaken"] * 10 + 1
        return dict(dev_s=e[1].elapsed_time(e[3]) / 1e3, gen_s=e[1].elapsed_time(e[2]) / 1e3,
                    relax_s=e[2].elapsed_time(e[3]) / 1e3, e2e_s=e[0].elapsed_time(e[4]) / 1e3,
                    upd=float(w.n * sweeps), sweeps=sweeps, iters=info["iterations"], shaken=info["shaken"],
                    ok=bool(info["converged"]) and cnt == 0 and abs(st["rho"] - w.rho_t) < 1e-9,
                    launches=5 * (sweeps + checks), relax_acc=acc, rho=st["rho"])

    dist = None
    if world > 1:
        import torch.distributed as dist
    for _ in range(args.warmup):
        one_step()
    res = []
    if dist:
        dist.barrier()
    with ClockSampler(local_rank) as clk:
        for _ in range(args.steps):
            res.append(one_step())
    dev = sum(r["dev_s"] for r in res)
    e2e = sum(r["e2e_s"] for r in res)
    upd = sum(r["upd"] for r in res)
    # replicas: the slowest rank's times, the updates of all ranks
    dev, e2e, upd = combine_ranks(dev, e2e, upd, dist, torch.device("cuda", local_rank))
    if rank != 0:
        return
    r0 = res[0]
    # the generation again in chunks of 10 iterations (same result), keeping
    # the states the reference is timed on: the start, the first past
    # rho = 2.5 and the house of cards at rho = 5; also the neighbour
    # alignment of the house of cards and after the relaxation
    g = srm.Platelets(w.box, w.x, w.u, w.a0, w.t0, w.lambda0, 1.0, w.seed, c_w=w.c_w, c_m=w.c_m, c_r=w.c_r,
                      stream=stream.cuda_stream)
    record, states = [(w.lambda0, 0)], [("start", w.x, w.u, w.lambda0)]
    while True:
        info = g.run_to_target(10)
        hx, hu, st = g.state()
        record.append((st["lambda_"], int(st["sweep"])))
        if len(states) == 1 and st["rho"] >= 0.5 * w.rho_t:
            states.append((f"rho={st['rho']:.2f}", hx, hu, st["lambda_"]))
        if info["converged"]:
            break
    states.append((f"rho={st['rho']:.2f}", hx, hu, st["lambda_"]))
    g.close()
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = platelet_cpu_baseline(w, states, record, last["relaxed"], relax, D)
    order = {"house_of_cards": alignment(hx, hu), "relaxed": alignment(*last["relaxed"]),
             "measure": "mean |n_i . n_j| over pairs of centres closer than D; 0.5 for random orientations"}
    line = {
        "metric": "platelet-updates/s and time to the target number density (Section 3.3)",
        "value": upd / dev, "unit": "particle-updates/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * dev / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"platelets: {w.n} spherodisks, aspect ratio {w.extra['aspect']:.0f}, unit box, "
                               f"bounding-sphere RSA start at 0.1, to number density {w.rho_t} (Eq. 1) with "
                               f"c_w={w.c_w}, c_m=0.02 D, c_r={w.c_r} (house of cards), then {relax} relaxation "
                               "sweeps with c_w=0, c_m=0.1 D, c_r=0.1",
                   "n": w.n, "rho_t": w.rho_t, "aspect": w.extra["aspect"],
                   "l2": "256 MiB buffer written between timed steps (L2 flushed)"},
        "time_to_target_s": sum(r["gen_s"] for r in res) / args.steps,
        "relaxation_s": sum(r["relax_s"] for r in res) / args.steps,
        "sweeps_per_step": r0["sweeps"], "iterations": r0["iters"], "shaken": r0["shaken"],
        "certified": all(r["ok"] for r in res), "alignment": order,
        "e2e": {"value": upd / e2e, "unit": "particle-updates/s",
                "h2d_bytes_per_step": int(2 * w.n * 3 * 8), "d2h_bytes_per_step": int(2 * w.n * 3 * 8 + w.n)},
        "cpu_baseline": cpu,
        "gpu_launches": int(sum(r["launches"] for r in res)),
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="poly_1m")
    ap.add_argument("--precision", type=int, default=32, choices=[32, 64])
    ap.add_argument("--compare-iters", type=int, default=20)
    ap.add_argument("--compare-fp64", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ensemble-count", type=int, default=256)
    ap.add_argument("--serve-jobs", type=int, default=200)
    ap.add_argument("--serve-slots", type=int, default=16)
    ap.add_argument("--serve-big", type=int, default=10_000_000)
    ap.add_argument("--regime-seconds", type=float, default=60.0)
    ap.add_argument("--c2-sweeps", type=int, default=168, help="sweeps of the GPU run of spheres_100k to target")
    ap.add_argument("--c3-sweeps", type=int, default=16711, help="sweeps of the GPU run of poly_1m to target")
    ap.add_argument("--oracle-members", type=int, default=32)
    ap.add_argument("--plt-relax", type=int, default=50, help="relaxation sweeps of the platelet workload")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "oracle_timing":
        run_oracle_timing(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    try:
        if args.workload == "ensemble":
            run_ensemble(args, rank, world, local_rank)
        elif args.workload == "serve":
            run_serve(args, rank, world, local_rank)
        elif args.workload == "regimes":
            run_regimes(args, rank, world, local_rank)
        elif args.workload == "platelets":
            run_platelets(args, rank, world, local_rank)
        else:
            run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
