"""Continuous-batching request loop for RVE generation.

Jobs (one RVE each) arrive over time.  The server keeps a few pools of
slots (for one dimension, or either); a pool is one batch
(srm_batch_create_slots) on its own CUDA stream,
all of whose slots are advanced by the same kernel launches.  A job is
admitted into a free slot of the first pool whose slot capacity (particles,
finest-grid cells) fits it, as soon as such a slot is free -- while the jobs
already admitted keep running.  Every pass of the loop enqueues a few
super-steps on every pool (pools on different streams overlap on the GPU),
polls for finished slots, certifies and reads back their RVEs and frees the
slots.  Times are wall-clock from arrival (queueing included) to the end of
the read-back; p50/p99 are reported with the throughput.

All device work goes through the C interface; this module only schedules.
"""
from __future__ import annotations

import dataclasses
import math
import time

import numpy as np

from . import Batch, PREC_F32, make_job, srm_job_footprint


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float           # seconds after the start of the run
    job: tuple               # (srm_job, keep) from make_job
    particles: int = 0
    cells: int = 0
    admitted: float = math.nan
    finished: float = math.nan
    pool: int = -1
    slot: int = -1
    result: tuple = None     # (positions, radii) when kept
    certified: tuple = None  # (pairs, min_gap, phi)
    sweeps: int = 0


@dataclasses.dataclass
class PoolSpec:
    slots: int
    max_particles: int
    max_cells: int
    stage_capacity: int = 0
    dim: int = 0  # dimension the pool's slots accept (0: either; one sweep launch per super-step if 2 or 3)


def slot_bytes(max_particles: int, max_cells: int) -> int:
    """Device memory of one slot (three cell-sorted copies of 48 bytes per
    particle, per-particle work arrays, per-cell counts and starts)."""
    return max_particles * (3 * (32 + 8 + 4 + 4) + 4 * 4 + 1 + 8 * 4) + max_cells * 8


class Server:
    def __init__(self, pools, precision=PREC_F32, memory_budget=None, advance=16, keep_results=False):
        import torch
        self.specs = list(pools)
        need = sum(p.slots * slot_bytes(p.max_particles, p.max_cells) for p in self.specs)
        if memory_budget is not None and need > memory_budget:
            raise ValueError(f"pools need {need} bytes of device memory, budget {memory_budget}")
        self.streams = [torch.cuda.Stream() for _ in self.specs]
        self.pools = [Batch(slots=p.slots, max_particles=p.max_particles, max_cells=p.max_cells, dim=p.dim,
                            precision=precision, stage_capacity=p.stage_capacity,
                            stream=s.cuda_stream) for p, s in zip(self.specs, self.streams)]
        self.free = [list(range(p.slots)) for p in self.specs]
        self.running = [dict() for _ in self.specs]
        self.advance = advance
        self.keep_results = keep_results

    def _fits(self, k, req):
        p = self.specs[k]
        return (req.particles <= p.max_particles and req.cells <= p.max_cells
                and (p.dim == 0 or p.dim == int(req.job[0].dim)))

    def run(self, requests, time_limit=3600.0):
        """Serves requests (sorted by arrival time) to completion."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        for r in reqs:
            r.particles, r.cells = srm_job_footprint(r.job[0])
            if not any(self._fits(k, r) for k in range(len(self.specs))):
                raise ValueError(f"request {r.rid} fits no pool")
        pending, queue, done = list(reqs), [], []
        t0 = time.perf_counter()
        while pending or queue or any(self.running):
            now = time.perf_counter() - t0
            if now > time_limit:
                raise TimeoutError("serving run exceeded its time limit")
            while pending and pending[0].arrival <= now:
                queue.append(pending.pop(0))
            # admission: first-come first-served, into the first pool that fits
            still = []
            for r in queue:
                placed = False
                for k in range(len(self.specs)):
                    if self.free[k] and self._fits(k, r):
                        s = self.free[k].pop(0)
                        self.pools[k].admit(s, r.job)
                        r.pool, r.slot, r.admitted = k, s, time.perf_counter() - t0
                        self.running[k][s] = r
                        placed = True
                        break
                if not placed:
                    still.append(r)
            queue = still
            busy = [k for k in range(len(self.specs)) if self.running[k]]
            if not busy:
                if pending:
                    time.sleep(max(0.0, min(0.002, pending[0].arrival - now)))
                continue
            for k in busy:
                self.pools[k].advance(self.advance)
            for k in busy:
                for s in self.pools[k].poll():
                    r = self.running[k].pop(s)
                    r.certified = self.pools[k].certify(s)
                    st = self.pools[k].state(s)
                    r.sweeps = int(st["sweeps"])
                    if self.keep_results:
                        r.result = self.pools[k].positions(s)
                    else:
                        self.pools[k].positions(s)  # the read-back is part of the service
                    r.finished = time.perf_counter() - t0
                    self.pools[k].release(s)
                    self.free[k].append(s)
                    done.append(r)
        wall = time.perf_counter() - t0
        return done, wall

    def close(self):
        for p in self.pools:
            p.close()


def summarize(done, wall):
    tt = np.array([r.finished - r.arrival for r in done])
    svc = np.array([r.finished - r.admitted for r in done])
    updates = float(sum(r.particles * r.sweeps for r in done))
    return {
        "jobs": len(done),
        "time_to_target_p50_s": float(np.percentile(tt, 50)),
        "time_to_target_p99_s": float(np.percentile(tt, 99)),
        "service_p50_s": float(np.percentile(svc, 50)),
        "service_p99_s": float(np.percentile(svc, 99)),
        "wall_s": wall,
        "particle_updates_per_s": updates / wall,
        "all_certified": all(r.certified is not None and r.certified[0] == 0 for r in done),
    }


def poisson_stream(n_jobs, rate, seed, make):
    """n_jobs requests with exponential inter-arrival times of mean 1/rate;
    make(i, rng) returns the job of request i."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    for i in range(n_jobs):
        t += rng.exponential(1.0 / rate)
        out.append(Request(rid=i, arrival=t, job=make(i, rng)))
    return out


def mixed_job(i, rng, precision=PREC_F32, n_lo=1e4, n_hi=1e6, phi_lo=0.30, phi_hi=0.50, place=None):
    """A 2D or 3D monodisperse job: N log-uniform in [n_lo, n_hi], target
    uniform in [phi_lo, phi_hi], RSA start at 0.1 in a unit box.  place(dim,
    box, radii, seed) -> positions, if given, places the start ahead of time
    (the job then carries explicit positions)."""
    dim = 2 if rng.random() < 0.5 else 3
    n = int(math.floor(n_lo * (n_hi / n_lo) ** rng.random()))
    phi = phi_lo + (phi_hi - phi_lo) * rng.random()
    if dim == 2:
        r_t = math.sqrt(phi / (n * math.pi))
    else:
        r_t = (phi * 3.0 / (4.0 * math.pi * n)) ** (1.0 / 3.0)
    r0 = r_t * (0.1 / phi) ** (1.0 / dim)
    if place is not None:
        radii = np.full(n, r0)
        x = place(dim, (1.0,) * dim, radii, 1000 + i)
        return make_job(dim, (1.0, 1.0, 1.0), radii, phi, seed=1000 + i, c_m=0.1 * r_t,
                        precision=precision, init="explicit", positions=x)
    return make_job(dim, (1.0, 1.0, 1.0), ("mono", r0), phi, seed=1000 + i, n=n, c_m=0.1 * r_t,
                    precision=precision, init="rsa", f0=0.1)
