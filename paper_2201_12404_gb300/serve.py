"""Continuous-batching job server for two-phase lattice Boltzmann simulations.

A request is a simulation job (lattice, size, temperature, viscosity, drop/film
geometry, step count).  The server keeps every admitted job's populations
resident on the GPU, admits waiting jobs whenever slots and HBM free up
(admission by lbm_footprint_bytes against a byte budget), and advances the
resident set in time slices: all resident D2Q9 jobs of one precision through one
persistent batched launch (lbm_batch_step), every D3Q27 job on its own CUDA
stream, so that their work overlaps on the device.  A job whose density turns
non-finite or non-positive ends as failed (expected at the lowest viscosities)
and frees its slot.  Reported: p50/p99 latency (arrival to result), aggregate
MLUPS, failures.

  python -m paper_2201_12404_gb300.serve [--jobs 200] [--seed 20220128] [--scale 0.1]

The scheduling logic (Scheduler) is plain host code; the GPU work goes through
the C ABI (GpuExecutor).
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import inputs as I
from . import lbm
from . import workloads as WL


@dataclass
class JobSpec:
    job_id: int
    D: int
    nx: int
    ny: int
    nz: int
    T_over_Tc: float
    nu: float
    R: float           # drop radius
    film: float        # film thickness / R (0: no film)
    U: float           # impact speed
    steps: int
    precision: int = lbm.LBM_FP32
    kappa: float = 0.01
    seed: int = 0

    @property
    def N(self):
        return self.nx * self.ny * self.nz

    def workload(self) -> WL.Workload:
        return WL.Workload(name=f"job{self.job_id}", D=self.D, nx=self.nx, ny=self.ny, nz=self.nz,
                           T_over_Tc=self.T_over_Tc, kappa=self.kappa, nu_liquid=self.nu, mu_ratio=0.0,
                           R=self.R, U=self.U, film=self.film, walls_axis=self.D - 1, steps=self.steps)

    def params(self, rv=None, rl=None):
        return WL.params(self.workload(), self.precision, rv=rv, rl=rl)


def random_jobs(n_jobs, seed=I.SEED_BASE, scale=1.0):
    """The mixed request stream: half D2Q9 squares with sides log-uniform in [64, 1024],
    half D3Q27 cubes with sides log-uniform in [64, 256]; T/Tc ~ U[0.6, 0.9], nu ~ U[0.002, 0.05]
    (both phases), drop radius in [0.1, 0.25] of the side, film in [0.1, 0.3] of the
    side, U ~ U[0, 0.05], steps ~ U{1000..10000} scaled by `scale` (at least 20)."""
    r = I.rng(seed)
    jobs = []
    for k in range(n_jobs):
        D = 2 if r.random() < 0.5 else 3
        side = int(round(math.exp(r.uniform(math.log(64), math.log(1024 if D == 2 else 256)))))
        side = max(16, side)
        R = r.uniform(0.1, 0.25) * side
        film_h = r.uniform(0.1, 0.3) * side
        jobs.append(JobSpec(job_id=k, D=D, nx=side, ny=side, nz=side if D == 3 else 1,
                            T_over_Tc=r.uniform(0.6, 0.9), nu=r.uniform(0.002, 0.05), R=R,
                            film=film_h / R, U=r.uniform(0.0, 0.05),
                            steps=max(20, int(round(r.integers(1000, 10001) * scale))), seed=I.SEED_BASE + k))
    return jobs


def poisson_arrivals(n_jobs, rate_per_s, seed):
    """Arrival times (seconds from the start) of a seeded Poisson process."""
    gaps = I.rng(seed + 1).exponential(1.0 / rate_per_s, size=n_jobs)
    return np.cumsum(gaps) - gaps[0]


# ---------------------------------------------------------------------------
# Scheduling (host logic only)
# ---------------------------------------------------------------------------

@dataclass
class Scheduler:
    """FIFO admission by device-memory footprint and slot count."""
    budget_bytes: int
    max_slots: int = 64
    waiting: list = field(default_factory=list)
    resident: dict = field(default_factory=dict)   # job_id -> footprint
    peak_bytes: int = 0

    def used(self):
        return sum(self.resident.values())

    def submit(self, job, footprint):
        if footprint > self.budget_bytes:
            raise ValueError(f"job {job.job_id} needs {footprint} B, more than the whole budget")
        self.waiting.append((job, footprint))

    def admit(self):
        """Admit waiting jobs in arrival order while they fit; returns the admitted jobs."""
        out = []
        while self.waiting and len(self.resident) < self.max_slots:
            job, fp = self.waiting[0]
            if self.used() + fp > self.budget_bytes:
                break
            self.waiting.pop(0)
            self.resident[job.job_id] = fp
            out.append(job)
        self.peak_bytes = max(self.peak_bytes, self.used())
        return out

    def release(self, job_id):
        self.resident.pop(job_id, None)


# ---------------------------------------------------------------------------
# GPU execution
# ---------------------------------------------------------------------------

class GpuExecutor:
    """Resident domains, one batch for the D2Q9 jobs of a slice, streams for D3Q27."""

    def __init__(self):
        lbm.load()
        self.doms = {}        # job_id -> (spec, Domain, remaining steps)
        self.coex = {}

    def _coexistence(self, T):
        if T not in self.coex:
            self.coex[T] = lbm.lbm_coexistence(lbm.lbm_default_params(T_over_Tc=T, **WL.PAPER_EOS))
        return self.coex[T]

    def start(self, spec: JobSpec):
        rv, rl, _ = self._coexistence(spec.T_over_Tc)
        wl = spec.workload()
        dom = lbm.Domain(spec.params(rv=rv, rl=rl))
        rho, u = WL.initial_fields(wl, rv, rl)
        dom.lbm_init_fields(rho, u)
        self.doms[spec.job_id] = [spec, dom, spec.steps]

    def slice(self, slice_steps):
        """Advance every resident job by up to slice_steps; returns the finished and failed
        job ids as (finished: {id: (rho, u)}, failed: {id: message})."""
        two = [v for v in self.doms.values() if v[0].D == 2]
        three = [v for v in self.doms.values() if v[0].D == 3]
        failed = {}
        if two:
            k = min(slice_steps, min(v[2] for v in two))
            by_prec = {}
            for v in two:
                by_prec.setdefault(v[0].precision, []).append(v)
            batches = []
            for group in by_prec.values():
                b = lbm.Batch([v[1] for v in group])
                b.lbm_batch_step(k)
                batches.append((b, group))
            for v in two:
                v[2] -= k
        for v in three:
            k3 = min(slice_steps, v[2])
            try:
                v[1].lbm_step(k3)
            except lbm.LBMError as e:
                failed[v[0].job_id] = str(e)
            v[2] -= k3
        if two:
            for b, group in batches:
                try:
                    b.lbm_batch_synchronize()
                except lbm.LBMError:
                    pass  # the failing domains are found below
                b.close()
        finished = {}
        for jid, (spec, dom, rem) in list(self.doms.items()):
            if jid in failed:
                continue
            try:
                dom.lbm_synchronize()
            except lbm.LBMError as e:
                failed[jid] = str(e)
                continue
            if rem <= 0:
                finished[jid] = dom.lbm_read_macroscopic()
        for jid in list(finished) + list(failed):
            self.doms[jid][1].close()
            del self.doms[jid]
        return finished, failed


def run_alone(spec: JobSpec):
    """The job on its own: create, init, step, read (the reference for the mix)."""
    ex = GpuExecutor()
    ex.start(spec)
    spec_, dom, _ = ex.doms[spec.job_id]
    try:
        dom.lbm_step(spec.steps)
        dom.lbm_synchronize()
        out = dom.lbm_read_macroscopic()
    except lbm.LBMError as e:
        out = str(e)
    dom.close()
    return out


def serve(jobs, arrivals, budget_bytes, slice_steps=200, max_slots=64, executor=None, keep_results=()):
    """Serve `jobs` arriving at `arrivals` (seconds from the start).  Returns a report."""
    ex = executor or GpuExecutor()
    sched = Scheduler(budget_bytes=budget_bytes, max_slots=max_slots)
    t0 = time.perf_counter()
    nxt = 0
    arrival_of = {j.job_id: float(a) for j, a in zip(jobs, arrivals)}
    done, fail, results = {}, {}, {}
    overlap_admissions = 0
    lups_done = 0
    while len(done) + len(fail) < len(jobs):
        now = time.perf_counter() - t0
        while nxt < len(jobs) and arrivals[nxt] <= now:
            j = jobs[nxt]
            sched.submit(j, lbm.lbm_footprint_bytes(j.params(*_coex_pair(ex, j))))
            nxt += 1
        for j in sched.admit():
            if ex.doms:
                overlap_admissions += 1
            ex.start(j)
        if not ex.doms:
            # idle: wait for the next arrival
            if nxt < len(jobs):
                time.sleep(max(0.0, min(0.01, arrivals[nxt] - (time.perf_counter() - t0))))
            continue
        finished, failed = ex.slice(slice_steps)
        t = time.perf_counter() - t0
        for jid, res in finished.items():
            done[jid] = t - arrival_of[jid]
            sched.release(jid)
            spec = jobs[jid]
            lups_done += spec.N * spec.steps
            if jid in keep_results:
                results[jid] = res
        for jid, msg in failed.items():
            fail[jid] = msg
            sched.release(jid)
    wall = time.perf_counter() - t0
    lat = np.array(sorted(done.values())) if done else np.array([0.0])
    return dict(jobs=len(jobs), completed=len(done), failed=len(fail), wall_s=wall,
                p50_latency_s=float(np.percentile(lat, 50)), p99_latency_s=float(np.percentile(lat, 99)),
                aggregate_mlups=lups_done / wall / 1e6, peak_resident_bytes=sched.peak_bytes,
                budget_bytes=budget_bytes, admissions_while_busy=overlap_admissions,
                failures=fail, results=results)


def _coex_pair(ex, j):
    if isinstance(ex, GpuExecutor):
        rv, rl, _ = ex._coexistence(j.T_over_Tc)
        return rv, rl
    return None, None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=200)
    ap.add_argument("--seed", type=int, default=I.SEED_BASE)
    ap.add_argument("--scale", type=float, default=0.1, help="fraction of each job's 1000-10000 steps to run")
    ap.add_argument("--rate", type=float, default=None, help="arrivals per second (default: ~80%% load)")
    ap.add_argument("--budget-frac", type=float, default=0.8, help="fraction of free HBM the resident jobs may hold")
    ap.add_argument("--slice", type=int, default=200)
    args = ap.parse_args()
    import torch
    free, _ = torch.cuda.mem_get_info()
    jobs = random_jobs(args.jobs, args.seed, args.scale)
    total_lups = sum(j.N * j.steps for j in jobs)
    # ~80% load at an expected ~9 GLUPS of mixed work
    rate = args.rate or 0.8 * len(jobs) / (total_lups / 9e9)
    arrivals = poisson_arrivals(len(jobs), rate, args.seed)
    rep = serve(jobs, arrivals, int(args.budget_frac * free), slice_steps=args.slice)
    rep.pop("results")
    rep["rate_per_s"] = rate
    rep["scale"] = args.scale
    rep["failures"] = len(rep["failures"])
    print(json.dumps(rep))


if __name__ == "__main__":
    main()
