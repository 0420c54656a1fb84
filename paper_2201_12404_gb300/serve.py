"""Continuous-batching job server for two-phase lattice Boltzmann simulations.

A request is a simulation job (lattice, size, temperature, viscosity, drop/film
geometry, step count).  The server keeps every admitted job's populations
resident on the GPU, admits waiting jobs whenever slots and HBM free up
(admission by lbm_footprint_bytes against a byte budget), and advances the
resident set in time slices: the resident D2Q9 jobs through one persistent
batched launch (lbm_batch_step) kept across slices, every D3Q27 job on its own
CUDA stream, so that their work overlaps on the device; the host runs a slice
ahead of the device and polls completions with events.  A job whose density turns
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


# Device throughput the arrival rate is sized against (lattice updates per second):
# about that of the step on a large D3Q27 domain, which dominates the mix's work.
CAPACITY_LUPS = 12e9


def rate_for_load(jobs, load=0.8, capacity=CAPACITY_LUPS):
    """Arrival rate (jobs per second) that offers `load` times the capacity."""
    return load * len(jobs) / (sum(j.N * j.steps for j in jobs) / capacity)


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
    """Resident domains and their slices of steps.

    Every D2Q9 job runs on one shared stream, the resident D2Q9 jobs with at least a
    slice of steps left as one persistent batch (lbm_batch_step), rebuilt only when
    that set changes; a D2Q9 job with fewer steps left finishes them with its own
    lbm_step on the same stream.  Every D3Q27 job has a stream of its own.  The host
    enqueues slice after slice and stays at most `in_flight` slices ahead of the
    device (it waits on the events of older slices); a job's completion is an event
    recorded after its last step, polled without blocking, and an instability
    surfaces through the library's non-blocking flag poll (lbm_step(0))."""

    def __init__(self, in_flight=2):
        import torch
        self.torch = torch
        lbm.load()
        self.in_flight = in_flight
        self.s2 = torch.cuda.Stream()     # all D2Q9 jobs
        self.doms = {}                   # job_id -> [spec, Domain, remaining steps, stream, done event]
        self.coex = {}
        self.batch, self.batch_ids = None, ()
        self.slices = []                 # events of the slices in flight
        self.batch_builds = 0

    def _coexistence(self, T):
        if T not in self.coex:
            self.coex[T] = lbm.lbm_coexistence(lbm.lbm_default_params(T_over_Tc=T, **WL.PAPER_EOS))
        return self.coex[T]

    def start(self, spec: JobSpec):
        rv, rl, _ = self._coexistence(spec.T_over_Tc)
        wl = spec.workload()
        stream = self.s2 if spec.D == 2 else self.torch.cuda.Stream()
        p = spec.params(rv=rv, rl=rl)
        p.stream = stream.cuda_stream
        dom = lbm.Domain(p)
        # the geometry of WL.initial_fields, built on the GPU: no host fields to
        # compute or copy while other jobs wait for their next slice
        dom.lbm_init_drop_on_film(wl.R, wl.film * wl.R, 2.0 * wl.W, wl.U, wl.W)
        self.doms[spec.job_id] = [spec, dom, spec.steps, stream, None]

    def _drop_batch(self):
        if self.batch is not None:
            self.batch.close()
        self.batch, self.batch_ids = None, ()

    def slice(self, slice_steps):
        """Enqueue up to slice_steps steps of every resident job that has steps left."""
        while len(self.slices) >= self.in_flight:
            for ev in self.slices.pop(0):
                ev.synchronize()
        evs = []
        two = [v for v in self.doms.values() if v[0].D == 2 and v[2] > 0]
        full = tuple(sorted(v[0].job_id for v in two if v[2] >= slice_steps))
        if full:
            if full != self.batch_ids:
                self._drop_batch()
                self.batch = lbm.Batch([self.doms[j][1] for j in full])
                self.batch_ids = full
                self.batch_builds += 1
            self.batch.lbm_batch_step(slice_steps)
            for j in full:
                self.doms[j][2] -= slice_steps
        for v in two:
            if 0 < v[2] < slice_steps:
                v[1].lbm_step(v[2])
                v[2] = 0
        if two:
            ev = self.torch.cuda.Event()
            ev.record(self.s2)
            evs.append(ev)
            for v in two:
                if v[2] == 0 and v[4] is None:
                    v[4] = ev
        for v in self.doms.values():
            if v[0].D == 3 and v[2] > 0:
                k = min(slice_steps, v[2])
                v[1].lbm_step(k)
                v[2] -= k
                ev = self.torch.cuda.Event()
                ev.record(v[3])
                evs.append(ev)
                if v[2] == 0:
                    v[4] = ev
        self.slices.append(evs)

    def idle(self):
        """Whether no resident job has steps left to enqueue."""
        return all(v[2] == 0 for v in self.doms.values())

    def poll(self):
        """Jobs that have finished or failed, without waiting for running work:
        (finished: {id: (rho, u)}, failed: {id: message})."""
        finished, failed = {}, {}
        for jid, (spec, dom, rem, stream, done) in list(self.doms.items()):
            try:
                dom.lbm_step(0)   # surfaces an instability found by earlier steps
            except lbm.LBMError as e:
                failed[jid] = str(e)
                continue
            if done is not None and done.query():
                try:
                    dom.lbm_synchronize()
                    finished[jid] = dom.lbm_read_macroscopic()
                except lbm.LBMError as e:
                    failed[jid] = str(e)
        gone = list(finished) + list(failed)
        if any(j in self.batch_ids for j in gone):
            self._drop_batch()
        for jid in gone:
            self.doms[jid][1].close()
            del self.doms[jid]
        return finished, failed


def run_alone(spec: JobSpec):
    """The job on its own: create, init, step, read (the reference for the mix)."""
    ex = GpuExecutor()
    ex.start(spec)
    dom = ex.doms[spec.job_id][1]
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
        if ex.idle():
            time.sleep(0.0005)  # only completions to wait for
        else:
            ex.slice(slice_steps)
        finished, failed = ex.poll()
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
                batch_builds=getattr(ex, "batch_builds", None), failures=fail, results=results)


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
    rate = args.rate or rate_for_load(jobs)
    arrivals = poisson_arrivals(len(jobs), rate, args.seed)
    rep = serve(jobs, arrivals, int(args.budget_frac * free), slice_steps=args.slice)
    rep.pop("results")
    rep["rate_per_s"] = rate
    rep["scale"] = args.scale
    rep["failures"] = len(rep["failures"])
    print(json.dumps(rep))


if __name__ == "__main__":
    main()
