"""Host logic of the job server: seeded request stream, admission by footprint
budget and slots, continuous admission while jobs are resident, and the latency
report, with a fake executor in place of the GPU (no GPU work)."""
import numpy as np
import pytest

from paper_2201_12404_gb300 import lbm, serve


def test_request_stream_is_seeded_and_in_range():
    a = serve.random_jobs(50, seed=7, scale=1.0)
    b = serve.random_jobs(50, seed=7, scale=1.0)
    assert [dataclass_tuple(x) for x in a] == [dataclass_tuple(x) for x in b]
    for j in a:
        lo, hi = (64, 1024) if j.D == 2 else (64, 256)
        assert lo <= j.nx <= hi and j.nx == j.ny
        assert 0.6 <= j.T_over_Tc <= 0.9 and 0.002 <= j.nu <= 0.05
        assert 1000 <= j.steps <= 10000
    assert {j.D for j in a} == {2, 3}
    t = serve.poisson_arrivals(50, 10.0, 7)
    assert t[0] == 0.0 and np.all(np.diff(t) >= 0)


def dataclass_tuple(j):
    return (j.D, j.nx, j.ny, j.nz, round(j.T_over_Tc, 12), round(j.nu, 12), j.steps)


def test_scheduler_admits_by_footprint_and_slots():
    s = serve.Scheduler(budget_bytes=100, max_slots=2)
    jobs = serve.random_jobs(4, seed=1, scale=0.01)
    for j, fp in zip(jobs, (60, 30, 20, 50)):
        s.submit(j, fp)
    got = s.admit()
    assert [j.job_id for j in got] == [0, 1]          # third would exceed the 2 slots
    assert s.used() == 90
    s.release(0)
    got = s.admit()
    assert [j.job_id for j in got] == [2]             # 30 + 20 fits; the 50 waits (FIFO)
    assert s.peak_bytes <= 100
    with pytest.raises(ValueError):
        s.submit(jobs[0], 101)


class FakeExecutor:
    """Enqueues slices instantly; a job completes one poll after its last slice (as a
    device a slice behind the host would report it); records how many were resident
    together."""

    def __init__(self):
        self.doms = {}
        self.max_resident = 0
        self.slices = 0

    def start(self, spec):
        self.doms[spec.job_id] = [spec, None, spec.steps, None, None]
        self.max_resident = max(self.max_resident, len(self.doms))

    def slice(self, k):
        self.slices += 1
        for v in self.doms.values():
            if v[2] > 0:
                v[2] -= min(k, v[2])
                if v[2] == 0:
                    v[4] = self.slices

    def idle(self):
        return all(v[2] == 0 for v in self.doms.values())

    def poll(self):
        finished = {}
        for jid, v in list(self.doms.items()):
            if v[4] is not None and self.slices > v[4] or (v[4] is not None and self.idle()):
                finished[jid] = ("rho", "u")
                del self.doms[jid]
        return finished, {}


def test_serve_loop_admits_continuously_and_reports():
    jobs = serve.random_jobs(20, seed=3, scale=0.02)
    arr = serve.poisson_arrivals(20, 2000.0, 3)
    # a small budget: only a few jobs fit at a time, the rest wait and are admitted as others finish
    fps = [lbm.lbm_footprint_bytes(j.params()) for j in jobs]
    budget = int(sorted(fps)[-1] * 2.5)
    ex = FakeExecutor()
    rep = serve.serve(jobs, arr, budget, slice_steps=10, executor=ex)
    assert rep["completed"] == 20 and rep["failed"] == 0
    assert rep["peak_resident_bytes"] <= budget
    assert rep["admissions_while_busy"] > 0
    assert ex.max_resident >= 2
    assert rep["p99_latency_s"] >= rep["p50_latency_s"] >= 0
