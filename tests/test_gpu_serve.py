"""The job server on the GPU: jobs arriving while others run are admitted as
memory and slots free up, and each job's result is the same alone and in the mix."""
import numpy as np
import pytest

from paper_2201_12404_gb300 import lbm, serve

pytestmark = pytest.mark.gpu


def small_jobs():
    r = np.random.Generator(np.random.PCG64(11))
    jobs = []
    for k in range(10):
        D = 2 if k % 2 == 0 else 3
        side = int(r.integers(64, 160)) if D == 2 else int(r.integers(24, 40))
        R = r.uniform(0.15, 0.25) * side
        jobs.append(serve.JobSpec(job_id=k, D=D, nx=side, ny=side, nz=side if D == 3 else 1,
                                  T_over_Tc=float(r.uniform(0.6, 0.9)), nu=float(r.uniform(0.02, 0.05)), R=R,
                                  film=0.2 * side / R, U=float(r.uniform(0.0, 0.03)), steps=int(r.integers(100, 400))))
    return jobs


def test_mix_equals_alone_and_admission_is_continuous():
    jobs = small_jobs()
    arrivals = serve.poisson_arrivals(len(jobs), 200.0, 11)
    fps = sorted(lbm.lbm_footprint_bytes(j.params()) for j in jobs)
    budget = fps[-1] + fps[-2] + fps[0]          # a few jobs at a time
    sample = (0, 3, 4, 7, 9)                     # five jobs, both lattices
    rep = serve.serve(jobs, arrivals, budget, slice_steps=50, keep_results=sample)
    assert rep["completed"] + rep["failed"] == len(jobs)
    assert rep["failed"] == 0, rep["failures"]
    assert rep["peak_resident_bytes"] <= budget
    assert rep["admissions_while_busy"] > 0
    for jid in sample:
        rho_mix, u_mix = rep["results"][jid]
        rho_a, u_a = serve.run_alone(jobs[jid])
        assert np.max(np.abs(rho_mix - rho_a)) <= 1e-6 * np.max(rho_a)
        assert np.max(np.abs(u_mix - u_a)) <= 1e-6 * max(np.max(np.abs(u_a)), 1e-12)
