"""Batched persistent stepping (lbm_batch_*): many D2Q9 domains of uneven sizes
advanced by one cooperative launch must give, domain by domain, exactly the
populations that stepping each domain alone gives (same per-tile arithmetic),
whatever the tile shape the tuner picks."""
import os
import tempfile

import numpy as np
import pytest

from cases import case, drop_state, lbm_params
from paper_2201_12404_gb300 import lbm

pytestmark = pytest.mark.gpu

JOBS = [
    dict(D=2, nx=64, ny=48, Tr=0.8),
    dict(D=2, nx=97, ny=33, Tr=0.7, walls=True),
    dict(D=2, nx=33, ny=70, Tr=0.9),
    dict(D=2, nx=130, ny=29, Tr=0.6, walls=True, kappa=0.005),
    dict(D=2, nx=5, ny=5, Tr=0.8, kappa=0.0),
    dict(D=2, nx=48, ny=40, Tr=0.7, gamma_mode=1, gamma_value=2.0),  # SRT (LBGK limit) job
]


def _domains(precision, states):
    out = []
    for j, kw in enumerate(JOBS):
        c = case(**kw, precision=precision)
        dom = lbm.Domain(lbm_params(c))
        dom.lbm_write_populations(states[j])
        out.append(dom)
    return out


def _states(precision):
    st = []
    for j, kw in enumerate(JOBS):
        f = drop_state(case(**kw, precision=precision), seed=40 + j)
        if precision == lbm.LBM_FP32:
            f = f.astype(np.float32).astype(np.float64)
        st.append(f)
    return st


@pytest.mark.parametrize("precision", [lbm.LBM_FP32, lbm.LBM_FP64, lbm.LBM_FP16DEV], ids=["fp32", "fp64", "fp16dev"])
def test_batch_equals_single_domain_steps(precision):
    st = _states(precision)
    alone = _domains(precision, st)
    batched = _domains(precision, st)
    # different A-A parities inside one batch: advance one job by a step first
    alone[1].lbm_step(1)
    batched[1].lbm_step(1)
    with lbm.Batch(batched) as b:
        for n in (3, 3, 4):  # repeated nsteps replays the captured graph
            b.lbm_batch_step(n)
            for d in alone:
                d.lbm_step(n)
        b.lbm_batch_synchronize()
        info = b.lbm_batch_info()
    for a, bd in zip(alone, batched):
        fa, fb = a.lbm_read_populations(), bd.lbm_read_populations()
        assert np.isfinite(fa).all()
        assert np.array_equal(fa, fb)
    assert info["grid"] >= 1
    for d in alone + batched:
        d.close()


def test_tuner_picks_a_shape_caches_it_and_keeps_results():
    st = _states(lbm.LBM_FP32)
    alone = _domains(lbm.LBM_FP32, st)
    batched = _domains(lbm.LBM_FP32, st)
    with tempfile.TemporaryDirectory() as tmp:
        cache = os.path.join(tmp, "tune.jsonl")
        with lbm.Batch(batched) as b:
            b.lbm_batch_tune(3, cache)
            first = b.lbm_batch_info()["block"]
            # tuning ran on copies: the jobs themselves did not advance
            for a, bd in zip(alone, batched):
                assert np.array_equal(a.lbm_read_populations(), bd.lbm_read_populations())
            b.lbm_batch_step(5)
            b.lbm_batch_synchronize()
        assert os.path.exists(cache)
        line = open(cache).read()
        assert '"block"' in line and '"key"' in line
        with lbm.Batch(batched) as b2:
            b2.lbm_batch_tune(3, cache)  # served from the cache
            assert b2.lbm_batch_info()["block"] == first
    for d in alone:
        d.lbm_step(5)
    for a, bd in zip(alone, batched):
        assert np.array_equal(a.lbm_read_populations(), bd.lbm_read_populations())
    for d in alone + batched:
        d.close()


def test_batch_rejects_mixed_precision_and_3d():
    a = lbm.Domain(lbm_params(case(2, 16, 16, precision=lbm.LBM_FP32)))
    b = lbm.Domain(lbm_params(case(2, 16, 16, precision=lbm.LBM_FP64)))
    c = lbm.Domain(lbm_params(case(3, 8, 8, 8, precision=lbm.LBM_FP32)))
    with pytest.raises(lbm.LBMError) as e:
        lbm.Batch([a, b])
    assert e.value.status == lbm.LBM_ERR_INVALID_ARG
    with pytest.raises(lbm.LBMError):
        lbm.Batch([a, c])
    with pytest.raises(lbm.LBMError):
        lbm.Batch([a, a])
    for d in (a, b, c):
        d.close()


def test_a_grid_barrier_wait_that_runs_out_reports_timeout_and_the_device_stays_usable():
    """The bounded device-side waits of the batched kernel, made to run out without
    any fault: block 0 skips its arrival at the grid barriers (a test switch), the
    other blocks' waits give up after a short poll limit (~2 ms), the kernel stops
    and lbm_batch_synchronize reports LBM_ERR_TIMEOUT.  A fresh batch on the same
    device then steps exactly as single domains do."""
    c = case(2, 16, 16, precision=lbm.LBM_FP32)
    f0 = drop_state(c).astype(np.float32).astype(np.float64)
    doms = []
    for _ in range(2):
        d = lbm.Domain(lbm_params(c))
        d.lbm_write_populations(f0)
        doms.append(d)
    b = lbm.Batch(doms)
    assert b.lbm_batch_info()["grid"] >= 2
    b.lbm_batch_set_wait(20000, skip_arrival=True)
    b.lbm_batch_step(2)
    with pytest.raises(lbm.LBMError) as e:
        b.lbm_batch_synchronize()
    assert e.value.status == lbm.LBM_ERR_TIMEOUT
    b.close()
    for d in doms:
        d.close()
    # the context is intact: a fresh batch gives the single-domain result
    alone = lbm.Domain(lbm_params(c))
    alone.lbm_write_populations(f0)
    fresh = [lbm.Domain(lbm_params(c)) for _ in range(2)]
    for d in fresh:
        d.lbm_write_populations(f0)
    with lbm.Batch(fresh) as b2:
        b2.lbm_batch_step(2)
        b2.lbm_batch_synchronize()
    alone.lbm_step(2)
    ref = alone.lbm_read_populations()
    for d in fresh:
        assert np.array_equal(d.lbm_read_populations(), ref)
    for d in fresh + [alone]:
        d.close()
