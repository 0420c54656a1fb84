"""lbm_step_noalloc: stepping caller-owned device populations without any
device allocation (for callers that cannot allocate: a framework that owns the
whole memory pool, a memory-capped process).  Its output must match the
handle-based lbm_step on the same state, call after call, within the parity
tolerances of the GPU tests, and the FP64 oracle within the same per-step bounds.
This file is collected last on purpose."""
import numpy as np
import pytest

import oracle as O
from cases import case, drop_state, lbm_params, oracle_params
from paper_2201_12404_gb300 import lbm

pytestmark = pytest.mark.gpu

TOL = {lbm.LBM_FP64: 1e-12, lbm.LBM_FP32: 2e-6}


def _scaled_diff(a, b, D):
    w = {2: np.array([1 / 36, 1 / 9, 1 / 36, 1 / 9, 4 / 9, 1 / 9, 1 / 36, 1 / 9, 1 / 36])}
    if D == 3:
        w1 = np.array([1 / 6, 2 / 3, 1 / 6])
        w3 = np.einsum("i,j,k->kji", w1, w1, w1).reshape(-1)
        wq = w3
    else:
        wq = w[2]
    rho = b.sum(axis=0, keepdims=True)
    return np.max(np.abs(a - b) / (wq.reshape(-1, 1, 1, 1) * rho))


@pytest.mark.parametrize("D,dims,precision", [
    (3, dict(nx=24, ny=16, nz=12, walls=True), lbm.LBM_FP32),
    (2, dict(nx=70, ny=37), lbm.LBM_FP64),
])
def test_noalloc_matches_lbm_step_on_two_calls(D, dims, precision):
    import torch
    c = case(D, **dims, precision=precision)
    f0 = drop_state(c)
    if precision == lbm.LBM_FP32:
        f0 = f0.astype(np.float32).astype(np.float64)
    p = lbm_params(c)
    dtype = torch.float32 if precision == lbm.LBM_FP32 else torch.float64
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    p.stream = stream.cuda_stream
    dev = torch.from_numpy(f0).to(dtype).cuda().contiguous()  # owned by the caller
    with lbm.Domain(lbm_params(c)) as dom:
        dom.lbm_write_populations(f0)
        for call in range(2):
            dom.lbm_step(2)
            ref = dom.lbm_read_populations()
            lbm.lbm_step_noalloc(p, dev.data_ptr(), 2)
            torch.cuda.synchronize()
            assert lbm.lbm_noalloc_status() == lbm.LBM_OK
            got = dev.double().cpu().numpy()
            assert np.isfinite(got).all()
            err = _scaled_diff(got, ref, D)
            assert err <= TOL[precision], (call, err)
    # both calls together against the oracle: four steps
    fo, _ = O.run(oracle_params(c), f0, 4)
    assert _scaled_diff(got, fo, D) <= 4 * TOL[precision]


def test_noalloc_rejects_beyond_scratch_and_odd_steps():
    import torch
    torch.cuda.set_device(0)
    c = case(3, 128, 128, 128, precision=lbm.LBM_FP32)
    p = lbm_params(c)
    dummy = torch.zeros(16, device="cuda")
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_step_noalloc(p, dummy.data_ptr(), 2)
    assert e.value.status == lbm.LBM_ERR_INVALID_ARG
    small = lbm_params(case(2, 16, 16, precision=lbm.LBM_FP32))
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_step_noalloc(small, dummy.data_ptr(), 3)
    assert e.value.status == lbm.LBM_ERR_INVALID_ARG
    # populations that do not start on a float32 boundary are refused before any launch
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_step_noalloc(small, dummy.data_ptr() + 2, 2)
    assert e.value.status == lbm.LBM_ERR_INVALID_ARG


def test_noalloc_status_reports_an_instability():
    """A non-finite population makes the density non-finite: the steps complete and
    lbm_noalloc_status reports LBM_ERR_UNSTABLE; a clean state afterwards reads OK
    again (each call clears the flag word)."""
    import torch
    torch.cuda.set_device(0)
    c = case(2, 32, 20, precision=lbm.LBM_FP64)
    p = lbm_params(c)
    p.stream = torch.cuda.current_stream().cuda_stream
    f0 = drop_state(c)
    bad = f0.copy()
    bad[4, 0, 7, 9] = np.nan
    dev = torch.from_numpy(bad).cuda().contiguous()
    lbm.lbm_step_noalloc(p, dev.data_ptr(), 2)
    torch.cuda.synchronize()
    assert lbm.lbm_noalloc_status() == lbm.LBM_ERR_UNSTABLE
    dev = torch.from_numpy(f0).cuda().contiguous()
    lbm.lbm_step_noalloc(p, dev.data_ptr(), 2)
    torch.cuda.synchronize()
    assert lbm.lbm_noalloc_status() == lbm.LBM_OK
