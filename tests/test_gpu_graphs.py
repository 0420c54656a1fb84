"""lbm_step replays captured CUDA graphs of two steps once a domain has run two
plain steps (with timing off); the graphs hold the same kernels with the same
arguments, so a domain stepped through them must match, bit for bit, one stepped
kernel by kernel (timing on), over odd and even step counts, both A-A parities and
a gamma record switched on midway (which makes lbm_step capture new graphs)."""
import numpy as np
import pytest

import oracle as O
from cases import case, drop_state, lbm_params, oracle_params, rel_err
from paper_2201_12404_gb300 import lbm

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("D,precision", [(3, lbm.LBM_FP32), (2, lbm.LBM_FP32), (3, lbm.LBM_FP64), (2, lbm.LBM_FP16DEV)],
                         ids=["d3q27_fp32", "d2q9_fp32", "d3q27_fp64", "d2q9_fp16dev"])
def test_graph_replay_equals_kernel_by_kernel_steps(D, precision):
    dims = dict(nx=40, ny=22, nz=13) if D == 3 else dict(nx=70, ny=37)
    c = case(D, **dims, precision=precision, walls=True)
    f0 = drop_state(c)
    if precision == lbm.LBM_FP32:
        f0 = f0.astype(np.float32).astype(np.float64)
    plain, graphed = lbm.Domain(lbm_params(c)), lbm.Domain(lbm_params(c))
    for d in (plain, graphed):
        d.lbm_write_populations(f0)
    plain.lbm_set_timing(True)  # events between kernels: launched one at a time
    n0 = graphed.lbm_launch_count()
    for n in (2, 7, 4):
        plain.lbm_step(n)
        graphed.lbm_step(n)
    # 13 steps, 3 kernels each, however they were launched
    assert graphed.lbm_launch_count() - n0 == 13 * 3
    plain.lbm_record_gamma(True)
    graphed.lbm_record_gamma(True)
    for n in (5, 2):
        plain.lbm_step(n)
        graphed.lbm_step(n)
    plain.lbm_synchronize()
    graphed.lbm_synchronize()
    fa, fb = plain.lbm_read_populations(), graphed.lbm_read_populations()
    ga = plain.lbm_read_diag(with_gamma=True)["gamma"]
    gb = graphed.lbm_read_diag(with_gamma=True)["gamma"]
    assert np.isfinite(fb).all()
    assert np.array_equal(fa, fb)
    assert np.array_equal(ga, gb)
    if precision != lbm.LBM_FP16DEV:
        fo, _ = O.run(oracle_params(c), f0, 20)
        tol = 20 * (1e-12 if precision == lbm.LBM_FP64 else 2e-6)
        assert rel_err(fb, fo, D).max() <= tol
    plain.close()
    graphed.close()
