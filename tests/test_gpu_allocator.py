"""The device allocator hook of lbm_params, wired to PyTorch's caching allocator.

While a domain lives, torch.cuda.memory_allocated() grows by the domain's
footprint (lbm_footprint_bytes, up to the allocator's 512-byte rounding of each
buffer); after lbm_destroy it returns to where it was.  A domain whose buffers
come from the hook steps exactly like one on cudaMalloc memory, and both agree
with the oracle.
"""
import numpy as np
import pytest

import oracle as O
from cases import case, drop_state, lbm_params, oracle_params, rel_err
from paper_2201_12404_gb300 import lbm

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("D,precision", [(3, lbm.LBM_FP32), (2, lbm.LBM_FP64), (3, lbm.LBM_FP16DEV)],
                         ids=["d3q27_fp32", "d2q9_fp64", "d3q27_fp16dev"])
def test_torch_allocator_holds_the_domain(D, precision):
    dims = dict(nx=40, ny=24, nz=12) if D == 3 else dict(nx=64, ny=40)
    c = case(D, **dims, precision=precision)
    p = lbm.use_torch_allocator(lbm_params(c))
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    with lbm.Domain(p) as dom:
        held = torch.cuda.memory_allocated() - before
        fp = lbm.lbm_footprint_bytes(p)
        assert fp <= held <= fp + 6 * 512, (held, fp)
        dom.lbm_record_gamma(True)
        dom.lbm_write_populations(drop_state(c))
        dom.lbm_step(2)
        dom.lbm_synchronize()
        # the gamma record (N float pairs) comes from the hook too
        assert torch.cuda.memory_allocated() - before >= fp + 8 * dom.N
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == before


@pytest.mark.parametrize("D,precision", [(3, lbm.LBM_FP32), (2, lbm.LBM_FP64)], ids=["d3q27_fp32", "d2q9_fp64"])
def test_parity_with_the_torch_allocator(D, precision):
    dims = dict(nx=37, ny=13, nz=11) if D == 3 else dict(nx=70, ny=37)
    c = case(D, **dims, precision=precision)
    f0 = drop_state(c)
    if precision == lbm.LBM_FP32:
        f0 = f0.astype(np.float32).astype(np.float64)
    out = []
    for hook in (True, False):
        p = lbm_params(c)
        if hook:
            lbm.use_torch_allocator(p)
        with lbm.Domain(p) as dom:
            dom.lbm_write_populations(f0)
            dom.lbm_step(3)
            dom.lbm_synchronize()
            out.append(dom.lbm_read_populations())
    assert np.array_equal(out[0], out[1])
    fo, _ = O.run(oracle_params(c), f0, 3)
    tol = 4 * (2e-6 if precision == lbm.LBM_FP32 else 1e-12)
    assert rel_err(out[0], fo, D).max() <= tol


def test_allocator_refusal_is_out_of_memory():
    """A hook that returns NULL makes lbm_create_domain fail with LBM_ERR_OOM and
    release what it had already taken."""
    taken, freed = [], []

    def alloc(nbytes, ctx):
        if len(taken) >= 2:
            return None
        ptr = int(torch.cuda.caching_allocator_alloc(int(nbytes)))
        taken.append(ptr)
        return ptr

    def free(ptr, ctx):
        freed.append(int(ptr))
        torch.cuda.caching_allocator_delete(int(ptr))

    hooks = (lbm.DEV_ALLOC(alloc), lbm.DEV_FREE(free))
    c = case(3, 20, 12, 8, precision=lbm.LBM_FP32)
    p = lbm_params(c)
    p.dev_alloc, p.dev_free = hooks
    with pytest.raises(lbm.LBMError) as e:
        lbm.Domain(p)
    assert e.value.status == lbm.LBM_ERR_OOM
    assert sorted(taken) == sorted(freed) and len(taken) == 2
