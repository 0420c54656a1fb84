"""Host buffers of lbm_host_alloc: the host-array calls give the same results
through them as through ordinary numpy arrays (they only change where the host
side of the copies lives), the buffers are page-locked and aligned, and
lbm_host_free takes back exactly what lbm_host_alloc gave."""
import ctypes
import os

import numpy as np
import pytest

from cases import case, lbm_params
from paper_2201_12404_gb300 import lbm

pytestmark = pytest.mark.gpu


class _PointerAttributes(ctypes.Structure):
    # the runtime's struct cudaPointerAttributes, reserved words included (the call
    # writes all of them)
    _fields_ = [("type", ctypes.c_int), ("device", ctypes.c_int), ("devicePointer", ctypes.c_void_p),
                ("hostPointer", ctypes.c_void_p), ("reserved", ctypes.c_long * 8)]


def _memory_type(ptr):
    """cudaPointerGetAttributes(ptr).type through the CUDA runtime the library loaded
    (0 unregistered host memory, 1 registered host memory, 2 device, 3 managed)."""
    lbm.load()
    path = next(line.split()[-1] for line in open("/proc/self/maps") if "libcudart.so" in line)
    rt = ctypes.CDLL(path)
    attr = _PointerAttributes()
    assert rt.cudaPointerGetAttributes(ctypes.byref(attr), ctypes.c_void_p(ptr)) == 0
    return attr.type


def _thp_bytes():
    try:
        if "[never]" in open("/sys/kernel/mm/transparent_hugepage/enabled").read():
            return 0
        return int(open("/sys/kernel/mm/transparent_hugepage/hpage_pmd_size").read())
    except OSError:
        return 0


@pytest.mark.parametrize("D", [3, 2], ids=["d3q27", "d2q9"])
def test_fields_through_host_buffers_equal_numpy_arrays(D):
    dims = dict(nx=40, ny=22, nz=13) if D == 3 else dict(nx=70, ny=37)
    c = case(D, **dims, precision=lbm.LBM_FP32, walls=True)
    rng = np.random.default_rng(20220128)
    shape = (c["nz"], c["ny"], c["nx"]) if D == 3 else (c["ny"], c["nx"])
    N = int(np.prod(shape))
    rho = 1.0 + 0.05 * rng.standard_normal(N)
    u = [0.01 * rng.standard_normal(N) for _ in range(D)]
    nb = N * 8
    with lbm.HostBuffer((1 + D) * nb) as hin, lbm.HostBuffer((1 + D) * nb) as hout:
        for k, a in enumerate([rho] + u):
            np.copyto(hin.array(np.float64, N, k * nb), a)
        ptrs_in = [hin.ptr + k * nb for k in range(1 + D)] + ([None] if D == 2 else [])
        ptrs_out = [hout.ptr + k * nb for k in range(1 + D)] + ([None] if D == 2 else [])
        a, b = lbm.Domain(lbm_params(c)), lbm.Domain(lbm_params(c))
        a.lbm_init_fields(rho.reshape(shape), [x.reshape(shape) for x in u])
        b.lbm_init_fields_ptr(*ptrs_in)
        for d in (a, b):
            d.lbm_step(5)
        ra, ua = a.lbm_read_macroscopic()
        b.lbm_read_macroscopic_ptr(*ptrs_out)
        assert np.array_equal(a.lbm_read_populations(), b.lbm_read_populations())
        assert np.array_equal(np.ravel(ra), hout.array(np.float64, N, 0))
        for k in range(D):
            assert np.array_equal(np.ravel(ua[k]), hout.array(np.float64, N, (1 + k) * nb))
        a.close()
        b.close()


def test_host_buffers_are_aligned_page_locked_and_freed_once():
    L = lbm.load()
    huge = _thp_bytes()
    page = os.sysconf("SC_PAGESIZE")
    sizes = (1, 3 * page + 5, 2 * max(huge, page))
    bufs = [lbm.HostBuffer(n) for n in sizes]
    for n, hb in zip(sizes, bufs):
        # huge-page aligned from half a huge page on, page aligned below
        assert hb.ptr % (huge if huge and n >= huge // 2 else page) == 0
        v = hb.array(np.uint8, hb.nbytes)
        assert not v.any()  # zero-filled
        v[:] = 7
        assert _memory_type(hb.ptr) == 1  # cudaMemoryTypeHost: registered, page-locked
        assert _memory_type(hb.ptr + hb.nbytes - 1) == 1
    p = bufs[0].ptr
    for hb in bufs:
        hb.close()
    # freed once: a second free of the same pointer is refused
    assert L.lbm_host_free(ctypes.c_void_p(p)) == lbm.LBM_ERR_INVALID_ARG
    assert L.lbm_host_free(None) == lbm.LBM_OK
