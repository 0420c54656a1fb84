"""Host-only checks of the C ABI: the library loads, exports every entry point
that include/lbm.h declares, validates parameters and solves the Maxwell
construction on the host (no GPU work is launched here)."""
import ctypes
import os
import re
import subprocess

import pytest

from oracle import thermo
from paper_2201_12404_gb300 import lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm.h")


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(lbm.LIB_PATH):
        from paper_2201_12404_gb300 import build
        build.build()
    return lbm.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lbm_create_domain", "lbm_init_fields", "lbm_step", "lbm_read_macroscopic", "lbm_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(L):
    out = subprocess.run(["nm", "-D", "--defined-only", lbm.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (lbm_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert hasattr(L, n)


def test_params_struct_layout_matches_header(L):
    # offsets of the C struct, computed by the C compiler from the header
    src = r'''
#include <stddef.h>
#include <stdio.h>
#include "lbm.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(lbm_params), offsetof(lbm_params, a),
         offsetof(lbm_params, body_force), offsetof(lbm_params, bc), offsetof(lbm_params, gamma_value),
         offsetof(lbm_params, eos_fp64), offsetof(lbm_params, stream), offsetof(lbm_params, dev_alloc),
         offsetof(lbm_params, dev_free), offsetof(lbm_params, alloc_ctx));
  return 0;
}
'''
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        vals = [int(x) for x in subprocess.check_output([exe]).split()]
    P = lbm.lbm_params
    assert vals == [ctypes.sizeof(P), P.a.offset, P.body_force.offset, P.bc.offset, P.gamma_value.offset,
                    P.eos_fp64.offset, P.stream.offset, P.dev_alloc.offset, P.dev_free.offset,
                    P.alloc_ctx.offset]


def test_default_params_and_footprint(L):
    p = lbm.lbm_default_params()
    assert (p.lattice, p.precision, p.nx, p.ny, p.nz) == (lbm.LBM_D2Q9, lbm.LBM_FP32, 64, 64, 1)
    assert (p.a, p.b, p.acentric) == (0.003, 0.095, 0.344)
    fp = lbm.lbm_footprint_bytes(p)
    # 9 float32 populations per node plus 4 padded float32 auxiliary fields
    assert fp >= 9 * 4 * 64 * 64 + 4 * 4 * 68 * 68
    p3 = lbm.lbm_default_params(lattice=lbm.LBM_D3Q27, nx=512, ny=512, nz=256)
    assert lbm.lbm_footprint_bytes(p3) > 27 * 4 * 512 * 512 * 256
    p64 = lbm.lbm_default_params(lattice=lbm.LBM_D3Q27, precision=lbm.LBM_FP64, nx=512, ny=512, nz=256)
    assert lbm.lbm_footprint_bytes(p64) > 2 * 27 * 4 * 512 * 512 * 256


@pytest.mark.parametrize("overrides,needle", [
    (dict(nx=4), "nx and ny"),
    (dict(nz=3), "nz must be 1"),
    (dict(lattice=lbm.LBM_D3Q27, nz=4), "nz must be >= 5"),
    (dict(precision=7), "precision"),
    (dict(precision=-1), "precision"),
    (dict(nu_liquid=0.0), "viscosities"),
    (dict(rho_vapour=2.0), "rho_liquid > rho_vapour"),
    (dict(bc=(1, 0, 0, 0, 0, 0)), "pairs"),
    (dict(kappa=-1.0), "kappa"),
    (dict(eos_fp64=5), "eos_fp64"),
    (dict(gamma_mode=3), "gamma_mode"),
])
def test_invalid_params_rejected_without_gpu(L, overrides, needle):
    p = lbm.lbm_default_params(**overrides)
    assert lbm.lbm_footprint_bytes(p) == 0
    with pytest.raises(lbm.LBMError) as e:
        lbm.Domain(p)
    assert e.value.status == lbm.LBM_ERR_INVALID_ARG
    assert needle in str(e.value)


@pytest.mark.parametrize("Tr", [0.59, 0.7, 0.8, 0.9, 0.95])
def test_library_maxwell_matches_oracle(L, Tr):
    p = lbm.lbm_default_params(T_over_Tc=Tr)
    rv, rl, ps = lbm.lbm_coexistence(p)
    orv, orl, ops_ = thermo.maxwell(Tr, a=p.a, b=p.b, R=p.R, acentric=p.acentric)
    assert rv == pytest.approx(orv, rel=1e-9)
    assert rl == pytest.approx(orl, rel=1e-10)
    assert ps == pytest.approx(ops_, rel=1e-9)


def test_version_string(L):
    assert "sm_103a" in lbm.lbm_version()


@pytest.mark.parametrize("Tr,a", [(0.59, 0.003), (0.8, 0.003), (0.95, 0.003), (1.2, 0.003), (0.7, 2.0 / 49.0), (3.0, 0.003),
                                  (0.6, 0.5), (0.9, 0.5)])
def test_psi_sign_changes_match_oracle_sign(L, Tr, a):
    """The densities where the library flips s (Sec. 2.3) reproduce the oracle's
    pointwise sign of P - rho cs^2 on a dense sample of (0, 1/b), and the sign
    flips across each of them."""
    import numpy as np
    import oracle as O
    from cases import case, oracle_params
    p = lbm.lbm_default_params(T_over_Tc=Tr, a=a)
    changes, s0 = lbm.lbm_psi_sign_changes(p)
    assert len(changes) <= 3 and changes == sorted(changes) and s0 in (-1.0, 1.0)
    op = oracle_params(case(2, 8, 8, Tr=Tr, rho_l=2.0, rho_v=1.0))
    op.a = a
    top = 1.0 / p.b
    grid = np.concatenate([top * np.logspace(-12, -3, 400), np.linspace(top * 1e-3, top * (1 - 1e-9), 6000)])

    def lib_sign(r):
        return s0 * (-1.0) ** sum(1 for t in changes if r >= t)

    mismatches = [r for r in grid if lib_sign(r) != O.psi(op, float(r))[1]]
    assert not mismatches, mismatches[:5]
    for t in changes:
        below, above = t * (1 - 1e-12), t * (1 + 1e-12)
        assert O.psi(op, below)[1] == lib_sign(below) and O.psi(op, above)[1] == lib_sign(above)
        assert lib_sign(below) == -lib_sign(above)


def test_host_buffer_arguments_checked_before_any_cuda_call(L):
    """lbm_host_alloc/lbm_host_free refuse what they cannot serve before they map or
    register anything (the buffers themselves are tested on the GPU)."""
    p = ctypes.c_void_p(1234)
    assert L.lbm_host_alloc(0, ctypes.byref(p)) == lbm.LBM_ERR_INVALID_ARG and p.value is None
    assert L.lbm_host_alloc(64, None) == lbm.LBM_ERR_INVALID_ARG
    assert L.lbm_host_alloc(ctypes.c_size_t(-1).value, ctypes.byref(p)) == lbm.LBM_ERR_INVALID_ARG
    assert L.lbm_host_free(None) == lbm.LBM_OK
    assert L.lbm_host_free(ctypes.c_void_p(4096)) == lbm.LBM_ERR_INVALID_ARG
    with pytest.raises(ValueError):
        hb = lbm.HostBuffer.__new__(lbm.HostBuffer)
        hb.ptr, hb.nbytes = 0, 0
        hb.array("f8", 1)
