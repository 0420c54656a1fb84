"""Benchmark workload parameters, checked without a GPU: the viscosity rules, the
walls and the EOS scaling that each workload states."""
import dataclasses

from paper_2201_12404_gb300 import lbm
from paper_2201_12404_gb300 import workloads as WL


def test_viscosity_rules():
    rv, rl = 0.01, 8.0
    nu_l, nu_v = WL.viscosities(WL.DROP_IMPACT_3D, rv, rl)
    assert nu_l == WL.DROP_IMPACT_3D.nu_liquid and abs(nu_v - nu_l * (rl / rv) / 50.0) < 1e-15
    nu_l, nu_v = WL.viscosities(WL.DROP_IMPACT_3D_PAPER, rv, rl)
    assert nu_v == 15.0 * nu_l                       # Sec. 3.2: nu_v / nu_l = 15
    nu_l, nu_v = WL.viscosities(WL.STATIC_DROP_2D, rv, rl)
    assert nu_l == nu_v                              # uniform viscosity


def test_params_carry_walls_sizes_and_eos():
    wl = WL.DROP_IMPACT_3D
    p = WL.params(wl, lbm.LBM_FP32, rv=0.01, rl=8.0)
    assert (p.lattice, p.nx, p.ny, p.nz) == (lbm.LBM_D3Q27, 512, 512, 256)
    assert list(p.bc) == [0, 0, 0, 0, 1, 1]          # walls across z only
    assert (p.a, p.b, p.R, p.acentric) == (0.003, 0.095, 1.0, 0.344)
    p2 = WL.params(WL.DROP_IMPACT_2D, lbm.LBM_FP32, rv=0.01, rl=8.0)
    assert list(p2.bc)[:4] == [0, 0, 1, 1] and p2.nz == 1
    scaled = dataclasses.replace(wl, a_scale=0.25)
    assert WL.eos(scaled)["a"] == 0.25 * 0.003 and WL.params(scaled, lbm.LBM_FP32, rv=0.01, rl=8.0).a == 0.25 * 0.003


def test_coexistence_does_not_depend_on_a():
    """With T/Tc fixed, P scales with a (Tc is proportional to a), so the coexistence
    densities depend on b and T/Tc only: scaling a keeps the workloads' densities."""
    rv1, rl1 = WL.coexistence(WL.DROP_IMPACT_3D)
    rv2, rl2 = WL.coexistence(dataclasses.replace(WL.DROP_IMPACT_3D, a_scale=0.3))
    assert abs(rv2 / rv1 - 1) < 1e-9 and abs(rl2 / rl1 - 1) < 1e-9
