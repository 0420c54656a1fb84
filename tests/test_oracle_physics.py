"""Pins of the whole oracle step against the paper's static checks (Sec. 3.1).

Coexistence (Sec. 3.1.1, Eq. Maxwell_equal_area): a flat liquid slab in a periodic
column relaxes to bulk densities that converge to the Maxwell construction as the
interface widens ("thermodynamically converged in the limit dr/W -> 0").  The
scheme is second order in dr/W, so the vapour error of two widths W1 < W2 is
extrapolated as e(W) = e_inf + c/W^2, and e_inf must lie within 1% at T/Tc = 0.6,
0.7, 0.8 and 0.9 (the liquid is within 0.1% at each width).

Laplace's law (Sec. 3.1.2, Eq. Laplace_equimolar): for a static drop the pressure
jump times the equimolar radius, Delta P R_e, is the surface tension and does not
depend on the radius; two drops of radii 16 and 24 agree within 1%.

The steady states are independent of the viscosity (the step's equilibria do not
depend on omega once the fluid is at rest, and Phi vanishes there), so the runs
use nu = 0.5, which damps the acoustic sloshing of the column fastest.  Every run
is a one-dimensional column (ny = 1) long enough, about 40 W, that the two
interfaces do not feel each other.  The runs execute in parallel processes.
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

PAPER_EOS = dict(a=0.003, b=0.095, R=1.0, acentric=0.344)

# (T/Tc, kappa, column length): two interface widths per temperature
FLAT_RUNS = [(0.6, 0.02, 320), (0.6, 0.035, 400),
             (0.7, 0.005, 200), (0.7, 0.02, 320),
             (0.8, 0.002, 160), (0.8, 0.005, 240),
             (0.9, 0.001, 200), (0.9, 0.002, 280)]
DROP_RUNS = [(0.7, 0.005, 64, 16.0), (0.7, 0.005, 96, 24.0)]


def _flat(args):
    """Steady flat interface: (T, kappa, L) -> vapour and liquid densities, W."""
    os.environ["OMP_NUM_THREADS"] = "1"
    import oracle as O
    from oracle import thermo
    Tr, kappa, L = args
    rv, rl, _ = thermo.maxwell(Tr, **PAPER_EOS)
    p = O.make_params(2, L, 1, T_over_Tc=Tr, kappa=kappa, nu_liquid=0.5, rho_liquid=rl, rho_vapour=rv, **PAPER_EOS)
    x = np.arange(L)
    d = np.abs(x - (L - 1) / 2) - L / 4          # liquid in the middle half
    rho = (0.5 * (rl + rv) - 0.5 * (rl - rv) * np.tanh(2 * d / 6.0)).reshape(1, 1, L)
    f = O.init_equilibrium(p, rho, np.zeros((2, 1, 1, L)))
    prev, quiet = None, 0
    for _ in range(100):                       # at most 200,000 steps
        f, _ = O.run(p, f, 2000)
        r, _ = O.macroscopic(p, f)
        r = r[0, 0]
        ev = r[0] / rv - 1
        quiet = quiet + 1 if prev is not None and abs(ev - prev) < 1e-5 else 0
        if quiet >= 3:
            break
        prev = ev
    W = (rl - rv) / np.max(np.abs(np.diff(r)))
    return dict(T=Tr, kappa=kappa, L=L, ev=float(ev), el=float(r[L // 2] / rl - 1), W=float(W))


def _drop(args):
    """Static drop: Delta P R_e after the drop has settled."""
    os.environ["OMP_NUM_THREADS"] = "1"
    import oracle as O
    from oracle import thermo
    from paper_2201_12404_gb300 import inputs as I
    Tr, kappa, n, R = args
    rv, rl, _ = thermo.maxwell(Tr, **PAPER_EOS)
    p = O.make_params(2, n, n, T_over_Tc=Tr, kappa=kappa, nu_liquid=0.5, rho_liquid=rl, rho_vapour=rv, **PAPER_EOS)
    rho = I.drop((1, n, n), ((n - 1) / 2, (n - 1) / 2, 0), R, rl, rv, 6.0, D=2)
    f = O.init_physical(p, rho, np.zeros((2, 1, n, n)))
    f, _ = O.run(p, f, 3000)
    r, _ = O.macroscopic(p, f)
    r = r[0]
    r_in, r_out = r[n // 2, n // 2], r[0, 0]
    Re = np.sqrt(np.sum(r - r_out) / (np.pi * (r_in - r_out)))
    dP = thermo.pressure(r_in, T_over_Tc=Tr, **PAPER_EOS) - thermo.pressure(r_out, T_over_Tc=Tr, **PAPER_EOS)
    return dict(T=Tr, R=R, sigma=float(dP * Re), Re=float(Re))


def _run(job):
    kind, args = job
    return _flat(args) if kind == "flat" else _drop(args)


@pytest.fixture(scope="module")
def steady_states():
    jobs = [("flat", a) for a in FLAT_RUNS] + [("drop", a) for a in DROP_RUNS]
    with mp.get_context("spawn").Pool(min(len(jobs), os.cpu_count() or 2)) as pool:
        res = pool.map(_run, jobs)
    return [r for r in res if "ev" in r], [r for r in res if "sigma" in r]


@pytest.mark.slow
@pytest.mark.parametrize("T", [0.6, 0.7, 0.8, 0.9])
def test_flat_interface_converges_to_maxwell(steady_states, T):
    flats, _ = steady_states
    a, b = sorted([r for r in flats if r["T"] == T], key=lambda r: r["W"])
    assert a["W"] < b["W"]
    for r in (a, b):
        assert abs(r["el"]) < 1e-3, r
    # the vapour error shrinks as the interface widens, and its W -> infinity limit is within 1%
    assert abs(b["ev"]) < abs(a["ev"]), (a, b)
    c = (a["ev"] - b["ev"]) / (a["W"] ** -2 - b["W"] ** -2)
    e_inf = b["ev"] - c * b["W"] ** -2
    assert abs(e_inf) < 1e-2, (a, b, e_inf)


@pytest.mark.slow
def test_laplace_law_delta_p_times_radius_is_constant(steady_states):
    _, drops = steady_states
    s = sorted(drops, key=lambda r: r["R"])
    assert abs(s[0]["Re"] - 16) < 1.5 and abs(s[1]["Re"] - 24) < 1.5
    assert s[0]["sigma"] > 0
    assert abs(s[1]["sigma"] / s[0]["sigma"] - 1) < 1e-2, s
