"""The window construction behind the full-size GPU parity test, checked on the
CPU: on domains small enough for the oracle to step whole, every checked node of
every window equals the same node of the whole-domain run (same arithmetic per
node, so bit for bit), across periodic seams and at the walls."""
import dataclasses

import numpy as np
import pytest

import oracle as O
from oracle import thermo
from paper_2201_12404_gb300 import workloads as WL
from windows import K, MARGIN, oracle_window, sample_nodes, window_axis

# larger than a window (2 MARGIN + VALID = 40 nodes) on every axis
SMALL = {
    3: dataclasses.replace(WL.DROP_IMPACT_3D, nx=48, ny=44, nz=42, R=8.0, film=0.25),
    2: dataclasses.replace(WL.DROP_IMPACT_2D, nx=70, ny=48, R=10.0, film=0.25),
}


@pytest.mark.parametrize("D", [3, 2])
def test_windows_reproduce_the_whole_domain_run(D):
    wl = SMALL[D]
    rv, rl, _ = thermo.maxwell(wl.T_over_Tc, **WL.eos(wl))
    rho0, u0 = WL.initial_fields(wl, rv, rl)
    n = (wl.nx, wl.ny, wl.nz)[:D]
    walls = [wl.walls_axis == a for a in range(D)]
    whole = [(0, m, ((1, 1) if w else (0, 0)), slice(0, m)) for m, w in zip(n, walls)]
    p, f0 = oracle_window(wl, rv, rl, rho0, u0, whole)
    ref, _ = O.run(p, f0, K)
    checked = 0
    for s in sample_nodes(wl):
        axes = [window_axis(c, m, w) for c, m, w in zip(s, n, walls)]
        assert all(a[1] < m for a, m in zip(axes, n))  # a true window on every axis
        po, fw = oracle_window(wl, rv, rl, rho0, u0, axes)
        out, _ = O.run(po, fw, K)
        idx = [(lo + np.arange(length))[valid] % m for (lo, length, _, valid), m in zip(axes, n)]
        if D == 2:
            idx.append(np.array([0]))
        sel = (slice(None),) + tuple(a[3] for a in reversed(axes))
        if D == 2:
            sel = (slice(None), slice(None)) + sel[1:]
        got = out[sel]
        want = ref[(slice(None),) + np.ix_(idx[2], idx[1], idx[0])]
        assert np.array_equal(got, want), s
        checked += got[0].size
    assert checked >= len(sample_nodes(wl)) * 4 ** D // 2


def window_matches(wl, rho0, u0, rv, rl, ref, steps, margin):
    """Whether every checked node of every sample window equals the whole run."""
    import windows
    n = (wl.nx, wl.ny, wl.nz)[:wl.D]
    walls = [wl.walls_axis == a for a in range(wl.D)]
    saved = windows.MARGIN
    windows.MARGIN = margin
    try:
        for s in sample_nodes(wl):
            axes = [windows.window_axis(c, m, w) for c, m, w in zip(s, n, walls)]
            po, fw = oracle_window(wl, rv, rl, rho0, u0, axes)
            out, _ = O.run(po, fw, steps)
            idx = [(lo + np.arange(length))[valid] % m for (lo, length, _, valid), m in zip(axes, n)]
            if wl.D == 2:
                idx.append(np.array([0]))
            sel = (slice(None),) + tuple(a[3] for a in reversed(axes))
            if wl.D == 2:
                sel = (slice(None), slice(None)) + sel[1:]
            if not np.array_equal(out[sel], ref[(slice(None),) + np.ix_(idx[2], idx[1], idx[0])]):
                return False
    finally:
        windows.MARGIN = saved
    return True


@pytest.mark.parametrize("D", [3, 2])
def test_the_margin_is_tight_for_one_step(D):
    """After one step the dependency radius is 4 + 2: the force stencil of the
    initial shift (2), the force stencil of the step (2), Phi's q formed with the
    force one node along each axis (1) and streaming (1).  A window with margin 6
    reproduces every checked node, and with two nodes less (the force chain alone)
    some node comes out wrong.  The sixth node is reached only through q: at the
    initial state the fluid velocity u + F/(2 rho) equals the requested velocity up
    to rounding, so that last dependency is at rounding level in the first step."""
    wl = SMALL[D]
    rv, rl, _ = thermo.maxwell(wl.T_over_Tc, **WL.eos(wl))
    rho0, u0 = WL.initial_fields(wl, rv, rl)
    n = (wl.nx, wl.ny, wl.nz)[:D]
    whole = [(0, m, ((1, 1) if wl.walls_axis == a else (0, 0)), slice(0, m)) for a, m in enumerate(n)]
    p, f0 = oracle_window(wl, rv, rl, rho0, u0, whole)
    ref, _ = O.run(p, f0, 1)
    assert window_matches(wl, rho0, u0, rv, rl, ref, 1, 6)
    assert not window_matches(wl, rho0, u0, rv, rl, ref, 1, 4)
