"""Windows of a large domain that the oracle can step exactly.

One node after K steps from lbm_init_fields depends only on the initial fields
within a radius of 4K + 2: the force reaches two nodes (Sec. 2, the stencils of
the pseudo-potential and of the Korteweg term), Phi one more (its q is formed
with the force of the neighbouring nodes), streaming one more per step, and the
initial velocity shift F/(2 rho) two.  A window with that margin around the
nodes it checks therefore gives those nodes exactly, whatever the window's own
faces do.  Windows wrap across periodic faces; along a wall axis they are clipped
to the domain and a face that is not a true wall gets a bounce-back wall.
"""
import numpy as np

import oracle as O
from paper_2201_12404_gb300 import inputs as I
from paper_2201_12404_gb300 import workloads as WL

K = 4                    # steps: even, odd, even, odd A-A parities
MARGIN = 4 * K + 2       # dependency radius of a node after K steps from lbm_init_fields
VALID = 4                # checked nodes per axis in a periodic window


def sample_nodes(wl, seed=20220128):
    """Nodes where the workload is most varied: the drop's interface (top, bottom
    and side), its centre, the film surface, the corners where the walls meet the
    periodic seams, the seams themselves, and a few seeded random nodes."""
    D = wl.D
    n = (wl.nx, wl.ny, wl.nz)[:D]
    h = wl.film * wl.R
    centre = [0.5 * (m - 1) for m in n[:-1]] + [h + wl.R + 2.0 * wl.W]
    def node(*c):
        return tuple(int(round(v)) % m for v, m in zip(c, n))
    up = lambda d: [0] * (D - 1) + [d]
    side = [wl.R] + [0] * (D - 1)
    out = [
        node(*(np.add(centre, up(wl.R)))), node(*(np.add(centre, up(-wl.R)))),
        node(*(np.add(centre, side))), node(*centre),
        node(*([m / 5 for m in n[:-1]] + [h])),
        node(*([0] * D)), node(*[m - 1 for m in n]),
        node(*([n[0] - 1] + [m / 5 for m in n[1:-1]] + [2])),
        node(*([n[0] / 3] + [0] * (D - 2) + [n[-1] / 2])),
    ]
    rng = I.rng(seed)
    for _ in range(4):
        out.append(tuple(int(rng.integers(0, m)) for m in n))
    return out


def window_axis(c, n, wall):
    """(origin, length, oracle bc pair, valid slice) of one axis of a window around c."""
    length = 2 * MARGIN + VALID
    if length >= n:
        return 0, n, ((1, 1) if wall else (0, 0)), slice(0, n)
    lo = c - VALID // 2 - MARGIN
    if not wall:
        return lo % n, length, (0, 0), slice(MARGIN, MARGIN + VALID)
    lo = min(max(lo, 0), n - length)
    first = 0 if lo == 0 else MARGIN
    last = length if lo + length == n else length - MARGIN
    return lo, length, (1, 1), slice(first, last)


def oracle_window(wl, rv, rl, rho0, u0, axes):
    """K oracle steps on the window of the initial fields given by axes (x, y[, z])."""
    nu_l, nu_v = WL.viscosities(wl, rv, rl)
    idx = [(lo + np.arange(length)) % n for (lo, length, _, _), n in zip(axes, (wl.nx, wl.ny, wl.nz))]
    if wl.D == 2:
        idx.append(np.array([0]))
    ix, iy, iz = idx
    rho = rho0[np.ix_(iz, iy, ix)]
    u = u0[(slice(None),) + np.ix_(iz, iy, ix)]
    bc = [0] * 6
    for a, (_, _, pair, _) in enumerate(axes):
        bc[2 * a], bc[2 * a + 1] = pair
    p = O.make_params(wl.D, len(ix), len(iy), len(iz), T_over_Tc=wl.T_over_Tc, kappa=wl.kappa, nu_liquid=nu_l,
                      nu_vapour=nu_v, rho_liquid=rl, rho_vapour=rv, bc=tuple(bc), **WL.eos(wl))
    return p, O.init_physical(p, rho, u)
