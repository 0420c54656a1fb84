"""The seeded input generators: the geometry and the interface width of the
paper's workloads, checked without a GPU."""
import numpy as np

from paper_2201_12404_gb300 import inputs as I

RL, RV = 8.8, 0.0083


def test_tanh_width_is_the_papers_interface_thickness():
    """Sec. 3.1.1 defines W = (rho_l - rho_v) / max |grad rho|; the profile
    (rho_l + rho_v)/2 - (rho_l - rho_v)/2 tanh(2 d / W) has exactly that width."""
    W = 5.0
    d = np.linspace(-40, 40, 80001)
    rho = I.tanh_profile(d, RL, RV, W)
    assert abs((RL - RV) / np.max(np.abs(np.gradient(rho, d))) - W) < 1e-6
    assert abs(rho[0] - RL) < 1e-6 * RL and abs(rho[-1] - RV) < 1e-6 * RL


def test_drop_on_film_geometry():
    """Secs. 3.2-3.3: film of thickness h on the low wall (the wall half a node below
    the first node), drop of radius R centred h + R + gap above, horizontally centred,
    moving down at U inside the drop only."""
    nz, ny, nx = 96, 64, 64
    R, h, U, W = 14.0, 6.0, 0.05, 4.0
    rho, u = I.drop_on_film((nz, ny, nx), 3, R, h, U, RL, RV, W)
    cz = h + R + 2 * W
    cx, cy = 0.5 * (nx - 1), 0.5 * (ny - 1)
    mid = (RL + RV) / 2
    # film surface at z = h - 1/2, drop surface at cz +- R: the mid density crosses there
    col = rho[:, 0, 0]                      # far from the drop: the film alone
    zs = np.arange(nz)
    cross = zs[:-1][(col[:-1] - mid) * (col[1:] - mid) < 0]
    assert len(cross) == 1 and abs(cross[0] + 0.5 - (h - 0.5)) <= 1.0
    axis = rho[:, int(cy), int(cx)]
    inside = np.where(axis > mid)[0]
    top = inside[inside > h + 2].max()
    assert abs(top - (cz + R)) <= 1.5
    assert u.shape == (3, nz, ny, nx)
    assert abs(u[2, int(round(cz)), int(cy), int(cx)] + U) < 1e-5 * U   # drop centre moves down at U (fraction 1 - 2e-6)
    assert np.all(u[:2] == 0) and abs(u[2, 2, 0, 0]) < 1e-6 * U            # film at rest


def test_seeded_generators_repeat_and_differ_by_seed():
    a = I.uniform_noise((4, 5, 6), 1e-6, 7)
    assert np.array_equal(a, I.uniform_noise((4, 5, 6), 1e-6, 7))
    assert not np.array_equal(a, I.uniform_noise((4, 5, 6), 1e-6, 8))
    assert np.max(np.abs(a)) <= 1e-6
    base = np.ones((9, 1, 4, 4))
    p = I.perturbed_populations(base, 0.01, 3)
    assert np.max(np.abs(p - 1)) <= 0.01 and np.array_equal(p, I.perturbed_populations(base, 0.01, 3))
