"""Drop-on-film initial state built on the GPU (lbm_init_drop_on_film) against
the same geometry built on the host by the seeded input generator and passed in
through lbm_init_fields; and the statistics of its white noise (Sec. 3.3)."""
import numpy as np
import pytest

from cases import case, lbm_params
from paper_2201_12404_gb300 import inputs as I
from paper_2201_12404_gb300 import lbm

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("D", [2, 3])
def test_gpu_geometry_equals_the_host_generator(D):
    dims = dict(nx=64, ny=48) if D == 2 else dict(nx=32, ny=28, nz=24)
    c = case(D, **dims, Tr=0.7, walls=True)
    shape = (c["nz"], c["ny"], c["nx"])
    R, film, gap, U, W = 8.0, 5.0, 4.0, 0.03, 4.0
    rho, u = I.drop_on_film(shape, D, R, film, U, c["rho_l"], c["rho_v"], W, gap=gap)
    with lbm.Domain(lbm_params(c)) as a, lbm.Domain(lbm_params(c)) as b:
        a.lbm_init_fields(rho, u)
        b.lbm_init_drop_on_film(R, film, gap, U, W)
        fa, fb = a.lbm_read_populations(), b.lbm_read_populations()
        ra, ua = a.lbm_read_macroscopic()
        rb, ub = b.lbm_read_macroscopic()
    assert np.max(np.abs(fa - fb) / np.abs(fa)) < 1e-12
    assert np.allclose(rb, rho, rtol=1e-12) and np.allclose(ub, u, rtol=0, atol=1e-13)


def test_white_noise_has_the_requested_spread_inside_the_drop_only():
    c = case(3, 48, 48, 48, Tr=0.7, walls=True)
    R, film, gap, U, W, noise = 12.0, 6.0, 4.0, 0.04, 4.0, 0.05
    fields = {}
    for seed in (7, 7, 8):
        with lbm.Domain(lbm_params(c)) as dom:
            dom.lbm_init_drop_on_film(R, film, gap, U, W, noise=noise, seed=seed)
            fields.setdefault(seed, []).append(dom.lbm_read_macroscopic()[1])
    u7, u7b, u8 = fields[7][0], fields[7][1], fields[8][0]
    assert np.array_equal(u7, u7b) and not np.array_equal(u7, u8)
    z, y, x = np.meshgrid(np.arange(48.0), np.arange(48.0), np.arange(48.0), indexing="ij")
    d_drop = np.sqrt((x - 23.5) ** 2 + (y - 23.5) ** 2 + (z - (film + R + gap)) ** 2) - R
    core = d_drop < -2 * W          # liquid fraction ~ 1
    far = (d_drop > 4 * W) & (z > film + 3 * W)  # vapour away from the drop and the film
    dev = [u7[0][core], u7[1][core], u7[2][core] + U]
    for comp in dev:
        assert np.std(comp) == pytest.approx(noise * U, rel=0.1)
        assert abs(np.mean(comp)) < 5 * noise * U / np.sqrt(comp.size)
    assert np.max(np.abs(u7[:, far])) < 1e-6
