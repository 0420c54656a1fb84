"""The benchmark workloads' labels carry the Weber and Reynolds numbers their
parameters give (Secs. 3.2-3.3: We = 2 rho_l R U^2 / sigma, Re = 2 U R / nu_l), with
the surface tension the Laplace-law sweep measured at T/Tc = 0.59."""
import re

import pytest

from oracle import thermo
from paper_2201_12404_gb300 import workloads as WL


@pytest.mark.parametrize("name", ["drop3d", "drop2d", "drop3d-small"])
def test_labels_state_the_achieved_we_and_re(name):
    wl = WL.by_name(name)
    rv, rl, _ = thermo.maxwell(wl.T_over_Tc, **WL.eos(wl))
    We = 2 * rl * wl.R * wl.U ** 2 / WL.SIGMA_T059
    Re = 2 * wl.U * wl.R / wl.nu_liquid
    we_label = float(re.search(r"We [~=] ([0-9.]+)", wl.name).group(1))
    re_label = float(re.search(r"Re [~=] ([0-9.]+)", wl.name).group(1))
    assert abs(We / we_label - 1) < 0.1, (We, wl.name)
    assert abs(Re / re_label - 1) < 0.05, (Re, wl.name)
