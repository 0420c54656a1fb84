"""The oracle's pins catch plausible mistakes: each case plants one mistake in a
copy of the oracle's C source (a dropped term, a wrong sign, factor or index, a
transposed operand), builds it into a separate library on the CPU, points the
oracle's wrapper at it and runs the pins named for it; at least one must fail.
The same is done for the Python thermodynamics (the Maxwell construction), whose
mutated copy replaces the module's functions while the pins run.  The oracle
itself is never modified.

One plausible edit is left out because no test can see it: taking the upper
branch of the pseudo-potential sign on a tie (P = rho cs^2 exactly), a set of
densities of measure zero in double precision.
"""
import os
import subprocess

import numpy as np
import pytest

import oracle as O
import test_oracle_pins as pins

PHI = "Phi[al * N + n] = -(1.0 - om / 2.0) * (qp - qm) / 2.0;"

# (name, text in lbm_oracle.c, replacement, [(pin, kwargs), ...])
MUTANTS = [
    ("force sign", "F[al * N + n] = -(2.0 * spsi[n] * g4[al]", "F[al * N + n] = (2.0 * spsi[n] * g4[al]",
     [("test_force_stencils_converge_to_continuum_force", {"D": 2})]),
    ("capillary term dropped", " + p->kappa * rho[n] * g3[al]) + rho[n] * p->g[al];", ") + rho[n] * p->g[al];",
     [("test_force_stencils_converge_to_continuum_force", {"D": 2})]),
    ("body force dropped", ") + rho[n] * p->g[al];", ");", [("test_poiseuille_between_bounce_back_walls", {})]),
    ("psi stencil coefficient", "(4.0 / 3.0 * psi1 - 1.0 / 6.0 * psi2)", "(4.0 / 3.0 * psi1 + 1.0 / 6.0 * psi2)",
     [("test_force_stencils_converge_to_continuum_force", {"D": 2})]),
    ("rho stencil second neighbour", "(2.0 * rho[n1] - rho[n2])", "(2.0 * rho[n1] - rho[n1])",
     [("test_force_stencils_converge_to_continuum_force", {"D": 2})]),
    ("stencil weight without 1/cs2", "g4[al] += (w[i] / CS2) * c[3 * i + al]", "g4[al] += w[i] * c[3 * i + al]",
     [("test_force_stencils_converge_to_continuum_force", {"D": 2})]),
    ("sign s dropped in the step", "double ps = orc_psi(p, r, &sg);\n    spsi[n] = sg * ps;",
     "double ps = orc_psi(p, r, &sg);\n    spsi[n] = ps;",
     [("test_mass_and_momentum_conserved_periodic", {"D": 2, "n": 32, "steps": 60})]),
    ("zeta* unshifted", "zeta[al] = CS2 + xi[al] * xi[al] + Phi[al] / rho;", "zeta[al] = CS2 + u[al] * u[al] + Phi[al] / rho;",
     [("test_fstar_central_moments_match_appendix", {"D": 2})]),
    ("xi* force not over rho", "xi[al] = u[al] + F[al] / rho;", "xi[al] = u[al] + F[al];",
     [("test_fstar_central_moments_match_appendix", {"D": 2})]),
    ("Phi dropped from zeta*", "xi[al] * xi[al] + Phi[al] / rho;", "xi[al] * xi[al];",
     [("test_fstar_central_moments_match_appendix", {"D": 2})]),
    ("Phi with the printed sign", PHI, "Phi[al * N + n] = (1.0 - om / 2.0) * (qp - qm) / 2.0;",
     [("test_diagonal_correction_makes_sound_damping_galilean_invariant", {"D": 2})]),
    ("Phi without (1 - omega/2)", PHI, "Phi[al * N + n] = -(qp - qm) / 2.0;", [("test_phi_central_difference", {})]),
    ("Phi dropped", PHI, "Phi[al * N + n] = 0.0;",
     [("test_diagonal_correction_makes_sound_damping_galilean_invariant", {"D": 2})]),
    ("q not negated across a wall", "double qp = q[al * N + np_] * (flp ? -1.0 : 1.0);", "double qp = q[al * N + np_];",
     [("test_walls_equal_the_mirrored_periodic_domain", {"D": 2})]),
    ("q from the bare velocity", "double v = u[al * N + n] + F[al * N + n] / (2.0 * rho[n]);", "double v = u[al * N + n];",
     [("test_phi_vanishes_for_a_fluid_at_rest", {"D": 2})]),
    ("q with the whole force", "double v = u[al * N + n] + F[al * N + n] / (2.0 * rho[n]);",
     "double v = u[al * N + n] + F[al * N + n] / rho[n];", [("test_phi_vanishes_for_a_fluid_at_rest", {"D": 2})]),
    ("q = rho u^2", "q[al * N + n] = rho[n] * v * (v * v + 3.0 * CS2 - 3.0 * CS2);", "q[al * N + n] = rho[n] * v * v;",
     [("test_diagonal_correction_makes_sound_damping_galilean_invariant", {"D": 2})]),
    ("equilibrium zeta without u^2", "zeta[al] = CS2 + u[al] * u[al]; }", "zeta[al] = CS2; }",
     [("test_feq_central_moments_vanish", {"D": 2})]),
    ("triplet c = +1 sign", "if (c == 1) return (xi + zeta) / 2.0;", "if (c == 1) return (-xi + zeta) / 2.0;",
     [("test_feq_central_moments_vanish", {"D": 2})]),
    ("gamma ratio sign", "gamma = 2.0 * (1.0 / omega - (1.0 - 1.0 / omega) * ratio);",
     "gamma = 2.0 * (1.0 / omega + (1.0 - 1.0 / omega) * ratio);",
     [("test_gamma_is_first_order_entropy_minimiser", {"D": 2})]),
    ("entropic weight 1/f^eq", "ds_dh += ds * dh / fs[i];", "ds_dh += ds * dh / feq[i];",
     [("test_gamma_is_first_order_entropy_minimiser", {"D": 2})]),
    ("mirror state uses s for h", "(1.0 - gamma) * h[i]", "(1.0 - gamma) * s[i]",
     [("test_gamma_two_is_textbook_edm_lbgk", {"D": 2})]),
    ("relaxation without the mirror half",
     "fp[i] = (1.0 - omega / 2.0) * f[i] + (omega / 2.0) * mirr + (fs[i] - feq[i]);",
     "fp[i] = (1.0 - omega) * f[i] + omega * mirr + (fs[i] - feq[i]);",
     [("test_gamma_two_is_textbook_edm_lbgk", {"D": 2})]),
    ("force increment dropped", "(omega / 2.0) * mirr + (fs[i] - feq[i]);", "(omega / 2.0) * mirr;",
     [("test_equilibrium_node_gets_fstar_increment_only", {})]),
    ("omega with dt instead of dt/2", "return 1.0 / (nu / CS2 + 0.5);", "return 1.0 / (nu / CS2 + 1.0);",
     [("test_omega_of_nu", {})]),
    ("viscosity interpolation reversed", "double nu = p->nu_vapour + phi * (p->nu_liquid - p->nu_vapour);",
     "double nu = p->nu_liquid + phi * (p->nu_vapour - p->nu_liquid);", [("test_omega_of_nu", {})]),
    ("EOS attraction sign", "- p->a * alpha * rho * rho / (1.0 + 2.0 * rho * b - b * b * rho * rho)",
     "+ p->a * alpha * rho * rho / (1.0 + 2.0 * rho * b - b * b * rho * rho)", [("test_oracle_pressure_matches_thermo", {})]),
    ("alpha without the square root", "double sq = 1.0 + m * (1.0 - sqrt(p->T_over_Tc));",
     "double sq = 1.0 + m * (1.0 - p->T_over_Tc);", [("test_oracle_pressure_matches_thermo", {})]),
    ("Tc without R", "return 0.0778 * p->a / (0.45724 * p->b * p->R);", "return 0.0778 * p->a / (0.45724 * p->b);",
     [("test_oracle_pressure_matches_thermo", {})]),
    ("H2 without cs^2", "return x * x - CS2;", "return x * x;", [("test_feq_central_moments_vanish", {"D": 2})]),
    ("shear moment put in H", "ROW(0, 1, 1, 0, 1); ROW(1, 0, 0, 0, 1); ROW(3, 0, 0, 0, 2);",
     "ROW(0, 1, 1, 0, 2); ROW(1, 0, 0, 0, 1); ROW(3, 0, 0, 0, 2);", [("test_shear_wave_decay_rate_matches_nu", {})]),
    ("trace put in S", "ROW(1, 0, 0, 0, 1); ROW(3, 0, 0, 0, 2);\n    ROW(0, 2, 1, 0, 2)",
     "ROW(1, 0, 0, 0, 1); ROW(3, 0, 0, 0, 1);\n    ROW(0, 2, 1, 0, 2)", [("test_kbc_split_structure", {"D": 2})]),
    ("raw instead of central moments", "v[al] = (al < D) ? (double)c[3 * i + al] - u[al] : 0.0;",
     "v[al] = (al < D) ? (double)c[3 * i + al] : 0.0;", [("test_feq_central_moments_vanish", {"D": 2})]),
    ("bounce-back not reversed", "if (wall) f_out[(Q - 1 - i) * N + n] = fp[i];", "if (wall) f_out[i * N + n] = fp[i];",
     [("test_walls_equal_the_mirrored_periodic_domain", {"D": 2})]),
    ("streaming backwards", "int t[3] = {x + c[3 * i], y + c[3 * i + 1], z + c[3 * i + 2]};",
     "int t[3] = {x - c[3 * i], y - c[3 * i + 1], z - c[3 * i + 2]};",
     [("test_mass_and_momentum_conserved_periodic", {"D": 2, "n": 32, "steps": 60})]),
    ("low wall streams periodically", "if (t[al] < 0) { if (p->bc[2 * al] == 1) wall = 1; else t[al] += n_ax[al]; }",
     "if (t[al] < 0) { t[al] += n_ax[al]; }", [("test_walls_equal_the_mirrored_periodic_domain", {"D": 2})]),
    ("initial shift sign", "ub[al * N + n] = u0[al * N + n] - F[al * N + n] / (2.0 * rho0[n]);",
     "ub[al * N + n] = u0[al * N + n] + F[al * N + n] / (2.0 * rho0[n]);",
     [("test_physical_initial_state_reports_the_requested_velocity", {"D": 2})]),
    ("reported velocity without the half force",
     "u_phys[al * N + n] = ub[al * N + n] + F[al * N + n] / (2.0 * rho[n]);", "u_phys[al * N + n] = ub[al * N + n];",
     [("test_physical_initial_state_reports_the_requested_velocity", {"D": 2})]),
    ("velocity index transposed", "c[3 * i + 0] = i % 3 - 1;\n    c[3 * i + 1] = (i / 3) % 3 - 1;",
     "c[3 * i + 1] = i % 3 - 1;\n    c[3 * i + 0] = (i / 3) % 3 - 1;", [("test_velocity_index_and_opposites", {})]),
]


@pytest.mark.parametrize("name,old,new,catchers", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_a_planted_mistake(name, old, new, catchers, tmp_path):
    src = open(O._SRC).read()
    assert src.count(old) == 1, f"the text to mutate must occur once in the oracle: {old!r}"
    c_file = tmp_path / "lbm_oracle_mutant.c"
    c_file.write_text(src.replace(old, new))
    so = tmp_path / "liblbm_oracle_mutant.so"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-o", str(so),
                           str(c_file), "-lm"])
    saved = O.lib()
    O._lib = O.load_library(str(so))
    failed = []
    try:
        for pin, kwargs in catchers:
            try:
                with np.errstate(all="ignore"):
                    getattr(pins, pin)(**kwargs)
            except (AssertionError, RuntimeError, FloatingPointError, ValueError) as e:
                failed.append((pin, type(e).__name__))
    finally:
        O._lib = saved
    assert failed, f"no pin caught the planted mistake '{name}'"


# Mistakes planted in a copy of the oracle's Python thermodynamics (the Maxwell
# construction and the Peng-Robinson helpers), loaded in place of the module's
# functions for the duration of the catchers.
PY_MUTANTS = [
    ("equal-area integral log argument inverted", "math.log((v + b - s2 * b) / (v + b + s2 * b))",
     "math.log((v + b + s2 * b) / (v + b - s2 * b))", [("test_maxwell_equal_area_by_quadrature", {})]),
    ("volume cubic coefficient", "c2 = P * (2 * b - b) - R * T", "c2 = P * (2 * b) - R * T",
     [("test_maxwell_equal_area_by_quadrature", {})]),
    ("alpha without the square root (python)", "(1.0 - math.sqrt(T_over_Tc))", "(1.0 - T_over_Tc)",
     [("test_oracle_pressure_matches_thermo", {})]),
    ("coexistence densities swapped", "return 1.0 / r[-1], 1.0 / r[0], Psat", "return 1.0 / r[0], 1.0 / r[-1], Psat",
     [("test_density_ratio_at_Tr_059_is_about_1e3", {})]),
    ("critical pressure constant", "return 0.0778 * R * critical_temperature(a, b, R) / b",
     "return 0.0788 * R * critical_temperature(a, b, R) / b", [("test_pr_critical_point", {})]),
]


@pytest.mark.parametrize("name,old,new,catchers", PY_MUTANTS, ids=[m[0] for m in PY_MUTANTS])
def test_pins_catch_a_planted_thermodynamics_mistake(name, old, new, catchers, monkeypatch):
    from oracle import thermo
    src = open(thermo.__file__).read()
    assert src.count(old) == 1, f"the text to mutate must occur once in thermo.py: {old!r}"
    ns = {"__name__": "thermo_mutant"}
    exec(compile(src.replace(old, new), "thermo_mutant", "exec"), ns)
    for attr in ("alpha_of", "critical_temperature", "critical_pressure", "pressure", "maxwell"):
        monkeypatch.setattr(thermo, attr, ns[attr])
    failed = []
    for pin, kwargs in catchers:
        try:
            with np.errstate(all="ignore"):
                getattr(pins, pin)(**kwargs)
        except (AssertionError, RuntimeError, FloatingPointError, ValueError, ZeroDivisionError) as e:
            failed.append((pin, type(e).__name__))
    assert failed, f"no pin caught the planted mistake '{name}'"


def test_the_unmutated_oracle_passes_every_catcher():
    """The catchers fail because of the planted mistake, not by themselves."""
    seen = set()
    for _, _, _, catchers in MUTANTS + PY_MUTANTS:
        for pin, kwargs in catchers:
            key = (pin, tuple(sorted(kwargs.items())))
            if key in seen:
                continue
            seen.add(key)
            getattr(pins, pin)(**kwargs)
