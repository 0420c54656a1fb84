"""Host logic of the SRT-versus-entropic studies (no GPU): job lists, operator
parameters and the power-law fit."""
import pytest

from paper_2201_12404_gb300 import lbm
from paper_2201_12404_gb300 import studies as S


def test_spurious_sweeps_pair_every_value_with_both_operators():
    for kind, vals in (("T", (0.5, 0.7, 0.9)), ("nu", (0.001, 0.1)), ("a", (0.003, 0.0011))):
        jobs = S.spurious_jobs(kind, vals)
        assert len(jobs) == 2 * len(vals)
        for v in vals:
            ops = sorted(j.operator for j in jobs if j.tags["value"] == v)
            assert ops == ["entropic", "srt"]
    j = S.spurious_jobs("a", (0.0011,))[0]
    assert j.a == 0.0011 and j.wl.T_over_Tc == 0.59 and j.wl.nu_liquid == 0.1
    j = S.spurious_jobs("T", (0.8,))[0]
    assert j.wl.T_over_Tc == 0.8 and j.wl.U == 0 and j.wl.walls_axis == -1


def test_srt_is_gamma_pinned_to_two_and_entropic_is_not():
    srt, ent = S.spurious_jobs("T", (0.8,))
    assert srt.operator == "srt"
    p = srt.params(0.2, 7.2)
    assert p.gamma_mode == lbm.LBM_GAMMA_FIXED and p.gamma_value == 2.0
    assert ent.params(0.2, 7.2).gamma_mode == lbm.LBM_GAMMA_ENTROPIC


def test_stability_jobs_follow_the_paper_setup():
    jobs = S.stability_jobs((0.005, 0.04), (0.0, 0.16), R0=50.0)
    assert len(jobs) == 8
    wl = jobs[0].wl
    assert (wl.nx, wl.ny) == (1200, 600) and wl.R == 50.0 and wl.W == 5.0 and wl.walls_axis == 1
    assert wl.film * wl.R == 50.0  # film thickness R0
    p = jobs[0].params(0.0083, 8.78)
    assert p.nu_vapour == pytest.approx(15 * p.nu_liquid)
    assert p.bc[2] == lbm.LBM_BC_BOUNCEBACK and p.bc[3] == lbm.LBM_BC_BOUNCEBACK and p.bc[0] == lbm.LBM_BC_PERIODIC


def test_power_fit_recovers_exponent_and_prefactor():
    xs = [0.05, 0.1, 0.2, 0.41]
    m, c = S.fit_power(xs, [3e-4 * x ** 2.2 for x in xs])
    assert m == pytest.approx(2.2, abs=1e-12) and c == pytest.approx(3e-4, rel=1e-12)


def test_laplace_measure_on_a_sharp_disc_and_the_pressure_law():
    """A step disc of radius 20 (densities 8 and 0.5) gives back its radius and bulk
    densities; the pressure is the Peng-Robinson law (ideal-gas limit at low density)."""
    import numpy as np
    n = 100
    yy, xx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    rho = np.where(np.hypot(xx - n / 2, yy - n / 2) < 20.0, 8.0, 0.5)
    r_in, r_out, Re, W = S.laplace_measure(rho, 20.0)
    assert r_in == 8.0 and r_out == 0.5 and Re == pytest.approx(20.0, rel=0.01)
    # a step of 7.5: central differences of 3.75 in both directions where the step
    # runs diagonally, max |grad rho| = 3.75 sqrt 2, W = sqrt 2
    assert W == pytest.approx(2 ** 0.5)
    T = 0.8
    Tc = 0.0778 * 0.003 / (0.45724 * 0.095)
    assert S.pr_pressure(1e-9, T) == pytest.approx(1e-9 * T * Tc, rel=1e-6)


def test_surface_tension_jobs_cover_every_temperature_and_radius():
    jobs = S.surface_tension_jobs((0.6, 0.9), (30.0, 45.0, 60.0), radii_near_tc=(60.0, 90.0, 120.0))
    assert len(jobs) == 6 and all(j.operator == "entropic" for j in jobs)
    assert {(j.tags["T"], j.tags["R"]) for j in jobs} == {(0.6, r) for r in (30.0, 45.0, 60.0)} | {
        (0.9, r) for r in (60.0, 90.0, 120.0)}
    assert jobs[0].wl.nx == 120 and jobs[-1].wl.nx == 480
    small_a = S.surface_tension_jobs((0.6,), (30.0,), a=0.0011)
    assert small_a[0].a == 0.0011 and small_a[0].tags["a"] == 0.0011 and small_a[0].eos()["a"] == 0.0011


def test_sigma_rows_fit_the_laplace_law_per_a(monkeypatch):
    """Stable drops whose pressure jump is exactly sigma/R_e give back sigma as the
    slope of Delta P against 1/R_e, for the drops of the requested a only."""
    sig = {0.6: 0.1, 0.7: 0.05}
    jobs = [dict(tags={"a": a, "T": T, "R": R}, stable=True, rho=R, final_max_u=0.0, steps_run=1)
            for a in (0.0017, 0.003) for T in sig for R in (30.0, 45.0, 60.0)]
    # the inside density carries the radius; the pressure of it is sigma/R, outside 0
    monkeypatch.setattr(S, "laplace_measure", lambda rho, R: (rho, 0.0, R, 5.0))
    monkeypatch.setattr(S, "pr_pressure", lambda r, T, a=None: sig[T] / r if r > 0 else 0.0)
    rows, fits = S._sigma_rows(jobs, (0.6, 0.7), 0.0017)
    assert [r["a"] for r in rows] == [0.0017, 0.0017]
    assert [len(r["drops"]) for r in rows] == [3, 3]
    for r in rows:
        assert abs(r["sigma"] - sig[r["T_over_Tc"]]) < 1e-12
    # sigma halves from 1 - T = 0.4 to 0.3: m = ln 2 / ln(4/3)
    import math
    assert abs(fits["m_below_0.8"] - math.log(2) / math.log(4 / 3)) < 1e-9


def test_paper_2d_impacts_reproduce_the_stated_we_and_re():
    """Sec. 3.2: We = 2 rho_l R0 U0^2 / sigma and Re = 2 U0 R0 / nu_l recomputed from the
    workloads give the paper's pairs; the box is 24 R0 x 12 R0 with a film of R0 and
    nu_v = 15 nu_l."""
    from paper_2201_12404_gb300 import lbm
    from paper_2201_12404_gb300 import workloads as WL
    rv, rl, _ = lbm.lbm_coexistence(lbm.lbm_default_params(T_over_Tc=0.59, **WL.PAPER_EOS))
    wls = S.paper_2d_impacts()
    assert [(w.extra["We"], w.extra["Re"]) for w in wls] == list(S.PAPER_2D_CASES)
    for w in wls:
        assert (w.nx, w.ny, w.R, w.film * w.R) == (2400, 1200, 100.0, 100.0)
        assert abs(2 * rl * w.R * w.U ** 2 / S.SIGMA_T059 - w.extra["We"]) < 1e-9 * w.extra["We"]
        assert abs(2 * w.U * w.R / w.nu_liquid - w.extra["Re"]) < 1e-9 * w.extra["Re"]
        nu_l, nu_v = WL.viscosities(w, rv, rl)
        assert nu_v == 15 * nu_l


def test_paper_3d_impacts_reproduce_the_stated_we_and_re_range():
    """Sec. 3.3: We 82, 167 and 328 in a 14 R0 x 14 R0 x 6 R0 box with R0 = 80 and
    h/2R0 = 0.22, one fluid for all three, so that Re grows as sqrt(We) and spans the
    stated 3500-6900 (to the rounding of the paper's figures); nu_v = 15 nu_l."""
    import math
    from paper_2201_12404_gb300 import lbm
    from paper_2201_12404_gb300 import workloads as WL
    rv, rl, _ = lbm.lbm_coexistence(lbm.lbm_default_params(T_over_Tc=0.59, **WL.PAPER_EOS))
    wls = S.paper_3d_impacts()
    assert [w.extra["We"] for w in wls] == [82, 167, 328]
    for w in wls:
        assert (w.nx, w.ny, w.nz, w.R, w.walls_axis) == (1120, 1120, 480, 80.0, 2)
        assert abs(w.film * w.R / (2 * w.R) - 0.22) < 1e-12 and w.noise == 0.05
        assert abs(2 * rl * w.R * w.U ** 2 / S.SIGMA_T059 - w.extra["We"]) < 1e-9 * w.extra["We"]
        assert abs(2 * w.U * w.R / w.nu_liquid - w.extra["Re"]) < 1e-9 * w.extra["Re"]
        assert w.nu_liquid == wls[0].nu_liquid
        nu_l, nu_v = WL.viscosities(w, rv, rl)
        assert nu_v == 15 * nu_l
    res = [w.extra["Re"] for w in wls]
    assert abs(res[0] - 3500) < 1e-6 and 6800 < res[-1] < 7100
    assert abs(res[-1] / res[0] - math.sqrt(328 / 82)) < 1e-9


def test_surface_tension_study_scales_radii_and_steps_with_a(monkeypatch):
    """Without a GPU: the study asks for drops whose radii grow as sqrt(a0/a) (the
    interface width at fixed kappa) and run a0/a times longer, for each a."""
    calls = []

    def fake_run(jobs, steps, chunk=500, keep_density=False, **kw):
        calls.append((jobs, steps))
        return dict(jobs=[dict(tags=j.tags, stable=False) for j in jobs], batched_mlups=1.0)

    monkeypatch.setattr(S, "run_jobs", fake_run)
    S.surface_tension_study(a_values=(0.003, 0.00075))
    by_a = {}
    for jobs, steps in calls:
        a = jobs[0].a
        by_a.setdefault(a, []).append((sorted({j.tags["R"] for j in jobs}), steps))
    assert set(by_a) == {0.003, 0.00075}
    for (r0, s0), (r1, s1) in zip(by_a[0.003], by_a[0.00075]):
        assert r1 == [2 * r for r in r0]          # sqrt(0.003 / 0.00075) = 2
        assert s1 == 4 * s0                        # 0.003 / 0.00075 = 4
    assert all(j.eos()["a"] == j.a for jobs, _ in calls for j in jobs)


def test_crown_fits_recover_the_exponent_of_each_window():
    """A radius growing as 3 sqrt(t - tc) early and as (t - tc)^0.9 later is fitted
    window by window; windows with fewer than three samples are skipped."""
    tau, tc = 1000.0, 40.0
    t = [tc + k * 5.0 for k in range(1, 401)]
    r = [3 * (x - tc) ** 0.5 if x - tc <= 100 else 3 * 100 ** 0.5 * ((x - tc) / 100) ** 0.9 for x in t]
    fits = S.crown_fits(t, r, tc, tau, ((0.01, 0.1), (0.2, 1.0), (3.0, 4.0)))
    assert [f["window_tau"] for f in fits] == [[0.01, 0.1], [0.2, 1.0]]
    assert abs(fits[0]["p"] - 0.5) < 1e-9 and abs(fits[0]["c"] - 3.0) < 1e-9
    assert abs(fits[1]["p"] - 0.9) < 1e-9


def test_crown_study_reports_contact_and_failure_of_a_run_that_diverges(monkeypatch):
    """Without a GPU (a fake domain): a run whose crown forms and that then diverges
    reports the step it reached and the contact step of its crown."""
    import dataclasses
    from paper_2201_12404_gb300 import workloads as WL

    class FakeDomain:
        def __init__(self, p):
            self.steps = 0

        def __enter__(self):
            return self

        def __exit__(self, *exc):
            return False

        def lbm_init_drop_on_film(self, *a, **k):
            pass

        def lbm_record_gamma(self, on):
            pass

        def lbm_step(self, n):
            if self.steps + n > 60:
                raise lbm.LBMError(lbm.LBM_ERR_UNSTABLE, "non-finite density")
            self.steps += n

        def lbm_crown_radius(self, layer):
            return 0.0 if self.steps < 30 else float(self.steps)

    monkeypatch.setattr(S.lbm, "Domain", FakeDomain)
    wl = dataclasses.replace(WL.DROP_IMPACT_2D, R=10.0, U=0.1)  # tau = 200 steps
    res = S.crown_study(wl=wl, t_end_tau=1.0, samples=20)      # samples every 10 steps
    assert res["failed"]["after_step"] == 60 and res["t_contact"] == 30
    assert res["t"] == [10, 20, 30, 40, 50, 60]
