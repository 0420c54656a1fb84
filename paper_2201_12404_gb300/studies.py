"""Single-relaxation-time versus entropic collision on the paper's 2-D studies.

The SRT operator is the LBGK limit of the same kernels, gamma pinned to 2
(lbm_params.gamma_mode = LBM_GAMMA_FIXED, gamma_value = 2); the entropic operator
computes gamma per node (Sec. 2.4).  Every study is a set of D2Q9 jobs advanced
together by persistent batched launches (lbm_batch_*), a chunk of steps at a time;
after each chunk every job's largest speed of the reported velocity u + F/(2 rho)
is read (lbm_max_speed, a GPU reduction), and a job whose density turns
non-finite or non-positive, or whose speed passes a limit, is recorded as
unstable at that chunk and leaves the batch.

  spurious currents (Sec. 3.1.2): static drops, max|u| after the run, swept over
    T/Tc at nu = 0.1, over nu at T/Tc = 0.59 and over the EOS constant a at
    T/Tc = 0.59, with the (1 - T/Tc)^m fit of the temperature sweep;
  stability domain (Sec. 3.2): drop impact on a film of thickness R0 (R0 = 50,
    W = 5, nu_v = 15 nu_l, walls at the bottom and top) over a grid of liquid
    viscosities and impact speeds;
  surface tension (Sec. 3.1.2, Eq. Laplace_equimolar): static drops of three radii
    per temperature (entropic operator), sigma from the pressure jump against the
    equimolar radius, and the exponents of sigma ~ (1 - T/Tc)^m above and below
    T/Tc = 0.8 (the paper: 3/2 and 11/9).

  python -m paper_2201_12404_gb300.studies spurious [--quick]
  python -m paper_2201_12404_gb300.studies stability [--quick]
  python -m paper_2201_12404_gb300.studies surface-tension [--quick]

and, for the entropic operator alone, the crown radius of the 2-D drop impact
(Sec. 3.2) sampled on the GPU (lbm_crown_radius, the layer just above the film)
with the fit r ~ (t - t0)^p over the first convective time after contact (the
paper: p = 1/2), and the 2/(omega gamma) field of its last step (Sec. 3.3):

  python -m paper_2201_12404_gb300.studies crown [--quick]
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import time
from dataclasses import dataclass

import numpy as np

from . import inputs as I
from . import lbm
from . import workloads as WL

OPERATORS = ("srt", "entropic")


@dataclass
class StudyJob:
    """One D2Q9 job of a study: a workload, the EOS constant a and the operator."""
    name: str
    wl: WL.Workload
    operator: str                  # "srt" (gamma = 2) or "entropic"
    a: float = WL.PAPER_EOS["a"]
    nu_vapour_ratio: float = 1.0   # nu_v / nu_l
    precision: int = lbm.LBM_FP32
    tags: dict = dataclasses.field(default_factory=dict)

    def eos(self):
        return dict(WL.PAPER_EOS, a=self.a)

    def coexistence(self):
        rv, rl, _ = lbm.lbm_coexistence(lbm.lbm_default_params(T_over_Tc=self.wl.T_over_Tc, **self.eos()))
        return rv, rl

    def params(self, rv, rl):
        wl = self.wl
        bc = [0] * 6
        if wl.walls_axis >= 0:
            bc[2 * wl.walls_axis] = bc[2 * wl.walls_axis + 1] = 1
        p = lbm.lbm_default_params(
            lattice=lbm.LBM_D2Q9, precision=self.precision, nx=wl.nx, ny=wl.ny, nz=1,
            T_over_Tc=wl.T_over_Tc, kappa=wl.kappa, nu_liquid=wl.nu_liquid,
            nu_vapour=wl.nu_liquid * self.nu_vapour_ratio, rho_liquid=rl, rho_vapour=rv, bc=bc,
            **self.eos())
        if self.operator == "srt":
            p.gamma_mode = lbm.LBM_GAMMA_FIXED
            p.gamma_value = 2.0
        return p


# ---------------------------------------------------------------------------
# Job lists (host logic only)
# ---------------------------------------------------------------------------

def static_drop(T, nu, R=40.0, side=None, kappa=0.01, W=5.0):
    side = side or int(4 * R)
    return WL.Workload(name=f"static drop {side}x{side} R={R:g} T/Tc={T:g} nu={nu:g}", D=2, nx=side, ny=side,
                       nz=1, T_over_Tc=T, kappa=kappa, nu_liquid=nu, mu_ratio=0.0, R=R, U=0.0, film=0.0, W=W)


def spurious_jobs(kind, values, R=40.0, kappa=0.01, nu=0.1, T=0.59, a=WL.PAPER_EOS["a"]):
    """Static-drop jobs for one sweep, both operators per value.  kind: "T" (T/Tc,
    at nu), "nu" (at T) or "a" (the EOS constant, at T and nu)."""
    jobs = []
    for v in values:
        Tv, nuv, av = (v, nu, a) if kind == "T" else ((T, v, a) if kind == "nu" else (T, nu, v))
        for op in OPERATORS:
            jobs.append(StudyJob(name=f"{kind}={v:g} {op}", wl=static_drop(Tv, nuv, R=R, kappa=kappa), operator=op,
                                 a=av, tags={"kind": kind, "value": v}))
    return jobs


def impact(nu, U, R0=50.0, T=0.59, kappa=0.01, W=5.0, width=24, height=12):
    """The 2-D drop impact of the stability study: a drop of radius R0 at speed U over
    a film of thickness R0 on the bottom wall, in a (width R0) x (height R0) box."""
    return WL.Workload(name=f"impact R0={R0:g} nu={nu:g} U={U:g}", D=2, nx=int(width * R0), ny=int(height * R0),
                       nz=1, T_over_Tc=T, kappa=kappa, nu_liquid=nu, mu_ratio=0.0, R=R0, U=U, film=1.0, W=W,
                       walls_axis=1)


def stability_jobs(nus, Us, R0=50.0, width=24, height=12):
    """Drop-impact jobs over the (nu, U0) grid, both operators, nu_v = 15 nu_l."""
    jobs = []
    for nu in nus:
        for U in Us:
            for op in OPERATORS:
                jobs.append(StudyJob(name=f"nu={nu:g} U={U:g} {op}", wl=impact(nu, U, R0=R0, width=width, height=height),
                                     operator=op, nu_vapour_ratio=15.0, tags={"nu": nu, "U": U}))
    return jobs


def fit_power(x, y):
    """Least-squares exponent m and prefactor c of y = c x^m (x, y > 0)."""
    lx, ly = np.log(np.asarray(x, float)), np.log(np.asarray(y, float))
    m, lc = np.polyfit(lx, ly, 1)
    return float(m), float(math.exp(lc))


def initial_fields(job: StudyJob, rv, rl):
    wl = job.wl
    if wl.U > 0 or wl.film > 0:
        return I.drop_on_film(wl.shape, 2, wl.R, wl.film * wl.R, wl.U, rl, rv, wl.W)
    return WL.initial_fields(wl, rv, rl)


# ---------------------------------------------------------------------------
# GPU execution
# ---------------------------------------------------------------------------

def run_jobs(jobs, steps, chunk=500, max_u_limit=0.5, keep_density=False):
    """Advance every job by up to `steps` in batched chunks.  Returns one record per
    job: steps completed, whether it stayed stable (finite positive density and
    max|u| below max_u_limit; u the reported velocity), the max|u| history (one
    value per chunk) and the final max|u| (with keep_density, the final density
    field of every stable job too); plus the batched throughput."""
    doms, recs = [], []
    lups, t_gpu = 0, 0.0
    try:
        for j in jobs:
            rv, rl = j.coexistence()
            d = lbm.Domain(j.params(rv, rl))
            rho, u = initial_fields(j, rv, rl)
            d.lbm_init_fields(rho, u)
            doms.append(d)
            recs.append(dict(name=j.name, operator=j.operator, tags=j.tags, rho_l=rl, rho_v=rv, steps=0, stable=True,
                             max_u=[], final_max_u=None))
        live = list(range(len(jobs)))
        done = 0
        while done < steps and live:
            n = min(chunk, steps - done)
            t0 = time.perf_counter()
            with lbm.Batch([doms[k] for k in live]) as b:
                b.lbm_batch_step(n)
                try:
                    b.lbm_batch_synchronize()
                except lbm.LBMError:
                    pass  # the failing jobs are found below
            t_gpu += time.perf_counter() - t0
            lups += n * sum(jobs[k].wl.N for k in live)
            done += n
            still = []
            for k in live:
                r = recs[k]
                try:
                    doms[k].lbm_synchronize()
                    mu = doms[k].lbm_max_speed()
                except lbm.LBMError:
                    mu = float("nan")
                r["max_u"].append(mu)
                if not (mu == mu) or mu > max_u_limit:
                    r["stable"] = False
                    r["failed_at"] = done
                    r["failure"] = "speed limit" if mu == mu and mu != float("inf") else "non-finite"
                else:
                    r["steps"] = done
                    r["final_max_u"] = mu
                    still.append(k)
            live = still
        if keep_density:
            for k in live:
                recs[k]["rho"] = doms[k].lbm_read_macroscopic()[0][0]
        return dict(jobs=recs, steps=steps, chunk=chunk, batched_mlups=lups / max(t_gpu, 1e-9) / 1e6)
    finally:
        for d in doms:
            d.close()


def pr_pressure(rho, T, a=WL.PAPER_EOS["a"], b=WL.PAPER_EOS["b"], R=WL.PAPER_EOS["R"], acentric=WL.PAPER_EOS["acentric"]):
    """Peng-Robinson pressure (Eq. PREoS) at reduced temperature T."""
    Tc = 0.0778 * a / (0.45724 * b * R)
    m = 0.37464 + 1.54226 * acentric - 0.26992 * acentric ** 2
    al = (1 + m * (1 - math.sqrt(T))) ** 2
    return rho * R * T * Tc / (1 - b * rho) - a * al * rho ** 2 / (1 + 2 * b * rho - b * b * rho ** 2)


def interface_width(rho, rho_in, rho_out):
    """W = (rho_l - rho_v) / max |grad rho| (the paper's interface thickness),
    central differences on the periodic 2-D field."""
    gy = 0.5 * (np.roll(rho, -1, 0) - np.roll(rho, 1, 0))
    gx = 0.5 * (np.roll(rho, -1, 1) - np.roll(rho, 1, 1))
    return float(abs(rho_in - rho_out) / np.max(np.hypot(gx, gy)))


def laplace_measure(rho, R0):
    """Pressure-jump inputs of a 2-D drop centred in its box: the equimolar radius
    R_e (the disc that holds the excess mass at the bulk jump), the interface width
    W, and the bulk densities inside (r < R_e - 4W) and outside (r > R_e + 4W).
    Starts from the initial radius R0 and refines once with the measured R_e, W."""
    ny, nx = rho.shape
    yy, xx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    r = np.hypot(xx - nx / 2, yy - ny / 2)
    r_out = float(np.mean(rho[r > R0 + 12]))
    r_in = float(np.mean(rho[r < R0 / 2]))
    Re, W = R0, 0.0
    for _ in range(2):
        Re = math.sqrt(float(np.sum(rho - r_out)) / (math.pi * (r_in - r_out)))
        W = interface_width(rho, r_in, r_out)
        inner, outer = r < max(Re - 4 * W, Re / 4), r > Re + 4 * W
        if outer.any():
            r_out = float(np.mean(rho[outer]))
        r_in = float(np.mean(rho[inner]))
    return r_in, r_out, Re, W


def surface_tension_jobs(Ts, radii, kappa=0.01, nu=0.1, radii_near_tc=None, t_near=0.85, a=WL.PAPER_EOS["a"]):
    """Static drops, entropic operator: every radius at every temperature (radii_near_tc
    instead at T/Tc >= t_near, where the interface is wider), EOS constant a."""
    jobs = []
    for T in Ts:
        for R in (radii_near_tc if (radii_near_tc and T >= t_near - 1e-12) else radii):
            jobs.append(StudyJob(name=f"a={a:g} T={T:g} R={R:g}", wl=static_drop(T, nu, R=R, kappa=kappa),
                                 operator="entropic", a=a, tags={"T": T, "R": R, "a": a}))
    return jobs


# The EOS constants a of the surface-tension sweep (three values at fixed kappa, as in
# Sec. 3.1.2; the interface width grows as sqrt(kappa/a)).
SIGMA_A_VALUES = (0.003, 0.0017, 0.0011)


def _sigma_rows(jobs, Ts, a):
    """Laplace-law sigma per temperature for the drops of EOS constant a, and the
    exponents of sigma ~ (1 - T/Tc)^m near and below T/Tc = 0.8."""
    rows = []
    for T in Ts:
        pts = []
        for r in jobs:
            if r["tags"]["a"] == a and r["tags"]["T"] == T and r["stable"]:
                r_in, r_out, Re, W = laplace_measure(r["rho"], r["tags"]["R"])
                dP = pr_pressure(r_in, T, a=a) - pr_pressure(r_out, T, a=a)
                pts.append(dict(R0=r["tags"]["R"], R_e=Re, W=W, rho_in=r_in, rho_out=r_out, dP=dP, dP_Re=dP * Re,
                                max_u=r["final_max_u"], steps=r["steps_run"]))
        row = dict(a=a, T_over_Tc=T, drops=pts)
        if len(pts) >= 2:
            # Delta P = sigma / R_e (2-D): slope of Delta P against 1/R_e
            slope, icpt = np.polyfit([1 / p["R_e"] for p in pts], [p["dP"] for p in pts], 1)
            row.update(sigma=float(slope), intercept=float(icpt))
        rows.append(row)
    fits = {}
    for name, lo, hi in (("m_near_critical", 0.8, 1.0), ("m_below_0.8", 0.0, 0.8 + 1e-9)):
        pts = [(1 - r["T_over_Tc"], r["sigma"]) for r in rows if "sigma" in r and r["sigma"] > 0 and lo <= r["T_over_Tc"] < hi]
        if len(pts) >= 2:
            fits[name] = fit_power([p[0] for p in pts], [p[1] for p in pts])[0]
    return rows, fits


def surface_tension_study(quick=False, a_values=None):
    """sigma(T) from the Laplace law at three radii per temperature, for each EOS
    constant a, and the exponents.  Radii scale with the interface width (as
    sqrt(a0/a)) and step counts with the settling time (as a0/a: the sound speed
    goes as sqrt(a) and the viscous time as R^2)."""
    a0 = WL.PAPER_EOS["a"]
    a_values = tuple(a_values or ((a0,) if quick else SIGMA_A_VALUES))
    if quick:
        groups = [((0.6, 0.75), (25.0, 40.0), 3000)]
    else:
        # near the critical point the interface is wider (R0/W > 10 needs larger drops)
        # and the drops take longer to settle at their Laplace-shifted densities
        groups = [((0.5, 0.55, 0.6, 0.65, 0.7, 0.75, 0.8), (30.0, 45.0, 60.0), 20000),
                  ((0.85, 0.9, 0.95), (120.0, 160.0, 200.0), 100000)]
    jobs_out, lups_s = [], []
    for a in a_values:
        scale = math.sqrt(a0 / a)
        for g_Ts, g_radii, g_steps in groups:
            radii = tuple(float(round(r * scale)) for r in g_radii)
            steps = int(round(g_steps * a0 / a / 500.0)) * 500
            r = run_jobs(surface_tension_jobs(g_Ts, radii, a=a), steps, chunk=max(500, steps // 10), keep_density=True)
            for j in r["jobs"]:
                j["steps_run"] = steps
            jobs_out += r["jobs"]
            lups_s.append(r["batched_mlups"])
    Ts = [T for g in groups for T in g[0]]
    rows, fits = [], []
    for a in a_values:
        ra, fa = _sigma_rows(jobs_out, Ts, a)
        rows += ra
        fits.append(dict(a=a, **fa))
    out = dict(groups=[dict(T_over_Tc=list(g[0]), radii=list(g[1]), steps=g[2]) for g in groups],
               a_values=list(a_values), rows=rows, fits=fits, batched_mlups=min(lups_s))
    out.update({k: v for k, v in fits[0].items() if k != "a"})  # the exponents at the first a
    return out


def crown_fits(t, r, tc, tau, windows):
    """Exponent p and prefactor c of r = c (t - tc)^p over each window [lo, hi] of
    t - tc, in units of tau (samples with r > 0 only; at least three per window)."""
    fits = []
    for lo, hi in windows:
        pts = [(ti - tc, ri) for ti, ri in zip(t, r) if lo * tau <= ti - tc <= hi * tau and ri > 0]
        if len(pts) >= 3:
            p, c = fit_power([q[0] for q in pts], [q[1] for q in pts])
            fits.append(dict(window_tau=[lo, hi], p=p, c=c, points=len(pts)))
    return fits


def crown_study(quick=False, wl=None, t_end_tau=2.0, samples=100, precision=lbm.LBM_FP32,
                fit_windows=((0.05, 1.0),)):
    """Crown radius r(t) of a 2-D drop impact (entropic operator), sampled on the
    GPU in the layer y = h + 2 above the film, the exponent p of r ~ (t - t0)^p over
    0.05 tau <= t - t0 <= tau (t0 = first sample with a crown, tau = 2R/U; more
    windows in fit_windows, the first one reported as "fit"), and the
    2/(omega gamma) field of the last step: its share of nodes within 5% of 1 and
    the same share at interface nodes (0.1 < phase fraction < 0.9)."""
    if wl is None:
        wl = WL.DROP_IMPACT_2D if not quick else dataclasses.replace(
            WL.DROP_IMPACT_2D, name="D2Q9 drop impact 512x256 (R = 32)", nx=512, ny=256, R=32.0)
    rv, rl = WL.coexistence(wl)
    tau = 2.0 * wl.R / wl.U
    n_end = int(round(t_end_tau * tau))
    every = max(1, n_end // samples)
    layer = int(round(wl.film * wl.R + 2))
    out = dict(workload=wl.name, tau=tau, layer=layer, every=every, t=[], r=[])
    with lbm.Domain(WL.params(wl, precision, rv=rv, rl=rl)) as dom:
        # the geometry of WL.initial_fields, built on the GPU (gap 2W above the film)
        dom.lbm_init_drop_on_film(wl.R, wl.film * wl.R, 2.0 * wl.W, wl.U, wl.W, noise=wl.noise, seed=I.SEED_BASE)
        t0 = time.perf_counter()
        done = 0
        try:
            for k in range(0, n_end, every):
                if k + every >= n_end:
                    dom.lbm_record_gamma(True)  # the last chunk's final step is recorded
                dom.lbm_step(every)
                done = k + every
                out["t"].append(done)
                out["r"].append(dom.lbm_crown_radius(layer))
        except lbm.LBMError as e:
            out["failed"] = dict(after_step=done, within=every, error=str(e)[:120])
            hit = [t for t, r in zip(out["t"], out["r"]) if r > 0]
            out["t_contact"] = hit[0] if hit else None  # the crown had formed before the failure
            return out
        out["seconds"] = time.perf_counter() - t0
        out["mlups"] = wl.N * n_end / out["seconds"] / 1e6
        out["interface_width"] = dom.lbm_interface_width()[0]
        small = wl.N <= 50_000_000  # full fields are read to the host only for small domains
        rel = dom.lbm_read_relaxation() if small else None
        rho = dom.lbm_read_macroscopic()[0] if small else None
    if rel is not None:
        near1 = np.abs(rel - 1.0) < 0.05
        out["relaxation"] = dict(share_within_5pct=float(near1.mean()))
        phi = (rho - rv) / (rl - rv)
        iface = (phi > 0.1) & (phi < 0.9)
        out["relaxation"].update(share_within_5pct_at_interfaces=float(near1[iface].mean()) if iface.any() else None,
                                 share_within_5pct_in_bulk=float(near1[~iface].mean()))
    hit = [i for i, r in enumerate(out["r"]) if r > 0]
    if hit:
        tc = out["t"][hit[0]]
        out["t_contact"] = tc
        out["fits"] = crown_fits(out["t"], out["r"], tc, tau, fit_windows)
        if out["fits"] and out["fits"][0]["window_tau"] == list(fit_windows[0]):
            out["fit"] = {k: v for k, v in out["fits"][0].items() if k != "window_tau"}
    return out


# The paper's 2-D impacts (Sec. 3.2): (We, Re) pairs with We = 2 rho_l R0 U0^2 / sigma and
# Re = 2 U0 R0 / nu_l, in a 24 R0 x 12 R0 box with a film h = R0, T/Tc = 0.59, nu_v = 15 nu_l.
PAPER_2D_CASES = ((57, 4000), (93, 4000), (238, 4000), (93, 100))
# sigma at T/Tc = 0.59 with a = 0.003 and kappa = 0.01: the Laplace-law sweep of
# surface_tension_study gives 0.203 at 0.55 and 0.169 at 0.6; linear in between.
SIGMA_T059 = WL.SIGMA_T059


def paper_2d_impacts(R0=100.0, sigma=SIGMA_T059, cases=PAPER_2D_CASES):
    """Workloads of the paper's 2-D impact cases: U0 from We and sigma, nu_l from Re."""
    T = 0.59
    rv, rl, _ = lbm.lbm_coexistence(lbm.lbm_default_params(T_over_Tc=T, **WL.PAPER_EOS))
    out = []
    for We, Re in cases:
        U = math.sqrt(We * sigma / (2.0 * rl * R0))
        nu = 2.0 * U * R0 / Re
        out.append(WL.Workload(name=f"paper 2-D impact We={We} Re={Re} ({int(24 * R0)}x{int(12 * R0)}, R0={R0:g})",
                               D=2, nx=int(24 * R0), ny=int(12 * R0), nz=1, T_over_Tc=T, kappa=0.01,
                               nu_liquid=nu, mu_ratio=0.0, R=R0, U=U, film=1.0, walls_axis=1,
                               extra={"nu_vapour_ratio": 15.0, "We": We, "Re": Re}))
    return out


# The paper's 3-D impacts (Sec. 3.3): We 82, 167 and 328 for one fluid (water/air), so
# Re grows as sqrt(We) over the stated 3500-6900; R0 = 80 in a 14 R0 x 14 R0 x 6 R0 box,
# a film h/2R0 = 0.22, 5% white noise on the drop's velocity, T/Tc = 0.59, nu_v = 15 nu_l.
PAPER_3D_WE = (82, 167, 328)
PAPER_3D_RE_AT_FIRST = 3500.0


def paper_3d_impacts(R0=80.0, sigma=SIGMA_T059, weber=PAPER_3D_WE, re_first=PAPER_3D_RE_AT_FIRST):
    """Workloads of the paper's 3-D impact cases at the paper's EOS and kappa: U0 from
    We and sigma, one liquid viscosity for all (Re = re_first at the first We)."""
    T = 0.59
    rv, rl, _ = lbm.lbm_coexistence(lbm.lbm_default_params(T_over_Tc=T, **WL.PAPER_EOS))
    U = [math.sqrt(We * sigma / (2.0 * rl * R0)) for We in weber]
    nu = 2.0 * U[0] * R0 / re_first
    out = []
    for We, u in zip(weber, U):
        Re = 2.0 * u * R0 / nu
        n, nz = int(14 * R0), int(6 * R0)
        out.append(WL.Workload(name=f"paper 3-D impact We={We} Re={Re:.0f} ({n}x{n}x{nz}, R0={R0:g})",
                               D=3, nx=n, ny=n, nz=nz, T_over_Tc=T, kappa=0.01, nu_liquid=nu, mu_ratio=0.0,
                               R=R0, U=u, film=0.44, walls_axis=2, noise=0.05,
                               extra={"nu_vapour_ratio": 15.0, "We": We, "Re": Re}))
    return out


def paper_3d_crown_study(quick=False, t_end_tau=1.0):
    """Crown radius series of the paper's three 3-D impact cases at the paper's size
    (6.0e8 nodes, 85 GB each; about a minute per convective time on one GB300); quick
    runs them at R0 = 20, where the same We needs twice the impact speed (and the
    faster cases diverge sooner).  A case that diverges is reported with the step it
    reached."""
    rows = []
    for wl in paper_3d_impacts(R0=20.0 if quick else 80.0):
        res = crown_study(wl=wl, t_end_tau=t_end_tau, samples=40)
        rows.append(dict(We=wl.extra["We"], Re=wl.extra["Re"], U0=wl.U, nu_l=wl.nu_liquid,
                         **{k: res[k] for k in ("tau", "t", "r", "t_contact", "fit", "failed", "seconds", "mlups",
                                                "interface_width") if k in res}))
    return dict(cases=rows)


def paper_crown_study(quick=False, t_end_tau=2.0):
    """Crown radius series of the paper's four 2-D impact cases and their exponents.
    The cases run at the paper's resolution (R0 = 100: under a second each on one
    GPU); quick stops at half a convective time."""
    if quick:
        t_end_tau = min(t_end_tau, 0.5)
    rows = []
    for wl in paper_2d_impacts():
        # the paper's square-root law is for the initial stages: fit 0.01-0.1 tau after
        # contact (samples every 0.005 tau), and report later windows beside it
        res = crown_study(wl=wl, t_end_tau=t_end_tau, samples=int(200 * t_end_tau),
                          fit_windows=((0.01, 0.1), (0.1, 0.5), (0.5, 2.0)))
        rows.append(dict(We=wl.extra["We"], Re=wl.extra["Re"], U0=wl.U, nu_l=wl.nu_liquid,
                         **{k: res[k] for k in ("tau", "t", "r", "t_contact", "fit", "fits", "failed", "seconds",
                                                "mlups", "relaxation") if k in res}))
    return dict(cases=rows)


def paper_coexistence_study(temps=(0.5, 0.55, 0.59, 0.65, 0.7, 0.75, 0.8, 0.85, 0.9, 0.95), kappa=0.005,
                            cap_steps=200000, chunk=2000, tol=1e-8, quick=False):
    """The coexistence test of Sec. 3.1.1 in the paper's geometry: an 800 x 10 periodic
    D2Q9 box, a 400-node liquid column in the middle, float64, entropic operator, run
    until max |rho(t + chunk) - rho(t)| / rho_l < tol (the steady state) or cap_steps.
    Reports the bulk densities against the Maxwell construction and the interface
    width W = (rho_l - rho_v) / max |grad rho|."""
    nx, ny = (200, 10) if quick else (800, 10)
    if quick:
        temps, cap_steps = temps[:2], min(cap_steps, 4000)
    rows = []
    for T in temps:
        rv, rl, _ = lbm.lbm_coexistence(lbm.lbm_default_params(T_over_Tc=T, **WL.PAPER_EOS))
        wl = WL.Workload(name=f"coexistence 800x10 T/Tc={T:g}", D=2, nx=nx, ny=ny, nz=1, T_over_Tc=T, kappa=kappa,
                         nu_liquid=0.1, mu_ratio=0.0, R=1.0, U=0.0, film=0.0)
        rho0 = I.slab((1, ny, nx), 0, nx / 4, 3 * nx / 4, rl, rv, 5.0)
        steps, steady, t0 = 0, False, time.perf_counter()
        with lbm.Domain(WL.params(wl, lbm.LBM_FP64, rv=rv, rl=rl)) as dom:
            dom.lbm_init_fields(rho0, np.zeros((2, 1, ny, nx)))
            prev = dom.lbm_read_macroscopic()[0]
            while steps < cap_steps:
                dom.lbm_step(chunk)
                steps += chunk
                rho = dom.lbm_read_macroscopic()[0]
                change = float(np.max(np.abs(rho - prev))) / rl
                prev = rho
                if change < tol:
                    steady = True
                    break
            W = dom.lbm_interface_width()[0]
        line = prev[0, ny // 2]
        r_l = float(np.mean(line[3 * nx // 8: 5 * nx // 8]))
        r_v = float(np.mean(np.concatenate([line[: nx // 8], line[-nx // 8:]])))
        rows.append(dict(T_over_Tc=T, rho_l=r_l, rho_v=r_v, rho_l_maxwell=rl, rho_v_maxwell=rv,
                         err_l=r_l / rl - 1.0, err_v=r_v / rv - 1.0, W=W, steps=steps, steady=steady,
                         last_change=change, seconds=time.perf_counter() - t0))
    return dict(geometry=f"{nx}x{ny}", kappa=kappa, tol=tol, rows=rows)


def spurious_study(quick=False):
    """The three spurious-current sweeps and the temperature exponent."""
    if quick:
        Ts, nus, As, R, steps = (0.59, 0.8), (0.01, 0.1), (0.003, 0.0017), 20.0, 2000
    else:
        Ts = (0.5, 0.55, 0.59, 0.65, 0.7, 0.75, 0.8, 0.85, 0.9, 0.95)
        nus = (0.001, 0.0025, 0.005, 0.01, 0.02, 0.03, 0.05, 0.1)
        As = (0.003, 0.0017, 0.0011)
        R, steps = 40.0, 20000
    out = {}
    for kind, vals in (("T", Ts), ("nu", nus), ("a", As)):
        res = run_jobs(spurious_jobs(kind, vals, R=R), steps, chunk=max(500, steps // 20))
        rows = []
        for v in vals:
            row = {"value": v}
            for r in res["jobs"]:
                if r["tags"]["value"] == v:
                    row[r["operator"]] = r["final_max_u"] if r["stable"] else None
                    row[r["operator"] + "_history"] = r["max_u"]
            rows.append(row)
        out[kind] = dict(rows=rows, steps=steps, batched_mlups=res["batched_mlups"])
    for op in OPERATORS:
        pts = [(1 - r["value"], r[op]) for r in out["T"]["rows"] if r.get(op)]
        if len(pts) >= 2:
            out["T"][f"m_{op}"] = fit_power([p[0] for p in pts], [p[1] for p in pts])[0]
    return out


def stability_study(quick=False):
    """The (nu, U0) stability domain of both operators."""
    if quick:
        nus, Us, R0, steps = (0.005, 0.05), (0.0, 0.08), 20.0, 2000
    else:
        nus = (0.0025, 0.005, 0.01, 0.02, 0.03, 0.04, 0.06, 0.1)
        Us = (0.0, 0.04, 0.08, 0.12, 0.16)
        R0, steps = 50.0, 5000
    res = run_jobs(stability_jobs(nus, Us, R0=R0), steps, chunk=500)
    table = {op: {f"{nu:g}": {f"{U:g}": None for U in Us} for nu in nus} for op in OPERATORS}
    for r in res["jobs"]:
        table[r["operator"]][f"{r['tags']['nu']:g}"][f"{r['tags']['U']:g}"] = (
            "stable" if r["stable"] else f"{r['failure']}@{r['failed_at']}")
    lowest = {}
    for op in OPERATORS:
        ok = [nu for nu in nus if all(table[op][f"{nu:g}"][f"{U:g}"] == "stable" for U in Us)]
        lowest[op] = min(ok) if ok else None
    return dict(R0=R0, steps=steps, nus=list(nus), Us=list(Us), table=table,
                lowest_nu_stable_for_all_U=lowest, batched_mlups=res["batched_mlups"])


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("study", choices=["spurious", "stability", "surface-tension", "crown", "coexistence"])
    ap.add_argument("--quick", action="store_true", help="small sizes and few steps")
    ap.add_argument("--workload", default=None, help="crown: a workload name (default drop2d; drop3d-paper: the paper's 3-D size at We ~ 20; paper-2d: the paper's four 2-D cases; paper-3d: the paper's three 3-D cases)")
    ap.add_argument("--tau", type=float, default=2.0, help="crown: simulated time in convective times 2R/U")
    ap.add_argument("--a", default=None, help="surface-tension: comma-separated EOS constants a (default 0.003,0.0017,0.0011)")
    args = ap.parse_args()
    lbm.load()
    if args.study == "crown" and args.workload == "paper-2d":
        res = paper_crown_study(args.quick, t_end_tau=args.tau)
    elif args.study == "crown" and args.workload == "paper-3d":
        res = paper_3d_crown_study(args.quick, t_end_tau=args.tau)
    elif args.study == "crown":
        res = crown_study(args.quick, wl=WL.by_name(args.workload) if args.workload else None, t_end_tau=args.tau)
    elif args.study == "coexistence":
        res = paper_coexistence_study(quick=args.quick)
    elif args.study == "surface-tension":
        a_values = tuple(float(v) for v in args.a.split(",")) if args.a else None
        res = surface_tension_study(args.quick, a_values=a_values)
    else:
        res = {"spurious": spurious_study, "stability": stability_study}[args.study](args.quick)
    print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
