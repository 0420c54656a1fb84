"""Accuracy of the reduced-precision paths against the float64 path on the GPU.

For each workload the same seeded initial fields are advanced with LBM_FP64,
LBM_FP32 and LBM_FP16DEV storage, and the float32/float16 results are compared
with the float64 one:

  - density L_inf error relative to the liquid density,
  - velocity L_inf error relative to max |u| of the float64 field,
  - spreading radius of the drop-impact workloads: the largest horizontal
    distance from the impact axis of a node with rho > (rho_l + rho_v)/2 in the
    layer two nodes above the initial film (Secs. 3.2-3.3),
  - mass drift of every path.

The static drop (Sec. 3.1.2) also reports the Laplace pressure jump
Delta P = P(rho_in) - P(rho_out) times the equimolar radius for two radii, the
two products being the same surface tension when Laplace's law holds.

  python -m paper_2201_12404_gb300.accuracy [--quick]

Prints one JSON object per workload.  Everything runs through the C ABI.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import lbm
from . import workloads as WL


def spreading_radius(rho, wl: WL.Workload, rv, rl):
    h = wl.film * wl.R
    layer = int(round(h)) + 2
    thr = 0.5 * (rl + rv)
    if wl.D == 2:
        row = rho[0, layer, :]
        xs = np.nonzero(row > thr)[0]
        if len(xs) == 0:
            return 0.0
        return float(np.max(np.abs(xs - 0.5 * (wl.nx - 1))))
    plane = rho[layer]
    ys, xs = np.nonzero(plane > thr)
    if len(xs) == 0:
        return 0.0
    return float(np.max(np.hypot(xs - 0.5 * (wl.nx - 1), ys - 0.5 * (wl.ny - 1))))


def run_path(wl, precision, rho0, u0, steps, rv, rl):
    p = WL.params(wl, precision, rv=rv, rl=rl)
    with lbm.Domain(p) as dom:
        dom.lbm_init_fields(rho0, u0)
        m0 = dom.lbm_read_diag()["mass"]
        t0 = time.perf_counter()
        status = "ok"
        try:
            dom.lbm_step(steps)
            dom.lbm_synchronize()
        except lbm.LBMError as e:
            status = str(e)
        dt = time.perf_counter() - t0
        if status != "ok":
            return dict(status=status, seconds=dt)
        rho, u = dom.lbm_read_macroscopic()
        m1 = dom.lbm_read_diag()["mass"]
    return dict(status=status, seconds=dt, rho=rho, u=u, mass_drift=(m1 - m0) / m0)


def compare(wl, steps, quick=False):
    rv, rl = WL.coexistence(wl)
    rho0, u0 = WL.initial_fields(wl, rv, rl)
    out = dict(workload=wl.name, steps=steps, rho_liquid=rl, rho_vapour=rv)
    ref = None
    for name, prec in (("fp64", lbm.LBM_FP64), ("fp32", lbm.LBM_FP32), ("fp16dev", lbm.LBM_FP16DEV)):
        r = run_path(wl, prec, rho0, u0, steps, rv, rl)
        entry = dict(status=r["status"], seconds=round(r["seconds"], 3),
                     mlups=wl.N * steps / r["seconds"] / 1e6 if r["status"] == "ok" else None)
        if r["status"] == "ok":
            entry["mass_drift"] = r["mass_drift"]
            if wl.U > 0:
                entry["spreading_radius"] = spreading_radius(r["rho"], wl, rv, rl)
            if name == "fp64":
                ref = r
            elif ref is not None:
                umax = float(np.max(np.abs(ref["u"])))
                entry["rho_linf_rel"] = float(np.max(np.abs(r["rho"] - ref["rho"])) / rl)
                entry["u_linf_rel"] = float(np.max(np.abs(r["u"] - ref["u"])) / max(umax, 1e-300))
                if "spreading_radius" in entry:
                    entry["spreading_radius_diff"] = entry["spreading_radius"] - out["fp64"].get("spreading_radius", 0.0)
        out[name] = entry
    return out


def laplace(wl_base, radii, steps):
    """Static drops of two radii (float64): Delta P R_e for each."""
    from . import inputs as I
    rv, rl = WL.coexistence(wl_base)
    res = []
    for R in radii:
        p = WL.params(wl_base, lbm.LBM_FP64, rv=rv, rl=rl)
        sh = wl_base.shape
        rho0 = I.drop(sh, (sh[2] / 2, sh[1] / 2, 0), R, rl, rv, wl_base.W, D=2)
        rho0 = rho0 + I.uniform_noise(sh, 1e-6, I.SEED_BASE + int(R))
        with lbm.Domain(p) as dom:
            dom.lbm_init_fields(rho0, np.zeros((2,) + sh))
            m0 = dom.lbm_read_diag()["mass"]
            dom.lbm_step(steps)
            rho, u = dom.lbm_read_macroscopic()
            m1 = dom.lbm_read_diag()["mass"]
        c = (sh[1] // 2, sh[2] // 2)
        r_in = float(rho[0, c[0], c[1]])
        r_out = float(rho[0, 0, 0])
        # equimolar radius of a 2-D drop: area of the excess mass over the jump
        excess = float(np.sum(rho - r_out))
        Re = math.sqrt(excess / (math.pi * (r_in - r_out)))
        pr = lbm.lbm_default_params(T_over_Tc=wl_base.T_over_Tc, **WL.PAPER_EOS)
        P = lambda r: _pressure(pr, r)
        dP = P(r_in) - P(r_out)
        res.append(dict(R0=R, rho_in=r_in, rho_out=r_out, R_e=Re, dP=dP, sigma=dP * Re,
                        max_u=float(np.max(np.abs(u))), mass_drift=(m1 - m0) / m0))
    return res


def _pressure(p, rho):
    Tc = 0.0778 * p.a / (0.45724 * p.b * p.R)
    m = 0.37464 + 1.54226 * p.acentric - 0.26992 * p.acentric ** 2
    al = (1 + m * (1 - math.sqrt(p.T_over_Tc))) ** 2
    return rho * p.R * p.T_over_Tc * Tc / (1 - p.b * rho) - p.a * al * rho ** 2 / (1 + 2 * p.b * rho - p.b ** 2 * rho ** 2)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--quick", action="store_true", help="fewer steps (a smoke run)")
    args = ap.parse_args()
    k = 10 if args.quick else 1
    lbm.load()
    static = WL.STATIC_DROP_2D
    print(json.dumps({"workload": static.name, "laplace_fp64": laplace(static, (20, 30), static.steps // k)}), flush=True)
    print(json.dumps(compare(static, static.steps // k)), flush=True)
    print(json.dumps(compare(WL.DROP_IMPACT_2D, WL.DROP_IMPACT_2D.steps // k)), flush=True)
    print(json.dumps(compare(WL.DROP_IMPACT_3D_SMALL, 1000 // k)), flush=True)


if __name__ == "__main__":
    main()
