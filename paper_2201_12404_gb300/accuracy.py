"""Accuracy of the reduced-precision paths against the float64 path on the GPU.

For each workload the same seeded initial fields are advanced with LBM_FP64,
LBM_FP32 and LBM_FP16DEV storage, and the float32/float16 results are compared
with the float64 one:

  - density L_inf error relative to the liquid density,
  - velocity L_inf error relative to max |u| of the float64 field,
  - the same two errors averaged over the domain (a moving interface shifted by
    one node already gives an L_inf density error of order one),
  - spreading radius of the drop-impact workloads: the largest horizontal
    distance from the impact axis of a node with rho > (rho_l + rho_v)/2 in the
    layer two nodes above the initial film (Secs. 3.2-3.3), at several times,
  - mass drift of every path.

The static drop (Sec. 3.1.2) also reports the Laplace pressure jump
Delta P = P(rho_in) - P(rho_out) times the equimolar radius for two radii, the
two products being the same surface tension when Laplace's law holds.

  python -m paper_2201_12404_gb300.accuracy [--quick] [--part coexistence]

The coexistence sweep (Sec. 3.1.1) runs 16 flat-interface jobs of uneven sizes in one
persistent batched launch and compares the bulk densities with the Maxwell
construction.

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


def compare(wl, checkpoints):
    """The three paths advanced in lockstep from the same initial fields; at every
    checkpoint the float32 and float16-deviation fields are compared with float64."""
    rv, rl = WL.coexistence(wl)
    rho0, u0 = WL.initial_fields(wl, rv, rl)
    names = (("fp64", lbm.LBM_FP64), ("fp32", lbm.LBM_FP32), ("fp16dev", lbm.LBM_FP16DEV))
    doms = {}
    out = dict(workload=wl.name, rho_liquid=rl, rho_vapour=rv, tau_steps=(2 * wl.R / wl.U if wl.U > 0 else None),
               checkpoints=[])
    try:
        for name, prec in names:
            doms[name] = lbm.Domain(WL.params(wl, prec, rv=rv, rl=rl))
            doms[name].lbm_init_fields(rho0, u0)
        mass0 = {k: d.lbm_read_diag()["mass"] for k, d in doms.items()}
        seconds = {k: 0.0 for k in doms}
        failed = {}
        done = 0
        for cp in checkpoints:
            snap = {}
            for k, d in doms.items():
                if k in failed:
                    continue
                t0 = time.perf_counter()
                try:
                    d.lbm_step(cp - done)
                    d.lbm_synchronize()
                except lbm.LBMError as e:
                    failed[k] = f"{e} (before step {cp})"
                    continue
                seconds[k] += time.perf_counter() - t0
                rho, u = d.lbm_read_macroscopic()
                snap[k] = dict(rho=rho, u=u, mass_drift=(d.lbm_read_diag()["mass"] - mass0[k]) / mass0[k])
            done = cp
            row = dict(step=cp)
            ref = snap.get("fp64")
            for k in doms:
                if k not in snap:
                    row[k] = dict(status=failed.get(k, "failed"))
                    continue
                e = dict(mass_drift=snap[k]["mass_drift"])
                if wl.U > 0:
                    e["spreading_radius"] = spreading_radius(snap[k]["rho"], wl, rv, rl)
                if k != "fp64" and ref is not None:
                    dr = np.abs(snap[k]["rho"] - ref["rho"]) / rl
                    umax = max(float(np.max(np.abs(ref["u"]))), 1e-300)
                    du = np.abs(snap[k]["u"] - ref["u"]) / umax
                    e.update(rho_linf_rel=float(dr.max()), rho_l1_rel=float(dr.mean()),
                             u_linf_rel=float(du.max()), u_l1_rel=float(du.mean()))
                    if "spreading_radius" in e:
                        e["spreading_radius_diff"] = e["spreading_radius"] - spreading_radius(ref["rho"], wl, rv, rl)
                row[k] = e
            out["checkpoints"].append(row)
        out["mlups"] = {k: (wl.N * done / seconds[k] / 1e6 if k not in failed and seconds[k] > 0 else None)
                        for k in doms}
    finally:
        for d in doms.values():
            d.close()
    return out


def laplace(wl_base, radii, steps):
    """Static drops (float64): Delta P and the equimolar radius R_e for each initial radius.
    Densities inside/outside are averages over the drop core (r < R_e/2) and over the
    far field (r > R_e + 12); Delta P uses the Peng-Robinson pressure of those densities."""
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
        yy, xx = np.meshgrid(np.arange(sh[1]), np.arange(sh[2]), indexing="ij")
        r = np.hypot(xx - sh[2] / 2, yy - sh[1] / 2)
        r_out = float(np.mean(rho[0][r > R + 12]))
        r_in0 = float(np.mean(rho[0][r < R / 2]))
        # equimolar radius of a 2-D drop: the disc holding the excess mass at the bulk jump
        excess = float(np.sum(rho - r_out))
        Re = math.sqrt(excess / (math.pi * (r_in0 - r_out)))
        r_in = float(np.mean(rho[0][r < Re / 2]))
        pr = lbm.lbm_default_params(T_over_Tc=wl_base.T_over_Tc, **WL.PAPER_EOS)
        dP = _pressure(pr, r_in) - _pressure(pr, r_out)
        res.append(dict(R0=R, steps=steps, rho_in=r_in, rho_out=r_out, R_e=Re, dP=dP, sigma=dP * Re,
                        max_u=float(np.max(np.abs(u))), mass_drift=(m1 - m0) / m0))
    return res


def coexistence_sweep(n_jobs=16, cap_steps=50000, chunk=1000, tol=1e-5, seed=None):
    """Flat-interface coexistence (Sec. 3.1.1) for n_jobs D2Q9 jobs of uneven sizes
    (n_x = 64 (1 + k mod 4), n_y = 4 n_x, assigned to the temperatures by a seeded
    shuffle), T/Tc evenly spaced over [0.5, 0.95], a liquid slab over the middle half of
    n_y, nu = 0.1, float32, all advanced by one persistent batched launch per chunk
    until max |rho(t + chunk) - rho(t)| / rho_l < tol for every job (or cap_steps).
    The bulk densities (averages over the middle quarter of the slab and the quarter of
    the domain farthest from it) are compared with the Maxwell construction."""
    from . import inputs as I
    seed = I.SEED_BASE if seed is None else seed
    sizes = [64 * (1 + (k % 4)) for k in range(n_jobs)]
    order = I.rng(seed).permutation(n_jobs)
    trs = [0.5 + 0.45 * k / (n_jobs - 1) for k in range(n_jobs)]
    doms, meta = [], []
    try:
        for k in range(n_jobs):
            nx = sizes[order[k]]
            ny = 4 * nx
            Tr = trs[k]
            rv, rl, _ = lbm.lbm_coexistence(lbm.lbm_default_params(T_over_Tc=Tr, **WL.PAPER_EOS))
            wl = WL.Workload(name=f"coex{k}", D=2, nx=nx, ny=ny, nz=1, T_over_Tc=Tr, kappa=0.005, nu_liquid=0.1,
                             mu_ratio=0.0, R=1.0, U=0.0, film=0.0)
            p = WL.params(wl, lbm.LBM_FP32, rv=rv, rl=rl)
            d = lbm.Domain(p)
            rho = I.slab((1, ny, nx), 1, ny / 4, 3 * ny / 4, rl, rv, 5.0)
            d.lbm_init_fields(rho, np.zeros((2, 1, ny, nx)))
            doms.append(d)
            meta.append(dict(T_over_Tc=Tr, nx=nx, ny=ny, rho_l_maxwell=rl, rho_v_maxwell=rv))
        prev = [d.lbm_read_macroscopic()[0] for d in doms]
        steps, done = 0, [False] * n_jobs
        t_gpu = 0.0
        with lbm.Batch(doms) as b:
            b.lbm_batch_tune(5)
            info = b.lbm_batch_info()
            while steps < cap_steps and not all(done):
                t0 = time.perf_counter()
                b.lbm_batch_step(chunk)
                b.lbm_batch_synchronize()
                t_gpu += time.perf_counter() - t0
                steps += chunk
                for k, d in enumerate(doms):
                    r = d.lbm_read_macroscopic()[0]
                    if not done[k] and np.max(np.abs(r - prev[k])) / meta[k]["rho_l_maxwell"] < tol:
                        done[k] = True
                        meta[k]["steady_at"] = steps
                    prev[k] = r
        nodes = sum(m["nx"] * m["ny"] for m in meta)
        rows = []
        for k, m in enumerate(meta):
            r = prev[k][0]
            ny = m["ny"]
            liquid = float(np.mean(r[3 * ny // 8: 5 * ny // 8]))
            vapour = float(np.mean(np.concatenate([r[: ny // 8], r[7 * ny // 8:]])))
            rows.append(dict(m, rho_l=liquid, rho_v=vapour, err_l=liquid / m["rho_l_maxwell"] - 1,
                             err_v=vapour / m["rho_v_maxwell"] - 1, steady=done[k]))
        return dict(workload="D2Q9 flat-interface coexistence sweep, 16 jobs 64x256..256x1024, FP32, one batched launch",
                    steps=steps, batch=info, batched_mlups=nodes * steps / t_gpu / 1e6, jobs=rows)
    finally:
        for d in doms:
            d.close()


def _pressure(p, rho):
    Tc = 0.0778 * p.a / (0.45724 * p.b * p.R)
    m = 0.37464 + 1.54226 * p.acentric - 0.26992 * p.acentric ** 2
    al = (1 + m * (1 - math.sqrt(p.T_over_Tc))) ** 2
    return rho * p.R * p.T_over_Tc * Tc / (1 - p.b * rho) - p.a * al * rho ** 2 / (1 + 2 * p.b * rho - p.b ** 2 * rho ** 2)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--quick", action="store_true", help="fewer steps (a smoke run)")
    ap.add_argument("--part", default="all", help="all, laplace, precision or coexistence")
    args = ap.parse_args()
    k = 10 if args.quick else 1
    lbm.load()
    if args.part == "coexistence":
        print(json.dumps(coexistence_sweep(cap_steps=50000 // k)), flush=True)
        return
    static = WL.STATIC_DROP_2D
    print(json.dumps({"workload": static.name, "laplace_fp64": laplace(static, (20, 25, 30), static.steps // k)}), flush=True)
    print(json.dumps({"workload": static.name, "laplace_fp64": laplace(static, (20, 25, 30), 10 * static.steps // k)}), flush=True)
    print(json.dumps(compare(static, [static.steps // k])), flush=True)
    d2 = WL.DROP_IMPACT_2D
    print(json.dumps(compare(d2, [c // k for c in (1000, 2500, 5000, 10000, 20000)])), flush=True)
    d3 = WL.DROP_IMPACT_3D_SMALL
    print(json.dumps(compare(d3, [c // k for c in (250, 500, 1000, 2000)])), flush=True)
    print(json.dumps(coexistence_sweep(cap_steps=50000 // k)), flush=True)

if __name__ == "__main__":
    main()
