"""Shared test cases: one parameter dictionary feeds both the CUDA library
(lbm_params) and the oracle (orc_params), plus seeded initial states."""
from __future__ import annotations

import numpy as np

import oracle as O
from oracle import thermo
from paper_2201_12404_gb300 import inputs as I
from paper_2201_12404_gb300 import lbm

PAPER_EOS = dict(a=0.003, b=0.095, R=1.0, acentric=0.344)


def case(D, nx, ny, nz=1, *, Tr=0.8, kappa=0.002, nu_l=0.05, nu_v=0.15, walls=False, g=(0.0, 0.0, 0.0),
         gamma_mode=0, gamma_value=2.0, precision=lbm.LBM_FP64, eos_fp64=1, rho_l=None, rho_v=None, a=None):
    if rho_l is None:
        rv, rl, _ = thermo.maxwell(Tr, **PAPER_EOS)
    else:
        rv, rl = rho_v, rho_l
    bc = [0] * 6
    # walls=True: bounce-back walls across the last axis; a tuple: across those axes
    axes = ((1 if D == 2 else 2),) if walls is True else (tuple(walls) if walls else ())
    for ax in axes:
        bc[2 * ax] = bc[2 * ax + 1] = 1
    return dict(D=D, nx=nx, ny=ny, nz=nz if D == 3 else 1, Tr=Tr, kappa=kappa, nu_l=nu_l, nu_v=nu_v,
                rho_l=rl, rho_v=rv, bc=tuple(bc), g=tuple(g), gamma_mode=gamma_mode,
                gamma_value=gamma_value, precision=precision, eos_fp64=eos_fp64,
                eos=dict(PAPER_EOS, **({} if a is None else {"a": a})))


def oracle_params(c):
    return O.make_params(c["D"], c["nx"], c["ny"], c["nz"], T_over_Tc=c["Tr"], kappa=c["kappa"],
                         nu_liquid=c["nu_l"], nu_vapour=c["nu_v"], rho_liquid=c["rho_l"],
                         rho_vapour=c["rho_v"], g=c["g"], bc=c["bc"], gamma_mode=c["gamma_mode"],
                         gamma_value=c["gamma_value"], **c.get("eos", PAPER_EOS))


def lbm_params(c):
    return lbm.lbm_default_params(
        lattice=lbm.LBM_D3Q27 if c["D"] == 3 else lbm.LBM_D2Q9, precision=c["precision"],
        nx=c["nx"], ny=c["ny"], nz=c["nz"], T_over_Tc=c["Tr"], kappa=c["kappa"],
        nu_liquid=c["nu_l"], nu_vapour=c["nu_v"], rho_liquid=c["rho_l"], rho_vapour=c["rho_v"],
        body_force=c["g"], bc=c["bc"], gamma_mode=c["gamma_mode"], gamma_value=c["gamma_value"],
        eos_fp64=c["eos_fp64"], **c.get("eos", PAPER_EOS))


def shape(c):
    return (c["nz"], c["ny"], c["nx"])


def drop_state(c, seed=11, perturb=0.01, W=5.0):
    """Oracle equilibrium of a drop (radius a quarter of the smallest side), then
    every population multiplied by (1 + eps), |eps| <= perturb: a non-equilibrium state."""
    D = c["D"]
    sh = shape(c)
    R = 0.25 * min(x for x in sh if x > 1)
    centre = (c["nx"] / 2 - 0.3, c["ny"] / 2 + 0.2, c["nz"] / 2 + 0.1)
    rho = I.drop(sh, centre, R, c["rho_l"], c["rho_v"], W, D=D)
    u = I.rng(seed).uniform(-0.02, 0.02, (D,) + sh)
    f = O.init_equilibrium(oracle_params(c), rho, u)
    return I.perturbed_populations(f, perturb, seed + 1)


def rel_err(f_gpu, f_orc, D):
    """e_i(r) = |f_gpu - f_orc| / (w_i rho(r)), the per-population error scaled by
    the population's natural size."""
    w = O.weights(D).reshape((-1, 1, 1, 1))
    rho = f_orc.sum(axis=0, keepdims=True)
    return np.abs(f_gpu - f_orc) / (w * rho)


def fp32_step_check(f_s, fg, fo, po, gamma_gpu, tol=2e-6, sample=None, seed=3):
    """Check one float32 GPU step fg against the oracle's fo from the same state f_s.

    Float32 resolves a population only to ~6e-8 of w_i rho.  Near equilibrium the
    higher-order part h = f - f^eq - s falls to ~1e-5 of w_i rho, so the entropic
    sums <ds|dh>, <dh|dh> built from it, and the gamma they give (Sec. 2.4), are
    float32 noise there; gamma multiplies h in the relaxation, so the population
    error that noise causes is (omega/2) |gamma_gpu - gamma_orc| |h| (reading A-9:
    no clipping, gamma noise is harmless where h is small).  Every population must
    therefore lie within tol w_i rho plus that term of the node it was streamed
    from (measured gamma_gpu, oracle gamma, omega and h), and where h is
    resolvable (max |h_i|/(w_i rho) >= 1e-3) gamma itself must agree to 2e-3.
    `sample` limits the conditioning check to that many seeded nodes.
    Returns (worst error over allowed bound, plain max error, nodes checked)."""
    D = po.D
    Q = O.Q_of(D)
    c = O.velocities(D)
    w = O.weights(D)
    e = rel_err(fg, fo, D)
    rho_d = fo.sum(axis=0)
    rho, u, spsi = O.aux_fields(po, f_s)
    F = O.force(po, rho, spsi)
    Phi = O.phi(po, rho, O.qflux(po, rho, u, F))
    cache = {}
    dims = [po.nx, po.ny, po.nz if D == 3 else 1]

    def node(z, y, x):
        key = (z, y, x)
        if key not in cache:
            f = f_s[:, z, y, x]
            om = O.omega(po, f.sum())
            res = O.collide_node(D, f, F[:, z, y, x], Phi[:, z, y, x], om)
            cache[key] = (res["h"], res["gamma"], om)
        return cache[key]

    worst = 0.0
    for i, z, y, x in np.argwhere(e > tol):
        src = [x - c[i, 0], y - c[i, 1], z - c[i, 2]]
        j = i
        for a in range(D):
            if src[a] < 0 or src[a] >= dims[a]:
                if po.bc[2 * a + (0 if src[a] < 0 else 1)] == 1:  # bounce-back: the node itself, reversed
                    src, j = [x, y, z], Q - 1 - i
                    break
                src[a] %= dims[a]
        sx, sy, sz = src
        h, g_orc, om = node(sz, sy, sx)
        allowed = tol * w[i] * rho_d[z, y, x] + 1.05 * 0.5 * om * abs(gamma_gpu[sz, sy, sx] - g_orc) * abs(h[j])
        worst = max(worst, abs(fg[i, z, y, x] - fo[i, z, y, x]) / allowed)
    # gamma where the entropic sums are resolvable
    shape = f_s.shape[1:]
    nodes = [(z, y, x) for z in range(shape[0]) for y in range(shape[1]) for x in range(shape[2])]
    if sample is not None and sample < len(nodes):
        pick = np.random.default_rng(seed).choice(len(nodes), sample, replace=False)
        nodes = [nodes[k] for k in pick]
    for z, y, x in nodes:
        h, g_orc, om = node(z, y, x)
        r = f_s[:, z, y, x].sum()
        if np.max(np.abs(h) / (w * r)) >= 1e-3:
            assert abs(gamma_gpu[z, y, x] - g_orc) <= 2e-3, ((z, y, x), gamma_gpu[z, y, x], g_orc)
    return worst, e.max(), len(nodes)
