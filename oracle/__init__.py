"""FP64 CPU oracle of the entropic MRT two-phase lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the library under
``paper_2201_12404_gb300`` never does, and the oracle imports nothing from it.

The arithmetic lives in ``lbm_oracle.c`` (plain C, IEEE double, compiled with
``-ffp-contract=off``); the Peng-Robinson thermodynamics used by the checks
(Maxwell construction) lives in ``thermo.py``.  This module only compiles the C
file and marshals numpy arrays.

Population arrays are numpy float64 of shape (Q, nz, ny, nx) (nz = 1 in 2-D),
velocity index i = (cx+1) + 3(cy+1) + 9(cz+1).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liblbm_oracle.so")
_lock = threading.Lock()
_lib = None

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


class Params(ctypes.Structure):
    """Mirror of ``orc_params`` in lbm_oracle.c."""

    _fields_ = [
        ("D", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("a", ctypes.c_double), ("b", ctypes.c_double), ("R", ctypes.c_double),
        ("T_over_Tc", ctypes.c_double), ("acentric", ctypes.c_double),
        ("kappa", ctypes.c_double),
        ("nu_liquid", ctypes.c_double), ("nu_vapour", ctypes.c_double),
        ("rho_liquid", ctypes.c_double), ("rho_vapour", ctypes.c_double),
        ("g", ctypes.c_double * 3),
        ("bc", ctypes.c_int * 6),
        ("gamma_mode", ctypes.c_int), ("gamma_value", ctypes.c_double),
    ]


def make_params(D, nx, ny, nz=1, *, a=2.0 / 49.0, b=2.0 / 21.0, R=1.0, T_over_Tc=0.8,
                acentric=0.344, kappa=0.0, nu_liquid=0.1, nu_vapour=None, rho_liquid=1.0,
                rho_vapour=1.0, g=(0.0, 0.0, 0.0), bc=(0, 0, 0, 0, 0, 0), gamma_mode=0,
                gamma_value=2.0) -> Params:
    p = Params()
    p.D, p.nx, p.ny, p.nz = D, nx, ny, (nz if D == 3 else 1)
    p.a, p.b, p.R, p.T_over_Tc, p.acentric = a, b, R, T_over_Tc, acentric
    p.kappa = kappa
    p.nu_liquid = nu_liquid
    p.nu_vapour = nu_liquid if nu_vapour is None else nu_vapour
    p.rho_liquid, p.rho_vapour = rho_liquid, rho_vapour
    for k in range(3):
        p.g[k] = g[k]
    for k in range(6):
        p.bc[k] = bc[k]
    p.gamma_mode, p.gamma_value = gamma_mode, gamma_value
    return p


def build(force: bool = False) -> str:
    """Compile lbm_oracle.c into oracle/_build (gcc, -O2 -ffp-contract=off, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def load_library(path: str):
    """Open a compiled oracle library and declare its C signatures."""
    L = ctypes.CDLL(path)
    P = ctypes.POINTER(Params)
    sig = {
        "orc_Q": (ctypes.c_int, [ctypes.c_int]),
        "orc_velocities": (None, [ctypes.c_int, _ip]),
        "orc_psi1": (ctypes.c_double, [ctypes.c_int, ctypes.c_double, ctypes.c_double]),
        "orc_product_form": (None, [ctypes.c_int, ctypes.c_double, _dp, _dp, _dp]),
        "orc_weights": (None, [ctypes.c_int, _dp]),
        "orc_feq": (None, [ctypes.c_int, ctypes.c_double, _dp, _dp]),
        "orc_fstar": (None, [ctypes.c_int, ctypes.c_double, _dp, _dp, _dp, _dp]),
        "orc_Tc": (ctypes.c_double, [P]),
        "orc_pressure": (ctypes.c_double, [P, ctypes.c_double]),
        "orc_psi": (ctypes.c_double, [P, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]),
        "orc_omega": (ctypes.c_double, [P, ctypes.c_double]),
        "orc_central_moments": (None, [ctypes.c_int, _dp, _dp, _dp]),
        "orc_basis_rows": (None, [ctypes.c_int, _ip, _ip, _ip]),
        "orc_kbc_split": (ctypes.c_int, [ctypes.c_int, _dp, _dp, _dp, _dp, _dp]),
        "orc_collide_node": (ctypes.c_int, [ctypes.c_int, _dp, _dp, _dp, ctypes.c_double,
                                            ctypes.c_int, ctypes.c_double, _dp,
                                            ctypes.POINTER(ctypes.c_double),
                                            _dp, _dp, _dp, _dp, _dp]),
        "orc_aux_fields": (None, [P, _dp, _dp, _dp, _dp]),
        "orc_qflux": (None, [P, _dp, _dp, _dp, _dp]),
        "orc_force": (None, [P, _dp, _dp, _dp]),
        "orc_phi": (None, [P, _dp, _dp, _dp]),
        "orc_init_equilibrium": (None, [P, _dp, _dp, _dp]),
        "orc_init_physical": (None, [P, _dp, _dp, _dp]),
        "orc_macroscopic": (None, [P, _dp, _dp, _dp]),
        "orc_step": (ctypes.c_long, [P, _dp, _dp, ctypes.c_void_p]),
        "orc_run": (ctypes.c_long, [P, _dp, ctypes.c_long]),
        "orc_totals": (None, [P, _dp, ctypes.POINTER(ctypes.c_double), _dp]),
        "orc_num_threads": (ctypes.c_int, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load_library(build())
    return _lib


def Q_of(D: int) -> int:
    return 9 if D == 2 else 27


def _shape(p: Params):
    return (p.nz if p.D == 3 else 1, p.ny, p.nx)


def _f64(x):
    return np.ascontiguousarray(x, dtype=np.float64)


# ---- lattice -------------------------------------------------------------------

def velocities(D: int) -> np.ndarray:
    c = np.zeros(Q_of(D) * 3, dtype=np.int32)
    lib().orc_velocities(D, c)
    return c.reshape(-1, 3)


def weights(D: int) -> np.ndarray:
    w = np.zeros(Q_of(D))
    lib().orc_weights(D, w)
    return w


def psi1(c: int, xi: float, zeta: float) -> float:
    return lib().orc_psi1(c, xi, zeta)


def product_form(D, rho, xi, zeta):
    out = np.zeros(Q_of(D))
    lib().orc_product_form(D, rho, _f64(np.resize(xi, 3)), _f64(np.resize(zeta, 3)), out)
    return out


def feq(D, rho, u):
    out = np.zeros(Q_of(D))
    lib().orc_feq(D, rho, _f64(np.resize(u, 3)), out)
    return out


def fstar(D, rho, u, F, Phi):
    out = np.zeros(Q_of(D))
    lib().orc_fstar(D, rho, _f64(np.resize(u, 3)), _f64(np.resize(F, 3)), _f64(np.resize(Phi, 3)), out)
    return out


# ---- thermodynamics ---------------------------------------------------------------

def Tc(p: Params) -> float:
    return lib().orc_Tc(ctypes.byref(p))


def pressure(p: Params, rho: float) -> float:
    return lib().orc_pressure(ctypes.byref(p), rho)


def psi(p: Params, rho: float):
    s = ctypes.c_double()
    v = lib().orc_psi(ctypes.byref(p), rho, ctypes.byref(s))
    return v, s.value


def omega(p: Params, rho: float) -> float:
    return lib().orc_omega(ctypes.byref(p), rho)


# ---- moments and collision ----------------------------------------------------------

def basis_rows(D):
    Q = Q_of(D)
    kind = np.zeros(Q, np.int32)
    e = np.zeros(3 * Q, np.int32)
    part = np.zeros(Q, np.int32)
    lib().orc_basis_rows(D, kind, e, part)
    return kind, e.reshape(Q, 3), part


def central_moments(D, u, f):
    a = np.zeros(Q_of(D))
    lib().orc_central_moments(D, _f64(np.resize(u, 3)), _f64(f), a)
    return a


def kbc_split(D, u, f):
    Q = Q_of(D)
    k, s, h = np.zeros(Q), np.zeros(Q), np.zeros(Q)
    rc = lib().orc_kbc_split(D, _f64(np.resize(u, 3)), _f64(f), k, s, h)
    if rc != 0:
        raise RuntimeError("singular moment basis")
    return k, s, h


def collide_node(D, f, F, Phi, omega_, gamma_mode=0, gamma_value=2.0):
    """One node of Eq. (LBGK) with the entropic mirror state.  Returns a dict."""
    Q = Q_of(D)
    fp, feq_, fs, k, s, h = (np.zeros(Q) for _ in range(6))
    g = ctypes.c_double()
    guard = lib().orc_collide_node(D, _f64(f), _f64(np.resize(F, 3)), _f64(np.resize(Phi, 3)),
                                   omega_, gamma_mode, gamma_value, fp, ctypes.byref(g),
                                   feq_, fs, k, s, h)
    if guard < 0:
        raise RuntimeError("singular moment basis")
    return dict(fp=fp, gamma=g.value, feq=feq_, fstar=fs, k=k, s=s, h=h, guard=guard)


# ---- fields ---------------------------------------------------------------------------

def aux_fields(p: Params, f):
    """(rho, bare u, s psi) of a state."""
    D = p.D
    sh = _shape(p)
    rho = np.zeros(sh)
    u = np.zeros((D,) + sh)
    spsi = np.zeros(sh)
    lib().orc_aux_fields(ctypes.byref(p), _f64(f), rho, u, spsi)
    return rho, u, spsi


def qflux(p: Params, rho, u, F):
    """q_a = rho v_a^3, v = u + F/(2 rho), the flux Phi differentiates."""
    q = np.zeros((p.D,) + _shape(p))
    lib().orc_qflux(ctypes.byref(p), _f64(rho), _f64(u), _f64(F), q)
    return q


def force(p: Params, rho, spsi):
    F = np.zeros((p.D,) + _shape(p))
    lib().orc_force(ctypes.byref(p), _f64(rho), _f64(spsi), F)
    return F


def phi(p: Params, rho, q):
    P = np.zeros((p.D,) + _shape(p))
    lib().orc_phi(ctypes.byref(p), _f64(rho), _f64(q), P)
    return P


def init_equilibrium(p: Params, rho0, u0):
    f = np.zeros((Q_of(p.D),) + _shape(p))
    lib().orc_init_equilibrium(ctypes.byref(p), _f64(rho0), _f64(u0), f)
    return f


def init_physical(p: Params, rho0, u0):
    """Equilibrium whose reported velocity u + F/(2 rho) is u0 (the library's lbm_init_fields)."""
    f = np.zeros((Q_of(p.D),) + _shape(p))
    lib().orc_init_physical(ctypes.byref(p), _f64(rho0), _f64(u0), f)
    return f


def macroscopic(p: Params, f):
    rho = np.zeros(_shape(p))
    u = np.zeros((p.D,) + _shape(p))
    lib().orc_macroscopic(ctypes.byref(p), _f64(f), rho, u)
    return rho, u


def step(p: Params, f, with_gamma=False):
    """One step; returns (f_next, guards[, gamma_field])."""
    f = _f64(f)
    out = np.zeros_like(f)
    gam = np.zeros(_shape(p)) if with_gamma else None
    g = lib().orc_step(ctypes.byref(p), f, out, gam.ctypes.data if with_gamma else None)
    if g < 0:
        raise RuntimeError("oracle step failed")
    return (out, g, gam) if with_gamma else (out, g)


def run(p: Params, f, nsteps: int):
    """nsteps steps in place on a copy; returns (f, guards)."""
    f = np.array(f, dtype=np.float64, copy=True, order="C")
    g = lib().orc_run(ctypes.byref(p), f, nsteps)
    if g < 0:
        raise RuntimeError("oracle run failed")
    return f, g


def totals(p: Params, f):
    m = ctypes.c_double()
    j = np.zeros(3)
    lib().orc_totals(ctypes.byref(p), _f64(f), ctypes.byref(m), j)
    return m.value, j


def num_threads() -> int:
    """OpenMP threads the oracle's step uses."""
    return int(lib().orc_num_threads())
