"""ctypes binding of liblbm.so (C ABI in include/lbm.h), same names as the C calls.

Only argument marshalling lives here: every step of the lattice Boltzmann path
runs in the CUDA kernels of the library.  The library must have been built
(``python -m paper_2201_12404_gb300.build`` or ``__graft_entry__.build()``);
there is no fallback, and loading fails loudly when it is missing.

Arrays: numpy float64, field arrays shaped (nz, ny, nx) (nz = 1 in 2-D) or flat;
populations shaped (Q, nz, ny, nx) or flat, canonical order i = (cx+1) + 3(cy+1)
+ 9(cz+1).  Torch tensors on the host are accepted through ``.numpy()``.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# LBM_LIBRARY may name another build of the library (the bounds-checked one of
# build.build_bounds_checked); the default is the in-tree liblbm.so.
LIB_PATH = os.environ.get("LBM_LIBRARY") or os.path.join(_HERE, "liblbm.so")

(LBM_OK, LBM_ERR_INVALID_ARG, LBM_ERR_OOM, LBM_ERR_CUDA, LBM_ERR_UNSTABLE, LBM_ERR_TIMEOUT, LBM_ERR_STATE,
 LBM_ERR_BOUNDS) = range(8)
LBM_D2Q9, LBM_D3Q27 = 0, 1
LBM_FP64, LBM_FP32, LBM_FP16DEV = 0, 1, 2
LBM_BC_PERIODIC, LBM_BC_BOUNCEBACK = 0, 1
LBM_GAMMA_ENTROPIC, LBM_GAMMA_FIXED = 0, 1

# Device allocator hooks of lbm_params: void* (*)(size_t, void*) and void (*)(void*, void*).
DEV_ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
DEV_FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

STATUS_NAMES = {0: "LBM_OK", 1: "LBM_ERR_INVALID_ARG", 2: "LBM_ERR_OOM", 3: "LBM_ERR_CUDA",
                4: "LBM_ERR_UNSTABLE", 5: "LBM_ERR_TIMEOUT", 6: "LBM_ERR_STATE", 7: "LBM_ERR_BOUNDS"}


class lbm_params(ctypes.Structure):
    """Mirror of lbm_params in include/lbm.h."""

    _fields_ = [
        ("lattice", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("a", ctypes.c_double), ("b", ctypes.c_double), ("R", ctypes.c_double),
        ("T_over_Tc", ctypes.c_double), ("acentric", ctypes.c_double),
        ("kappa", ctypes.c_double),
        ("nu_liquid", ctypes.c_double), ("nu_vapour", ctypes.c_double),
        ("rho_liquid", ctypes.c_double), ("rho_vapour", ctypes.c_double),
        ("body_force", ctypes.c_double * 3),
        ("bc", ctypes.c_int32 * 6),
        ("gamma_mode", ctypes.c_int32), ("gamma_value", ctypes.c_double),
        ("eos_fp64", ctypes.c_int32),
        ("stream", ctypes.c_void_p),
        ("dev_alloc", DEV_ALLOC), ("dev_free", DEV_FREE), ("alloc_ctx", ctypes.c_void_p),
    ]


class LBMError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None
_lock = threading.Lock()
_dp = ctypes.POINTER(ctypes.c_double)


def load():
    """Load liblbm.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first "
                                  "(python -m paper_2201_12404_gb300.build)")
            L = ctypes.CDLL(LIB_PATH)
            H = ctypes.c_void_p
            P = ctypes.POINTER(lbm_params)
            st = ctypes.c_int
            sig = {
                "lbm_default_params": (st, [P]),
                "lbm_create_domain": (st, [P, ctypes.POINTER(H)]),
                "lbm_init_fields": (st, [H, _dp, _dp, _dp, _dp]),
                "lbm_step": (st, [H, ctypes.c_int64]),
                "lbm_synchronize": (st, [H]),
                "lbm_read_macroscopic": (st, [H, _dp, _dp, _dp, _dp]),
                "lbm_destroy": (st, [H]),
                "lbm_read_populations": (st, [H, _dp, ctypes.c_size_t]),
                "lbm_write_populations": (st, [H, _dp, ctypes.c_size_t]),
                "lbm_read_populations_window": (st, [H, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                                     _dp, ctypes.c_size_t]),
                "lbm_read_diag": (st, [H, _dp, _dp, _dp, _dp]),
                "lbm_record_gamma": (st, [H, ctypes.c_int]),
                "lbm_max_speed": (st, [H, _dp]),
                "lbm_init_drop_on_film": (st, [H, ctypes.POINTER(lbm_drop_on_film)]),
                "lbm_interface_width": (st, [H, _dp, _dp]),
                "lbm_crown_radius": (st, [H, ctypes.c_int32, _dp]),
                "lbm_read_relaxation": (st, [H, _dp]),
                "lbm_guard_count": (st, [H, ctypes.POINTER(ctypes.c_uint64)]),
                "lbm_footprint_bytes": (ctypes.c_size_t, [P]),
                "lbm_coexistence": (st, [P, _dp, _dp, _dp]),
                "lbm_psi_sign_changes": (st, [P, _dp, ctypes.POINTER(ctypes.c_int), _dp]),
                "lbm_set_timing": (st, [H, ctypes.c_int]),
                "lbm_kernel_times": (st, [H, _dp, ctypes.POINTER(ctypes.c_int64)]),
                "lbm_launch_count": (ctypes.c_int64, [H]),
                "lbm_last_error": (ctypes.c_char_p, [H]),
                "lbm_version": (ctypes.c_char_p, []),
                "lbm_step_noalloc": (st, [P, ctypes.c_void_p, ctypes.c_int64]),
                "lbm_noalloc_status": (st, []),
                "lbm_host_alloc": (st, [ctypes.c_size_t, ctypes.POINTER(ctypes.c_void_p)]),
                "lbm_host_free": (st, [ctypes.c_void_p]),
                "lbm_batch_create": (st, [ctypes.POINTER(H), ctypes.c_int32, ctypes.POINTER(H)]),
                "lbm_batch_step": (st, [H, ctypes.c_int64]),
                "lbm_batch_synchronize": (st, [H]),
                "lbm_batch_tune": (st, [H, ctypes.c_int32, ctypes.c_char_p]),
                "lbm_batch_info": (st, [H] + [ctypes.POINTER(ctypes.c_int32)] * 4),
                "lbm_batch_set_wait": (st, [H, ctypes.c_uint32, ctypes.c_int32]),
                "lbm_batch_destroy": (st, [H]),
                "lbm_batch_last_error": (ctypes.c_char_p, [H]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(_dp) if a is not None else None


def _check(status, handle=None):
    if status != LBM_OK:
        msg = load().lbm_last_error(handle).decode()
        raise LBMError(status, msg)


def lbm_default_params(**overrides) -> lbm_params:
    p = lbm_params()
    _check(load().lbm_default_params(ctypes.byref(p)))
    for k, v in overrides.items():
        if k in ("body_force", "bc"):
            arr = getattr(p, k)
            for i, x in enumerate(v):
                arr[i] = x
        else:
            setattr(p, k, v)
    return p


def _torch_alloc(nbytes, ctx):
    import torch
    try:
        return int(torch.cuda.caching_allocator_alloc(int(nbytes)))
    except Exception:  # out of memory: the library reports LBM_ERR_OOM
        return None


def _torch_free(ptr, ctx):
    import torch
    torch.cuda.caching_allocator_delete(int(ptr))


# module-level so that the C function pointers stay valid for every domain's lifetime
_TORCH_HOOKS = (DEV_ALLOC(_torch_alloc), DEV_FREE(_torch_free))


def use_torch_allocator(p: lbm_params) -> lbm_params:
    """Route the device buffers of domains created from p through PyTorch's caching
    allocator (torch.cuda.caching_allocator_alloc/delete) on the current device."""
    p.dev_alloc, p.dev_free = _TORCH_HOOKS
    p.alloc_ctx = None
    return p


def lbm_footprint_bytes(p: lbm_params) -> int:
    return int(load().lbm_footprint_bytes(ctypes.byref(p)))


def lbm_coexistence(p: lbm_params):
    rv, rl, ps = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(load().lbm_coexistence(ctypes.byref(p), ctypes.byref(rv), ctypes.byref(rl), ctypes.byref(ps)))
    return rv.value, rl.value, ps.value


def lbm_psi_sign_changes(p: lbm_params):
    """(densities where P - rho cs^2 changes sign, ascending; sign below the first)."""
    ch = (ctypes.c_double * 3)()
    n, s0 = ctypes.c_int(), ctypes.c_double()
    _check(load().lbm_psi_sign_changes(ctypes.byref(p), ch, ctypes.byref(n), ctypes.byref(s0)))
    return [ch[k] for k in range(n.value)], s0.value


def lbm_version() -> str:
    return load().lbm_version().decode()


def lbm_step_noalloc(p: lbm_params, populations_ptr: int, nsteps: int) -> None:
    """Allocation-free stepping of caller-owned device populations (see include/lbm.h)."""
    st = load().lbm_step_noalloc(ctypes.byref(p), ctypes.c_void_p(populations_ptr), int(nsteps))
    if st != LBM_OK:
        raise LBMError(st, "lbm_step_noalloc failed (invalid parameters, odd nsteps, misaligned populations, "
                           "a domain beyond the 16 MiB scratch, or a CUDA error)")


def lbm_noalloc_status() -> int:
    """Status of the last lbm_step_noalloc on the current device (after its stream completed)."""
    return int(load().lbm_noalloc_status())


class HostBuffer:
    """Page-locked host memory from lbm_host_alloc (huge-page backed where the kernel
    allows), for the calls that take host arrays.  `array(dtype, count, offset)`
    gives a numpy view; the views are valid until close()."""

    def __init__(self, nbytes: int):
        ptr = ctypes.c_void_p()
        st = load().lbm_host_alloc(int(nbytes), ctypes.byref(ptr))
        if st != LBM_OK:
            raise LBMError(st, f"lbm_host_alloc of {int(nbytes)} bytes failed")
        self.ptr, self.nbytes = int(ptr.value), int(nbytes)

    def array(self, dtype, count: int, offset: int = 0):
        import numpy as np
        dt = np.dtype(dtype)
        if offset < 0 or offset % dt.itemsize or offset + count * dt.itemsize > self.nbytes or not self.ptr:
            raise ValueError("view outside the host buffer")
        raw = (ctypes.c_char * (count * dt.itemsize)).from_address(self.ptr + offset)
        return np.frombuffer(raw, dtype=dt, count=count)

    def close(self):
        if self.ptr:
            st = load().lbm_host_free(ctypes.c_void_p(self.ptr))
            self.ptr = 0
            if st != LBM_OK:
                raise LBMError(st, "lbm_host_free failed")

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False


class lbm_drop_on_film(ctypes.Structure):
    _fields_ = [("radius", ctypes.c_double), ("film", ctypes.c_double), ("gap", ctypes.c_double),
                ("speed", ctypes.c_double), ("width", ctypes.c_double), ("noise", ctypes.c_double),
                ("seed", ctypes.c_uint64)]


class Domain:
    """One simulation domain (owns an lbm_handle)."""

    def __init__(self, params: lbm_params):
        L = load()
        self.params = params
        self.D = 3 if params.lattice == LBM_D3Q27 else 2
        self.Q = 27 if self.D == 3 else 9
        self.shape = (params.nz if self.D == 3 else 1, params.ny, params.nx)
        self.N = int(np.prod(self.shape))
        h = ctypes.c_void_p()
        _check(L.lbm_create_domain(ctypes.byref(params), ctypes.byref(h)), None)
        self.handle = h

    # -- lifetime
    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            load().lbm_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _c(self, status):
        _check(status, self.handle)

    def _field(self, a):
        a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
        if a.size != self.N:
            raise ValueError(f"field has {a.size} values, domain has {self.N}")
        return a

    # -- C calls
    def lbm_init_fields(self, rho, u):
        r = self._field(rho)
        comps = [self._field(u[a]) for a in range(self.D)]
        uz = comps[2] if self.D == 3 else None
        self._c(load().lbm_init_fields(self.handle, _ptr(r), _ptr(comps[0]), _ptr(comps[1]), _ptr(uz)))

    def lbm_init_fields_ptr(self, rho_ptr, ux_ptr, uy_ptr, uz_ptr=None):
        """Same call with raw host pointers (e.g. pinned torch tensors' data_ptr())."""
        c = lambda p: ctypes.cast(ctypes.c_void_p(p), _dp) if p else None
        self._c(load().lbm_init_fields(self.handle, c(rho_ptr), c(ux_ptr), c(uy_ptr), c(uz_ptr)))

    def lbm_init_drop_on_film(self, radius, film, gap, speed, width, noise=0.0, seed=0):
        g = lbm_drop_on_film(radius, film, gap, speed, width, noise, seed)
        self._c(load().lbm_init_drop_on_film(self.handle, ctypes.byref(g)))

    def lbm_step(self, nsteps: int):
        self._c(load().lbm_step(self.handle, int(nsteps)))

    def lbm_synchronize(self):
        self._c(load().lbm_synchronize(self.handle))

    def lbm_read_macroscopic(self):
        rho = np.empty(self.N)
        u = np.empty((self.D, self.N))
        self._c(load().lbm_read_macroscopic(self.handle, _ptr(rho), _ptr(u[0]), _ptr(u[1]),
                                            _ptr(u[2]) if self.D == 3 else None))
        return rho.reshape(self.shape), u.reshape((self.D,) + self.shape)

    def lbm_read_macroscopic_ptr(self, rho_ptr, ux_ptr, uy_ptr, uz_ptr=None):
        c = lambda p: ctypes.cast(ctypes.c_void_p(p), _dp) if p else None
        self._c(load().lbm_read_macroscopic(self.handle, c(rho_ptr), c(ux_ptr), c(uy_ptr), c(uz_ptr)))

    def lbm_read_populations(self):
        out = np.empty(self.Q * self.N)
        self._c(load().lbm_read_populations(self.handle, _ptr(out), out.size))
        return out.reshape((self.Q,) + self.shape)

    def lbm_read_populations_window(self, origin, extent):
        """Populations of the box origin + [0, extent) (x, y, z order; wraps across
        faces) as an array (Q, ez, ey, ex)."""
        o = (ctypes.c_int64 * 3)(*[int(v) for v in (tuple(origin) + (0, 0, 0))[:3]])
        e = (ctypes.c_int64 * 3)(*[int(v) for v in (tuple(extent) + (1, 1, 1))[:3]])
        out = np.empty(self.Q * e[0] * e[1] * e[2])
        self._c(load().lbm_read_populations_window(self.handle, o, e, _ptr(out), out.size))
        return out.reshape((self.Q, e[2], e[1], e[0]))

    def lbm_write_populations(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(-1)
        if f.size != self.Q * self.N:
            raise ValueError("populations must hold Q*N values")
        self._c(load().lbm_write_populations(self.handle, _ptr(f), f.size))

    def lbm_read_diag(self, with_gamma=False):
        m, mx = ctypes.c_double(), ctypes.c_double()
        mom = np.zeros(3)
        g = np.empty(self.N) if with_gamma else None
        self._c(load().lbm_read_diag(self.handle, ctypes.byref(m), _ptr(mom), ctypes.byref(mx), _ptr(g)))
        out = dict(mass=m.value, momentum=mom, max_u=mx.value)
        if with_gamma:
            out["gamma"] = g.reshape(self.shape)
        return out

    def lbm_max_speed(self) -> float:
        v = ctypes.c_double()
        self._c(load().lbm_max_speed(self.handle, ctypes.byref(v)))
        return v.value

    def lbm_interface_width(self):
        """(W, max |grad rho|) of the current state."""
        w, g = ctypes.c_double(), ctypes.c_double()
        self._c(load().lbm_interface_width(self.handle, ctypes.byref(w), ctypes.byref(g)))
        return w.value, g.value

    def lbm_crown_radius(self, layer: int) -> float:
        r = ctypes.c_double()
        self._c(load().lbm_crown_radius(self.handle, int(layer), ctypes.byref(r)))
        return r.value

    def lbm_read_relaxation(self):
        out = np.empty(self.N)
        self._c(load().lbm_read_relaxation(self.handle, _ptr(out)))
        return out.reshape(self.shape)

    def lbm_record_gamma(self, enable=True):
        self._c(load().lbm_record_gamma(self.handle, 1 if enable else 0))

    def lbm_guard_count(self) -> int:
        c = ctypes.c_uint64()
        self._c(load().lbm_guard_count(self.handle, ctypes.byref(c)))
        return int(c.value)

    def lbm_set_timing(self, enable=True):
        self._c(load().lbm_set_timing(self.handle, 1 if enable else 0))

    def lbm_kernel_times(self):
        ms = (ctypes.c_double * 2)()
        cnt = (ctypes.c_int64 * 2)()
        self._c(load().lbm_kernel_times(self.handle, ms, cnt))
        return [ms[0], ms[1]], [cnt[0], cnt[1]]

    def lbm_launch_count(self) -> int:
        return int(load().lbm_launch_count(self.handle))

    def lbm_last_error(self) -> str:
        return load().lbm_last_error(self.handle).decode()


class Batch:
    """Several D2Q9 domains advanced by one persistent launch (lbm_batch_*)."""

    def __init__(self, domains):
        L = load()
        self.domains = list(domains)
        arr = (ctypes.c_void_p * len(self.domains))(*[d.handle.value for d in self.domains])
        h = ctypes.c_void_p()
        st = L.lbm_batch_create(arr, len(self.domains), ctypes.byref(h))
        if st != LBM_OK:
            raise LBMError(st, L.lbm_batch_last_error(None).decode())
        self.handle = h

    def _c(self, st):
        if st != LBM_OK:
            raise LBMError(st, load().lbm_batch_last_error(self.handle).decode())

    def lbm_batch_step(self, nsteps: int):
        self._c(load().lbm_batch_step(self.handle, int(nsteps)))

    def lbm_batch_synchronize(self):
        self._c(load().lbm_batch_synchronize(self.handle))

    def lbm_batch_tune(self, trial_steps: int, cache_path=None):
        self._c(load().lbm_batch_tune(self.handle, int(trial_steps), cache_path.encode() if cache_path else None))

    def lbm_batch_set_wait(self, poll_limit: int, skip_arrival: bool = False):
        self._c(load().lbm_batch_set_wait(self.handle, int(poll_limit), 1 if skip_arrival else 0))

    def lbm_batch_info(self):
        v = [ctypes.c_int32() for _ in range(4)]
        self._c(load().lbm_batch_info(self.handle, *[ctypes.byref(x) for x in v]))
        return dict(block=(v[0].value, v[1].value), grid=v[2].value, graph=bool(v[3].value))

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            load().lbm_batch_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
