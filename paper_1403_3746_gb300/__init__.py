"""Python binding of the D2V16-FFT-TLB CUDA library (C ABI in include/lbm_d2v16.h).

Argument marshalling only: every step of the method runs in the library's CUDA kernels.
The shared library is built in-tree by `paper_1403_3746_gb300.build.build()`; importing
this module does not build it, and every call fails loudly if it is missing.

Host arrays are numpy float64 (C-contiguous, shape (ny, nx) for fields and (16, ny, nx)
for the distributions). Device arrays are torch CUDA float64 tensors of the same shapes.
"""
import ctypes
import os

import numpy as np

from .build import LIB as LIB_PATH

LBM_OK = 0
LBM_FP64 = 0
LBM_MIXED = 1
LBM_MIXED_RHO64 = 2
LBM_FLAG_NO_ADVECTION = 1
LBM_FLAG_NO_COLLISION = 2
LBM_FLAG_NO_FORCE = 4
LBM_FLAG_EULER = 8
LBM_FLAG_ISOTHERMAL = 16
KERNELS = {"col": 0, "macro": 1, "flux": 2, "update": 3, "rho64": 4}
LBM_COL_DIRECT = 0
LBM_COL_TMA = 1
LBM_COL_LOOKAHEAD = 2
LBM_COL_TMA1 = 3
LBM_FAULT_NONE = 0
LBM_FAULT_STARVE_COPIES = 1
LBM_FAULT_WITHHOLD_COMPLETION = 2
LBM_BATCH_GRAPH = 0
LBM_BATCH_PERSISTENT = 1
LBM_ERR_TIMEOUT = -5

_lib = None


class LbmError(RuntimeError):
    def __init__(self, msg, code=None):
        super().__init__(msg)
        self.code = code


class lbm_params(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double), ("dt", ctypes.c_double), ("dx", ctypes.c_double),
                ("dy", ctypes.c_double), ("K", ctypes.c_double), ("H", ctypes.c_double),
                ("q", ctypes.c_double), ("zeta", ctypes.c_double), ("b", ctypes.c_double),
                ("eta0", ctypes.c_double), ("win_alpha", ctypes.c_double), ("win_p", ctypes.c_double),
                ("precision", ctypes.c_int), ("flags", ctypes.c_int), ("T_iso", ctypes.c_double),
                ("keff_terms", ctypes.c_int), ("reserved", ctypes.c_int),
                ("filter_alpha", ctypes.c_double), ("filter_p", ctypes.c_double)]


_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_SIGS = {
    "lbm_default_params": (None, [ctypes.POINTER(lbm_params)]),
    "lbm_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(lbm_params), _P,
                                  ctypes.POINTER(_P)]),
    "lbm_init": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "lbm_init_device": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "lbm_step": (ctypes.c_int, [_P, ctypes.c_int]),
    "lbm_moments": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "lbm_moments_device": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "lbm_get_f": (ctypes.c_int, [_P, _P]),
    "lbm_set_f": (ctypes.c_int, [_P, _P]),
    "lbm_diagnostics": (ctypes.c_int, [_P, _D]),
    "lbm_synchronize": (ctypes.c_int, [_P]),
    "lbm_destroy": (None, [_P]),
    "lbm_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "lbm_last_error": (ctypes.c_char_p, []),
    "lbm_maxwell": (ctypes.c_int, [ctypes.c_double, _D, _D]),
    "lbm_timing": (ctypes.c_int, [_P, ctypes.c_int]),
    "lbm_timing_read": (ctypes.c_int, [_P, ctypes.c_int, _D, ctypes.POINTER(ctypes.c_longlong)]),
    "lbm_device_bytes": (ctypes.c_size_t, [_P]),
    "lbm_diagnostics_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                               _P, _P, _P, _P, _P, _D]),
    "lbm_batch_create": (ctypes.c_int, [ctypes.c_int, _P, _P, ctypes.POINTER(lbm_params), _P,
                                        ctypes.POINTER(_P)]),
    "lbm_batch_count": (ctypes.c_int, [_P]),
    "lbm_batch_init": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, _P]),
    "lbm_batch_step": (ctypes.c_int, [_P, ctypes.c_int]),
    "lbm_batch_moments": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, _P]),
    "lbm_batch_get_f": (ctypes.c_int, [_P, ctypes.c_int, _P]),
    "lbm_batch_diagnostics": (ctypes.c_int, [_P, ctypes.c_int, _D]),
    "lbm_batch_destroy": (None, [_P]),
    "lbm_geometry": (ctypes.c_int, [_P, _P]),
    "lbm_set_geometry": (ctypes.c_int, [_P, _P]),
    "lbm_structure_factor": (ctypes.c_int, [_P, ctypes.c_int, _P, _P]),
    "lbm_batch_structure_factor": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, _P]),
    "lbm_autotune": (ctypes.c_int, [_P, _P, _P]),
    "lbm_batch_autotune": (ctypes.c_int, [_P]),
    "lbm_batch_geometry": (ctypes.c_int, [_P, ctypes.c_int, _P]),
    "lbm_launch_plan": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _P]),
    "lbm_state_bytes": (ctypes.c_size_t, [ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "lbm_pass_kinds": (ctypes.c_int, [_P, _P]),
    "lbm_batch_set_form": (ctypes.c_int, [_P, ctypes.c_int]),
    "lbm_diagnostics_begin": (ctypes.c_int, [_P]),
    "lbm_diagnostics_end": (ctypes.c_int, [_P, _D]),
    "lbm_batch_form": (ctypes.c_int, [_P]),
    "lbm_batch_synchronize": (ctypes.c_int, [_P]),
    "lbm_batch_fault_inject": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_longlong]),
    "lbm_set_pass_kinds": (ctypes.c_int, [_P, _P]),
    "lbm_fault_inject": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_longlong]),
    "lbm_params_hash": (ctypes.c_ulonglong, [ctypes.POINTER(lbm_params)]),
    "lbm_get_state": (ctypes.c_int, [_P, _P, ctypes.c_size_t]),
    "lbm_set_state": (ctypes.c_int, [_P, _P, ctypes.c_size_t]),
    "lbm_batch_get_state": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_size_t]),
    "lbm_batch_set_state": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_size_t]),
}


def lib():
    """The loaded shared library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise LbmError(f"CUDA library not built: {LIB_PATH} is missing "
                           "(run paper_1403_3746_gb300.build.build())")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc):
    if rc != LBM_OK:
        L = lib()
        raise LbmError(f"{L.lbm_strerror(rc).decode()} ({rc}): {L.lbm_last_error().decode()}", rc)


def default_params(**kw):
    """lbm_params with the library defaults (phase-separation set), overridden by kw."""
    p = lbm_params()
    lib().lbm_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def maxwell(T):
    """Coexisting (rho_liquid, rho_vapour) of the van der Waals fluid at temperature T."""
    rl, rv = ctypes.c_double(), ctypes.c_double()
    _check(lib().lbm_maxwell(float(T), ctypes.byref(rl), ctypes.byref(rv)))
    return rl.value, rv.value


def diagnostics_noalloc(params, rho, ux, uy, T, stream=None):
    """lbm_diagnostics_noalloc: mass, px, py, energy, umax of moment fields held in CUDA
    float64 tensors (ny, nx), for callers that cannot allocate device memory; the library
    uses its built-in scratch array (nx * ny <= 2^20). The grid spacings, K, window and k_eff
    series length come from `params`. Not for a stream under graph capture (LbmError)."""
    ny, nx = tuple(rho.shape)
    ps = [_dev_ptr(a, (ny, nx)) for a in (rho, ux, uy, T)]
    out = (ctypes.c_double * 5)()
    s = ctypes.c_void_p(stream) if isinstance(stream, int) else (stream or ctypes.c_void_p())
    _check(lib().lbm_diagnostics_noalloc(nx, ny, params.dx, params.dy, params.K, params.win_alpha,
                                         params.win_p, params.keff_terms, *ps, s, out))
    return dict(zip(("mass", "px", "py", "energy", "umax"), list(out)))


def state_bytes(nx, ny, precision=LBM_FP64):
    """lbm_state_bytes: size of the checkpoint blob of an nx x ny simulation (0 for bad sizes)."""
    return int(lib().lbm_state_bytes(int(nx), int(ny), int(precision)))


def params_hash(params):
    """lbm_params_hash: the 64-bit parameter hash a checkpoint blob carries."""
    return int(lib().lbm_params_hash(ctypes.byref(params)))


def _blob_in(blob):
    b = bytes(blob)
    return ctypes.create_string_buffer(b, len(b)), len(b)


PLAN_KEYS = ("col_width", "col_threads", "col_smem", "macro_rows", "macro_threads", "macro_smem", "macro_serial",
             "update_rows", "update_smem", "update_ax", "rowd_rows", "rowd_threads", "rowd_smem",
             "pass_thread_cap", "macro_thread_cap", "cta_smem_cap", "update_ctas_per_row", "col_ctas_per_cluster")


def launch_plan(nx, ny, precision=LBM_FP64):
    """lbm_launch_plan: the default launch shapes of an nx x ny grid and what each pass needs,
    computed on the host (a dict keyed by PLAN_KEYS)."""
    out = (ctypes.c_int * 18)()
    _check(lib().lbm_launch_plan(int(nx), int(ny), int(precision), out))
    return dict(zip(PLAN_KEYS, list(out)))


def _host_out(out, shape):
    """Four writable host arrays for a moments call: new ones, or the caller's after a check."""
    if out is None:
        return [np.empty(shape) for _ in range(4)]
    out = list(out)
    if len(out) != 4 or not all(isinstance(a, np.ndarray) and a.dtype == np.float64 and a.shape == tuple(shape)
                                and a.flags.c_contiguous and a.flags.writeable for a in out):
        raise ValueError(f"out: four writable C-contiguous float64 arrays of shape {tuple(shape)}")
    return out


def _host(a, shape):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.shape != shape:
        raise ValueError(f"expected shape {shape}, got {a.shape}")
    return a


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _dev_ptr(t, shape):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("device arrays must be contiguous float64 CUDA tensors")
    if tuple(t.shape) != shape:
        raise ValueError(f"expected shape {shape}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


class Simulation:
    """One D2V16 simulation on an nx x ny periodic grid (lbm_create .. lbm_destroy)."""

    def __init__(self, nx, ny, params=None, stream=None):
        self.nx, self.ny = int(nx), int(ny)
        self.params = params if params is not None else default_params()
        h = ctypes.c_void_p()
        s = ctypes.c_void_p(stream) if isinstance(stream, int) else (stream or ctypes.c_void_p())
        _check(lib().lbm_create(self.nx, self.ny, ctypes.byref(self.params), s, ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().lbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def shape(self):
        return (self.ny, self.nx)

    def init(self, rho, ux, uy, T):
        """f := f^eq(rho, u, T); host numpy arrays or CUDA float64 tensors of shape (ny, nx)."""
        if type(rho).__module__.startswith("torch"):
            ps = [_dev_ptr(a, self.shape) for a in (rho, ux, uy, T)]
            _check(lib().lbm_init_device(self._h, *ps))
        else:
            arrs = [_host(a, self.shape) for a in (rho, ux, uy, T)]
            _check(lib().lbm_init(self._h, *[_ptr(a) for a in arrs]))

    def step(self, n=1):
        _check(lib().lbm_step(self._h, int(n)))

    def synchronize(self):
        _check(lib().lbm_synchronize(self._h))

    def moments(self, out=None):
        """(rho, u_x, u_y, T) as host numpy arrays; `out`: four C-contiguous float64 arrays of
        shape (ny, nx) to fill instead (pinned ones take the fast copy path)."""
        out = _host_out(out, self.shape)
        _check(lib().lbm_moments(self._h, *[_ptr(a) for a in out]))
        return tuple(out)

    def moments_device(self, rho, ux, uy, T):
        ps = [_dev_ptr(a, self.shape) if a is not None else ctypes.c_void_p() for a in (rho, ux, uy, T)]
        _check(lib().lbm_moments_device(self._h, *ps))

    def get_f(self):
        f = np.empty((16,) + self.shape)
        _check(lib().lbm_get_f(self._h, _ptr(f)))
        return f

    def set_f(self, f):
        f = _host(f, (16,) + self.shape)
        _check(lib().lbm_set_f(self._h, _ptr(f)))

    def get_state(self):
        """Checkpoint blob (bytes): distributions, moments, step counter, parameter hash."""
        n = state_bytes(self.nx, self.ny, self.params.precision)
        buf = ctypes.create_string_buffer(n)
        _check(lib().lbm_get_state(self._h, buf, n))
        return buf.raw

    def set_state(self, blob):
        """Resume from a blob of get_state (same size and parameters)."""
        buf, n = _blob_in(blob)
        _check(lib().lbm_set_state(self._h, buf, n))

    def diagnostics(self):
        """dict(mass, px, py, energy, umax, steps)."""
        out = (ctypes.c_double * 6)()
        _check(lib().lbm_diagnostics(self._h, out))
        return dict(zip(("mass", "px", "py", "energy", "umax", "steps"), list(out)))

    def diagnostics_begin(self):
        """Issue the diagnostics of the current state without waiting (lbm_diagnostics_begin)."""
        _check(lib().lbm_diagnostics_begin(self._h))

    def diagnostics_end(self):
        """Wait for the oldest pending request and return its dict (lbm_diagnostics_end)."""
        out = (ctypes.c_double * 6)()
        _check(lib().lbm_diagnostics_end(self._h, out))
        return dict(zip(("mass", "px", "py", "energy", "umax", "steps"), list(out)))

    def timing(self, enable=True):
        _check(lib().lbm_timing(self._h, 1 if enable else 0))

    def timing_read(self, kernel):
        ms, cnt = ctypes.c_double(), ctypes.c_longlong()
        _check(lib().lbm_timing_read(self._h, KERNELS.get(kernel, kernel), ctypes.byref(ms), ctypes.byref(cnt)))
        return ms.value, cnt.value

    def device_bytes(self):
        return int(lib().lbm_device_bytes(self._h))

    def structure_factor(self, nbins):
        """(S, count): circularly averaged structure factor of the density, nbins shells."""
        S, cnt = np.empty(nbins), np.empty(nbins)
        _check(lib().lbm_structure_factor(self._h, int(nbins), _ptr(S), _ptr(cnt)))
        return S, cnt

    def geometry(self):
        """(column tile width, rows per CTA of the macro pass, rows per CTA of the update pass,
        flux column tile width)."""
        g = (ctypes.c_int * 4)()
        _check(lib().lbm_geometry(self._h, ctypes.cast(g, _P)))
        return tuple(g)

    def set_geometry(self, geometry):
        g = (ctypes.c_int * 4)(*[int(v) for v in geometry])
        _check(lib().lbm_set_geometry(self._h, ctypes.cast(g, _P)))

    def pass_kinds(self):
        """(column pass kind, flux column pass kind, update CTAs per row): each column kind
        LBM_COL_DIRECT, LBM_COL_TMA, LBM_COL_LOOKAHEAD or LBM_COL_TMA1; 1, 2 or 4."""
        k = (ctypes.c_int * 3)()
        _check(lib().lbm_pass_kinds(self._h, ctypes.cast(k, _P)))
        return tuple(k)

    def set_pass_kinds(self, kinds):
        """kinds: (column, flux) or (column, flux, update CTAs per row; default: unchanged)."""
        kinds = list(kinds)
        if len(kinds) == 2:
            kinds.append(self.pass_kinds()[2])
        k = (ctypes.c_int * 3)(*[int(v) for v in kinds])
        _check(lib().lbm_set_pass_kinds(self._h, ctypes.cast(k, _P)))

    def fault_inject(self, what, wait_cycles=0):
        """Test hook: LBM_FAULT_STARVE_COPIES makes the TMA column pass's bounded wait run out."""
        _check(lib().lbm_fault_inject(self._h, int(what), int(wait_cycles)))

    def autotune(self):
        """Times the launch-shape candidates on this simulation and keeps the fastest;
        returns (geometry, ms per pass)."""
        g = (ctypes.c_int * 4)()
        ms = (ctypes.c_double * 4)()
        _check(lib().lbm_autotune(self._h, ctypes.cast(g, _P), ctypes.cast(ms, _P)))
        return tuple(g), tuple(ms)


class Batch:
    """Independent simulations advanced together (lbm_batch_create .. lbm_batch_destroy).
    sizes: list of (nx, ny), one per instance; all share `params`."""

    def __init__(self, sizes, params=None, stream=None):
        self.sizes = [(int(nx), int(ny)) for nx, ny in sizes]
        self.params = params if params is not None else default_params()
        cnt = len(self.sizes)
        nxs = (ctypes.c_int * max(cnt, 1))(*[s[0] for s in self.sizes])
        nys = (ctypes.c_int * max(cnt, 1))(*[s[1] for s in self.sizes])
        h = ctypes.c_void_p()
        s = ctypes.c_void_p(stream) if isinstance(stream, int) else (stream or ctypes.c_void_p())
        _check(lib().lbm_batch_create(cnt, ctypes.cast(nxs, _P), ctypes.cast(nys, _P),
                                      ctypes.byref(self.params), s, ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().lbm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __len__(self):
        return int(lib().lbm_batch_count(self._h))

    def _shape(self, k):
        nx, ny = self.sizes[k]
        return (ny, nx)

    def init(self, k, rho, ux, uy, T):
        arrs = [_host(a, self._shape(k)) for a in (rho, ux, uy, T)]
        _check(lib().lbm_batch_init(self._h, int(k), *[_ptr(a) for a in arrs]))

    def step(self, n=1):
        _check(lib().lbm_batch_step(self._h, int(n)))

    def moments(self, k, out=None):
        out = _host_out(out, self._shape(k))
        _check(lib().lbm_batch_moments(self._h, int(k), *[_ptr(a) for a in out]))
        return tuple(out)

    def get_f(self, k):
        f = np.empty((16,) + self._shape(k))
        _check(lib().lbm_batch_get_f(self._h, int(k), _ptr(f)))
        return f

    def get_state(self, k):
        nx, ny = self.sizes[k]
        n = state_bytes(nx, ny, self.params.precision)
        buf = ctypes.create_string_buffer(n)
        _check(lib().lbm_batch_get_state(self._h, int(k), buf, n))
        return buf.raw

    def set_state(self, k, blob):
        buf, n = _blob_in(blob)
        _check(lib().lbm_batch_set_state(self._h, int(k), buf, n))

    def diagnostics(self, k):
        out = (ctypes.c_double * 6)()
        _check(lib().lbm_batch_diagnostics(self._h, int(k), out))
        return dict(zip(("mass", "px", "py", "energy", "umax", "steps"), list(out)))

    def autotune(self):
        _check(lib().lbm_batch_autotune(self._h))

    def set_form(self, form):
        """LBM_BATCH_GRAPH or LBM_BATCH_PERSISTENT (one persistent kernel launch per step)."""
        _check(lib().lbm_batch_set_form(self._h, int(form)))

    def form(self):
        return int(lib().lbm_batch_form(self._h))

    def synchronize(self):
        _check(lib().lbm_batch_synchronize(self._h))

    def fault_inject(self, what, wait_cycles=0):
        """Test hook: LBM_FAULT_WITHHOLD_COMPLETION makes the persistent kernel's waits run out."""
        _check(lib().lbm_batch_fault_inject(self._h, int(what), int(wait_cycles)))

    def structure_factor(self, k, nbins):
        S, cnt = np.empty(nbins), np.empty(nbins)
        _check(lib().lbm_batch_structure_factor(self._h, int(k), int(nbins), _ptr(S), _ptr(cnt)))
        return S, cnt

    def geometry(self, k):
        g = (ctypes.c_int * 4)()
        _check(lib().lbm_batch_geometry(self._h, int(k), ctypes.cast(g, _P)))
        return tuple(g)
