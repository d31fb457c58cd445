"""Python binding of the tomo C ABI (``include/tomo.h``): argument marshalling only.

Every computation runs in ``libtomo.so`` (CUDA, sm_103a).  Arrays may be torch tensors (on
the grid's CUDA device or on the CPU) or numpy arrays; their data pointers are handed to the
library, which stages host arrays itself.  If the library is not built this module raises
on load: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# TOMO_LIB=checked selects the bounds-checked build (tomo_check_report)
LIB_PATH = os.path.join(_HERE, "_lib", "libtomo_checked.so" if os.environ.get("TOMO_LIB") ==
                        "checked" else "libtomo.so")

FP64, FP32 = 0, 1
PRECOND_MG, PRECOND_JACOBI = 0, 1
STATUS = {0: "TOMO_OK", 1: "TOMO_EINVAL", 2: "TOMO_ENOMEM", 3: "TOMO_ENOCONV", 4: "TOMO_ENAN",
          5: "TOMO_ETIMEOUT", 6: "TOMO_ECUDA", 7: "TOMO_EBUSY"}


class TomoError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class GridDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("h", ctypes.c_double), ("E0", ctypes.c_double), ("Emin", ctypes.c_double),
                ("nu", ctypes.c_double), ("penal", ctypes.c_double), ("rmin", ctypes.c_double),
                ("fixed_dof", ctypes.POINTER(ctypes.c_uint8)),
                ("f", ctypes.POINTER(ctypes.c_double)),
                ("precision", ctypes.c_int32), ("precond", ctypes.c_int32),
                ("rtol", ctypes.c_double), ("maxit", ctypes.c_int32),
                ("mg_levels", ctypes.c_int32), ("smoother_degree", ctypes.c_int32),
                ("coarse_degree", ctypes.c_int32),
                ("cheb_ratio", ctypes.c_double), ("cheb_lmax", ctypes.c_double),
                ("rr_every", ctypes.c_int32),
                ("stream", ctypes.c_void_p)]


class TuneResult(ctypes.Structure):
    _fields_ = [("fine_degree", ctypes.c_int32), ("coarse_degree", ctypes.c_int32),
                ("iters", ctypes.c_int32), ("status", ctypes.c_int32), ("ms", ctypes.c_double),
                ("lam", ctypes.c_double), ("w_levels", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("ratio", ctypes.c_double)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("rel_res", ctypes.c_double),
                ("status", ctypes.c_int32), ("mg_levels", ctypes.c_int32)]


class Result(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_int64), ("status", ctypes.c_int32),
                ("compliance", ctypes.c_double), ("info", SolveInfo),
                ("queue_ms", ctypes.c_double), ("run_ms", ctypes.c_double),
                ("message_len", ctypes.c_int32), ("message", ctypes.c_char * 256)]


class BatchTuneResult(ctypes.Structure):
    _fields_ = [("tile_rows", ctypes.c_int32), ("waves", ctypes.c_int32),
                ("status", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("ms", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("grids_created", ctypes.c_int64), ("evictions", ctypes.c_int64),
                ("resident_bytes", ctypes.c_uint64), ("peak_bytes", ctypes.c_uint64),
                ("resident_grids", ctypes.c_int32), ("queued", ctypes.c_int32),
                ("batches", ctypes.c_int64)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libtomo.so is not built ({LIB_PATH}); run "
                          "`python -c 'import __graft_entry__ as g; g.build()'` first")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    G = ctypes.c_void_p
    st = ctypes.c_int
    sig = {
        "tomo_default_desc": (None, [ctypes.POINTER(GridDesc)]),
        "tomo_create_grid": (st, [ctypes.POINTER(GridDesc), ctypes.POINTER(ctypes.c_void_p)]),
        "tomo_destroy_grid": (st, [G]),
        "tomo_set_stream": (st, [G, P]),
        "tomo_set_warm_start": (st, [G, ctypes.c_int32]),
        "tomo_set_smoother": (st, [G, ctypes.c_int32, ctypes.c_int32, ctypes.c_double]),
        "tomo_get_smoother": (st, [G, ctypes.POINTER(ctypes.c_int32),
                                   ctypes.POINTER(ctypes.c_int32),
                                   ctypes.POINTER(ctypes.c_double)]),
        "tomo_set_smoother_bound": (st, [G, ctypes.c_double]),
        "tomo_set_cycle": (st, [G, ctypes.c_uint32]),
        "tomo_set_coarse_tail": (st, [G, ctypes.c_int32]),
        "tomo_get_coarse_tail": (st, [G, ctypes.POINTER(ctypes.c_int32)]),
        "tomo_get_cycle": (st, [G, ctypes.POINTER(ctypes.c_uint32)]),
        "tomo_get_smoother_bound": (st, [G, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_int64)]),
        "tomo_autotune_smoother": (st, [G, P, P, ctypes.c_int32, ctypes.c_int32, P,
                                        ctypes.POINTER(ctypes.c_int32)]),
        "tomo_autotune_smoother_d": (st, [G, P, P, ctypes.c_int32, ctypes.c_int32, P,
                                          ctypes.POINTER(ctypes.c_int32)]),
        "tomo_autotune_smoother_multi": (st, [G, P, ctypes.c_int32, P, ctypes.c_int32,
                                              ctypes.c_int32, P,
                                              ctypes.POINTER(ctypes.c_int32)]),
        "tomo_autotune_smoother_multi_d": (st, [G, P, ctypes.c_int32, P, ctypes.c_int32,
                                                ctypes.c_int32, P,
                                                ctypes.POINTER(ctypes.c_int32)]),
        "tomo_server_create": (st, [ctypes.c_int32, ctypes.c_uint64,
                                    ctypes.POINTER(ctypes.c_void_p)]),
        "tomo_server_submit": (st, [P, ctypes.POINTER(GridDesc), ctypes.c_int64, P, P, P,
                                    ctypes.POINTER(ctypes.c_int64)]),
        "tomo_server_submit_optimize": (st, [P, ctypes.POINTER(GridDesc), ctypes.c_int64, P,
                                             ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                             P, ctypes.POINTER(ctypes.c_int64)]),
        "tomo_server_wait": (st, [P, ctypes.c_int64, ctypes.POINTER(Result)]),
        "tomo_server_get_stats": (st, [P, ctypes.POINTER(ServerStats)]),
        "tomo_server_set_batching": (st, [P, ctypes.c_int32, ctypes.c_int32]),
        "tomo_server_destroy": (st, [P]),
        "tomo_server_last_error": (ctypes.c_char_p, [P]),
        "tomo_grid_device_bytes": (st, [G, ctypes.POINTER(ctypes.c_size_t)]),
        "tomo_estimate_device_bytes": (st, [ctypes.POINTER(GridDesc),
                                            ctypes.POINTER(ctypes.c_size_t)]),
        "tomo_batch_create": (st, [ctypes.c_int32, ctypes.POINTER(ctypes.c_void_p)]),
        "tomo_batch_append": (st, [P, G]),
        "tomo_batch_size": (st, [P, ctypes.POINTER(ctypes.c_int32)]),
        "tomo_batch_set_lockstep": (st, [P, ctypes.c_int32]),
        "tomo_batch_lockstep_runs": (st, [P, ctypes.POINTER(ctypes.c_int64)]),
        "tomo_batch_phase_times": (st, [P, P]),
        "tomo_inject_fault": (st, [ctypes.c_char_p, ctypes.c_int32]),
        "tomo_check_report": (st, [ctypes.POINTER(ctypes.c_int32),
                                   ctypes.POINTER(ctypes.c_uint64)]),
        "tomo_batch_set_persistent": (st, [P, ctypes.c_int32]),
        "tomo_batch_set_tiles": (st, [P, ctypes.c_int32, ctypes.c_int32]),
        "tomo_batch_get_tiles": (st, [P, ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(ctypes.c_int32)]),
        "tomo_batch_autotune_tiles": (st, [P, P, P, ctypes.c_int32, P,
                                           ctypes.POINTER(ctypes.c_int32)]),
        "tomo_batch_set_wait_limit": (st, [P, ctypes.c_int64]),
        "tomo_batch_persistent_phase_ns": (st, [P, P, P, ctypes.c_int32,
                                                ctypes.POINTER(ctypes.c_int32),
                                                ctypes.POINTER(ctypes.c_int64)]),
        "tomo_batch_persistent_info": (st, [P, ctypes.POINTER(ctypes.c_int32),
                                            ctypes.POINTER(ctypes.c_int32),
                                            ctypes.POINTER(ctypes.c_int64)]),
        "tomo_batch_gradient": (st, [P, P, ctypes.POINTER(ctypes.c_double), P, P,
                                     ctypes.POINTER(SolveInfo)]),
        "tomo_batch_destroy": (st, [P]),
        "tomo_batch_last_error": (ctypes.c_char_p, [P]),
        "tomo_filter": (st, [G, P, P, ctypes.c_int]),
        "tomo_filter_d": (st, [G, P, P, ctypes.c_int]),
        "tomo_adjoint_gradient": (st, [G, P, P, ctypes.POINTER(ctypes.c_double), P,
                                       ctypes.POINTER(SolveInfo), ctypes.POINTER(SolveInfo)]),
        "tomo_adjoint_gradient_d": (st, [G, P, P, ctypes.POINTER(ctypes.c_double), P,
                                         ctypes.POINTER(SolveInfo), ctypes.POINTER(SolveInfo)]),
        "tomo_coarse_grain": (st, [G, P, ctypes.c_int32, P]),
        "tomo_coarse_grain_d": (st, [G, P, ctypes.c_int32, P]),
        "tomo_apply_stiffness": (st, [G, P, P, P]),
        "tomo_apply_stiffness_d": (st, [G, P, P, P]),
        "tomo_residual": (st, [G, P, P, P, P]),
        "tomo_residual_d": (st, [G, P, P, P]),
        "tomo_solve": (st, [G, P, P, ctypes.POINTER(SolveInfo)]),
        "tomo_solve_d": (st, [G, P, P, ctypes.POINTER(SolveInfo)]),
        "tomo_sensitivity": (st, [G, P, P, P, P]),
        "tomo_sensitivity_d": (st, [G, P, P, P, P]),
        "tomo_oc_step": (st, [G, P, P, P, ctypes.c_double, ctypes.c_double, P, P]),
        "tomo_oc_step_d": (st, [G, P, P, P, ctypes.c_double, ctypes.c_double, P, P]),
        "tomo_oc_step_noalloc": (st, [ctypes.c_int64, ctypes.c_double, P, P, P, ctypes.c_double,
                                      ctypes.c_double, P, P, P]),
        "tomo_gradient": (st, [G, P, P, P, P, ctypes.POINTER(SolveInfo)]),
        "tomo_gradient_d": (st, [G, P, P, P, P, ctypes.POINTER(SolveInfo)]),
        "tomo_get_displacement": (st, [G, P]),
        "tomo_get_displacement_d": (st, [G, P]),
        "tomo_get_counts": (st, [G, ctypes.POINTER(ctypes.c_int64),
                                 ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32)]),
        "tomo_get_launch_count": (st, [G, ctypes.POINTER(ctypes.c_int64)]),
        "tomo_profile_enable": (st, [G, ctypes.c_int]),
        "tomo_profile_phases": (st, [G, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_int64)]),
        "tomo_profile_levels": (st, [G, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_int64), ctypes.c_int]),
        "tomo_profile_read": (st, [G, ctypes.POINTER(ctypes.c_int64),
                                   ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_double)]),
        "tomo_last_error": (ctypes.c_char_p, [G]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = None


def coarse_dims(nx, ny, nz, block):
    """Elements per axis of the two-scale coarse grid: ceil(n / block)."""
    if block < 1:
        raise ValueError("block must be >= 1")
    return (-(-nx // block), -(-ny // block), -(-nz // block))


def lib():
    global _lib
    if _lib is None:
        _lib = _load()
    return _lib


def exported_symbols():
    """Names the binding expects the library to export."""
    return ["tomo_default_desc", "tomo_create_grid", "tomo_destroy_grid", "tomo_set_stream",
            "tomo_set_warm_start", "tomo_set_smoother", "tomo_get_smoother",
            "tomo_set_smoother_bound", "tomo_get_smoother_bound",
            "tomo_server_submit_optimize",
            "tomo_autotune_smoother", "tomo_autotune_smoother_d", "tomo_set_cycle",
            "tomo_autotune_smoother_multi", "tomo_autotune_smoother_multi_d",
            "tomo_set_coarse_tail", "tomo_get_coarse_tail",
            "tomo_get_cycle",
            "tomo_server_create", "tomo_server_submit",
            "tomo_server_wait", "tomo_server_get_stats", "tomo_server_destroy",
            "tomo_server_set_batching",
            "tomo_server_last_error", "tomo_grid_device_bytes", "tomo_estimate_device_bytes",
            "tomo_batch_create", "tomo_batch_append", "tomo_batch_size",
            "tomo_batch_set_lockstep", "tomo_batch_lockstep_runs", "tomo_batch_phase_times",
            "tomo_batch_set_persistent", "tomo_batch_set_wait_limit", "tomo_inject_fault",
            "tomo_check_report",
            "tomo_batch_persistent_info", "tomo_batch_persistent_phase_ns",
            "tomo_batch_set_tiles", "tomo_batch_get_tiles", "tomo_batch_autotune_tiles",
            "tomo_batch_gradient", "tomo_batch_destroy", "tomo_batch_last_error",
            "tomo_filter", "tomo_filter_d", "tomo_coarse_grain", "tomo_coarse_grain_d",
            "tomo_adjoint_gradient", "tomo_adjoint_gradient_d",
            "tomo_apply_stiffness", "tomo_apply_stiffness_d",
            "tomo_residual", "tomo_residual_d", "tomo_solve", "tomo_solve_d", "tomo_sensitivity", "tomo_sensitivity_d",
            "tomo_oc_step", "tomo_oc_step_d", "tomo_oc_step_noalloc", "tomo_gradient",
            "tomo_gradient_d",
            "tomo_get_displacement", "tomo_get_displacement_d", "tomo_get_counts",
            "tomo_get_launch_count", "tomo_profile_enable", "tomo_profile_phases",
            "tomo_profile_levels",
            "tomo_profile_read",
            "tomo_last_error"]


def _ptr(a, dtype, count, name):
    """Data pointer of a torch tensor or numpy array after type/size checks."""
    if a is None:
        return None
    try:
        import torch
        if isinstance(a, torch.Tensor):
            want = torch.float32 if dtype == np.float32 else torch.float64
            if a.dtype != want:
                raise TypeError(f"{name}: expected {want}, got {a.dtype}")
            if not a.is_contiguous():
                raise ValueError(f"{name}: tensor must be contiguous")
            if a.numel() != count:
                raise ValueError(f"{name}: expected {count} values, got {a.numel()}")
            return ctypes.c_void_p(a.data_ptr())
    except ImportError:
        pass
    if isinstance(a, np.ndarray):
        if a.dtype != dtype:
            raise TypeError(f"{name}: expected {np.dtype(dtype)}, got {a.dtype}")
        if not a.flags.c_contiguous:
            raise ValueError(f"{name}: array must be C-contiguous")
        if a.size != count:
            raise ValueError(f"{name}: expected {count} values, got {a.size}")
        return ctypes.c_void_p(a.ctypes.data)
    raise TypeError(f"{name}: expected a torch tensor or numpy array")


def inject_fault(site, nth=1):
    """Arm host-side fault injection (tomo_inject_fault): the nth pass through site
    ("alloc", "sync", "graph", "nan_input" or "slow_request") fails once; nth = 0
    disarms."""
    st = lib().tomo_inject_fault(str(site).encode(), int(nth))
    if st != 0:
        raise TomoError(st, f"unknown fault site {site!r} or nth < 0")


def check_report():
    """(checked build?, first recorded index violation or 0) from tomo_check_report; the
    records are cleared.  The word holds the site in bits 48-63 and the index below."""
    c, w = ctypes.c_int32(), ctypes.c_uint64()
    st = lib().tomo_check_report(ctypes.byref(c), ctypes.byref(w))
    if st != 0:
        raise TomoError(st, "tomo_check_report")
    return bool(c.value), w.value


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return ctypes.c_void_p(0)


def oc_step_noalloc(n_el, h, z, dcdz, dvdz, volfrac, move, z_new, change=None, stream=None):
    """tomo_oc_step_noalloc: FP32 device arrays, no grid handle, no allocation.  The call
    runs with z's device current and (unless ``stream`` is given) on that device's current
    torch stream; arrays on any other device are rejected by the library."""
    args = [_ptr(a, np.float32, n_el, nm) for a, nm in
            ((z, "z"), (dcdz, "dcdz"), (dvdz, "dvdz"))]
    zn = _ptr(z_new, np.float32, n_el, "z_new")
    ch = None
    if change is not None:
        ch = _ptr(change, np.float64, 1, "change")

    def call():
        return lib().tomo_oc_step_noalloc(
            ctypes.c_int64(n_el), ctypes.c_double(h), *args, ctypes.c_double(volfrac),
            ctypes.c_double(move), zn, ch, stream if stream is not None else _current_stream())

    dev = getattr(z, "device", None)
    if dev is not None and dev.type == "cuda":
        import torch
        with torch.cuda.device(dev):
            st = call()
    else:
        st = call()
    if st != 0:
        raise TomoError(st, lib().tomo_last_error(None).decode())


@dataclass
class Info:
    iters: int
    rel_res: float
    status: int
    mg_levels: int


class Grid:
    """A tomo grid handle (``tomo_create_grid``).  Float entry points for FP32 grids,
    double for FP64 grids; the same Python method serves both."""

    def __init__(self, nx, ny, nz, fixed, f, *, h=1.0, E0=1.0, Emin=1e-9, nu=0.3, penal=3.0,
                 rmin=1.5, precision=FP32, precond=PRECOND_MG, rtol=1e-6, maxit=2000,
                 mg_levels=0, smoother_degree=2, coarse_degree=0, cheb_ratio=20.0, cheb_lmax=0.0,
                 rr_every=50, stream=None):
        L = lib()
        d = GridDesc()
        L.tomo_default_desc(ctypes.byref(d))
        nn = (nx + 1) * (ny + 1) * (nz + 1)
        self._fixed = np.ascontiguousarray(np.asarray(fixed).astype(np.uint8).ravel())
        self._f = np.ascontiguousarray(np.asarray(f, dtype=np.float64).ravel())
        if self._fixed.size != 3 * nn or self._f.size != 3 * nn:
            raise ValueError(f"fixed and f must have 3*N_n = {3 * nn} entries")
        d.nx, d.ny, d.nz = nx, ny, nz
        d.h, d.E0, d.Emin, d.nu, d.penal, d.rmin = h, E0, Emin, nu, penal, rmin
        d.fixed_dof = self._fixed.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
        d.f = self._f.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        d.precision, d.precond = precision, precond
        d.rtol, d.maxit, d.mg_levels = rtol, maxit, mg_levels
        d.smoother_degree, d.cheb_ratio, d.rr_every = smoother_degree, cheb_ratio, rr_every
        d.coarse_degree = coarse_degree
        d.cheb_lmax = cheb_lmax
        d.stream = stream if stream is not None else _current_stream()
        h_out = ctypes.c_void_p()
        st = L.tomo_create_grid(ctypes.byref(d), ctypes.byref(h_out))
        if st != 0:
            raise TomoError(st, L.tomo_last_error(None).decode())
        self._h = h_out
        self.nx, self.ny, self.nz = nx, ny, nz
        self.n_el = nx * ny * nz
        self.n_nodes = nn
        self.precision = precision
        self.dtype = np.float64 if precision == FP64 else np.float32
        self._sfx = "_d" if precision == FP64 else ""

    @classmethod
    def from_problem(cls, p, **kw):
        d = p.dims
        return cls(d.nx, d.ny, d.nz, p.fixed, p.f, h=p.h, E0=p.E0, Emin=p.Emin, nu=p.nu,
                   penal=p.penal, rmin=p.rmin, **kw)

    # -- helpers --------------------------------------------------------------------------
    def _call(self, name, *args):
        st = getattr(lib(), name + self._sfx)(self._h, *args)
        if st != 0:
            raise TomoError(st, lib().tomo_last_error(self._h).decode())

    def _e(self, a, name):
        return _ptr(a, self.dtype, self.n_el, name)

    def _n(self, a, name):
        return _ptr(a, self.dtype, 3 * self.n_nodes, name)

    # -- entry points ---------------------------------------------------------------------
    def set_stream(self, stream):
        st = lib().tomo_set_stream(self._h, ctypes.c_void_p(stream))
        if st != 0:
            raise TomoError(st, lib().tomo_last_error(self._h).decode())

    def set_warm_start(self, on=True):
        """Start later gradient solves from the previous displacement (tomo_set_warm_start)."""
        st = lib().tomo_set_warm_start(self._h, int(bool(on)))
        if st != 0:
            raise TomoError(st, lib().tomo_last_error(self._h).decode())

    def set_smoother(self, fine_degree, coarse_degree, ratio=None):
        """Chebyshev degrees of the finest and the coarser levels (tomo_set_smoother); the
        interval ratio stays unless given."""
        if ratio is None:
            ratio = self.smoother()[2]
        st = lib().tomo_set_smoother(self._h, int(fine_degree), int(coarse_degree),
                                     float(ratio))
        if st != 0:
            raise TomoError(st, lib().tomo_last_error(self._h).decode())

    def smoother(self):
        """(fine_degree, coarse_degree, ratio) of the multigrid smoother."""
        f, c, r = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
        lib().tomo_get_smoother(self._h, ctypes.byref(f), ctypes.byref(c), ctypes.byref(r))
        return f.value, c.value, r.value

    def set_smoother_bound(self, lam):
        """Upper end of the smoothing interval (tomo_set_smoother_bound); lam <= 0 selects
        the element bound."""
        st = lib().tomo_set_smoother_bound(self._h, float(lam))
        if st != 0:
            raise TomoError(st, lib().tomo_last_error(self._h).decode())

    def smoother_bound(self):
        """(lam in use, element bound, solves redone at the element bound so far)."""
        lam, b, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
        lib().tomo_get_smoother_bound(self._h, ctypes.byref(lam), ctypes.byref(b),
                                      ctypes.byref(n))
        return lam.value, b.value, n.value

    def set_cycle(self, w_levels):
        """Multigrid cycle (tomo_set_cycle): bit l set = two coarse-grid corrections at
        level l (a W-cycle there); 0 = V-cycle."""
        st = lib().tomo_set_cycle(self._h, int(w_levels))
        if st != 0:
            raise TomoError(st, lib().tomo_last_error(self._h).decode())

    def set_coarse_tail(self, on=True):
        """Coarse levels of the V-cycle in one cluster launch (tomo_set_coarse_tail)."""
        st = lib().tomo_set_coarse_tail(self._h, int(bool(on)))
        if st != 0:
            raise TomoError(st, lib().tomo_last_error(self._h).decode())

    def coarse_tail(self):
        """Entry level of the coarse tail in use (0: off) (tomo_get_coarse_tail)."""
        l = ctypes.c_int32()
        lib().tomo_get_coarse_tail(self._h, ctypes.byref(l))
        return l.value

    def cycle(self):
        """The W-cycle level mask (tomo_get_cycle)."""
        w = ctypes.c_uint32()
        lib().tomo_get_cycle(self._h, ctypes.byref(w))
        return w.value

    def autotune(self, z, candidates=None, reps=2):
        """Time the state solve on design z (or on each design of a list: the medians are
        summed, tomo_autotune_smoother_multi) for each (fine, coarse) degree pair at the
        current bound, cycle and ratio, or for the built-in stages when None, and keep the
        fastest (tomo_autotune_smoother); returns (best (fine, coarse, lam, w_levels, ratio),
        list of dicts with fine, coarse, lam, w, ratio, ms, iters, status per candidate)."""
        if candidates is None:
            pairs, n = None, 23
        else:
            flat = [int(v) for pq in candidates for v in pq]
            pairs = (ctypes.c_int32 * len(flat))(*flat)
            n = len(candidates)
        res = (TuneResult * n)()
        best = ctypes.c_int32(-1)
        pp = ctypes.cast(pairs, ctypes.c_void_p) if pairs else None
        if isinstance(z, (list, tuple)):
            zs = (ctypes.c_void_p * len(z))(*[self._e(a, "z") for a in z])
            st = getattr(lib(), "tomo_autotune_smoother_multi" + self._sfx)(
                self._h, ctypes.cast(zs, ctypes.c_void_p), len(z), pp, n, int(reps),
                ctypes.cast(res, ctypes.c_void_p), ctypes.byref(best))
        else:
            st = getattr(lib(), "tomo_autotune_smoother" + self._sfx)(
                self._h, self._e(z, "z"), pp, n, int(reps), ctypes.cast(res, ctypes.c_void_p),
                ctypes.byref(best))
        if st != 0:
            raise TomoError(st, lib().tomo_last_error(self._h).decode())
        rows = [dict(fine=r.fine_degree, coarse=r.coarse_degree, lam=r.lam, w=r.w_levels,
                     ratio=r.ratio, ms=r.ms, iters=r.iters, status=r.status) for r in res]
        b = rows[best.value]
        return (b["fine"], b["coarse"], b["lam"], b["w"], b["ratio"]), rows

    def filter(self, x, out, transpose=False):
        self._call("tomo_filter", self._e(x, "in"), self._e(out, "out"), int(bool(transpose)))

    def coarse_grain(self, z, block, out):
        """Two-scale coarse design: out = block means of z over block^3 element blocks
        (``coarse_dims`` gives the coarse grid)."""
        if block >= 1:
            cx, cy, cz = coarse_dims(self.nx, self.ny, self.nz, block)
            count = cx * cy * cz
        else:   # the library rejects the block size (TOMO_EINVAL)
            count = int(out.numel() if hasattr(out, "numel") else np.asarray(out).size)
        self._call("tomo_coarse_grain", self._e(z, "z"), int(block),
                   _ptr(out, self.dtype, count, "z_coarse"))

    def apply_stiffness(self, rho, x, y):
        self._call("tomo_apply_stiffness", self._e(rho, "rho"), self._n(x, "x"), self._n(y, "y"))

    def residual(self, rho, u, r, u_lo=None):
        if self.precision == FP64:
            if u_lo is not None:
                raise ValueError("u_lo is for FP32 grids")
            self._call("tomo_residual", self._e(rho, "rho"), self._n(u, "u"), self._n(r, "r"))
        else:
            self._call("tomo_residual", self._e(rho, "rho"), self._n(u, "u"),
                       self._n(u_lo, "u_lo") if u_lo is not None else None, self._n(r, "r"))

    def solve(self, rho, u) -> Info:
        info = SolveInfo()
        name = "tomo_solve"
        st = getattr(lib(), name + self._sfx)(self._h, self._e(rho, "rho"), self._n(u, "u"),
                                              ctypes.byref(info))
        if st not in (0,):
            raise TomoError(st, lib().tomo_last_error(self._h).decode())
        return Info(info.iters, info.rel_res, info.status, info.mg_levels)

    def sensitivity(self, rho, u, dc=None) -> float:
        c = ctypes.c_double()
        self._call("tomo_sensitivity", self._e(rho, "rho"), self._n(u, "u"), ctypes.byref(c),
                   self._e(dc, "dc") if dc is not None else None)
        return c.value

    def oc_step(self, z, dcdz, dvdz, volfrac, move, z_new) -> float:
        ch = ctypes.c_double()
        self._call("tomo_oc_step", self._e(z, "z"), self._e(dcdz, "dcdz"), self._e(dvdz, "dvdz"),
                   ctypes.c_double(volfrac), ctypes.c_double(move), self._e(z_new, "z_new"),
                   ctypes.byref(ch))
        return ch.value

    def gradient(self, z, dcdz, dvdz=None):
        """Returns (compliance, Info)."""
        c = ctypes.c_double()
        info = SolveInfo()
        self._call("tomo_gradient", self._e(z, "z"), ctypes.byref(c), self._e(dcdz, "dcdz"),
                   self._e(dvdz, "dvdz") if dvdz is not None else None, ctypes.byref(info))
        return c.value, Info(info.iters, info.rel_res, info.status, info.mg_levels)

    def adjoint_gradient(self, z, l, djdz):
        """J = l^T u and dJ/dz through the adjoint (Eq. 3); returns (J, info_u, info_l)."""
        J = ctypes.c_double()
        iu, il = SolveInfo(), SolveInfo()
        self._call("tomo_adjoint_gradient", self._e(z, "z"), self._n(l, "l"), ctypes.byref(J),
                   self._e(djdz, "djdz"), ctypes.byref(iu), ctypes.byref(il))
        mk = lambda i: Info(i.iters, i.rel_res, i.status, i.mg_levels)  # noqa: E731
        return J.value, mk(iu), mk(il)

    def device_bytes(self) -> int:
        """Device memory held by this grid (tomo_grid_device_bytes)."""
        n = ctypes.c_size_t()
        st = lib().tomo_grid_device_bytes(self._h, ctypes.byref(n))
        if st != 0:
            raise TomoError(st, "tomo_grid_device_bytes")
        return n.value

    def get_displacement(self, u):
        self._call("tomo_get_displacement", self._n(u, "u"))

    def counts(self):
        ne, nn, nl = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        st = lib().tomo_get_counts(self._h, ctypes.byref(ne), ctypes.byref(nn), ctypes.byref(nl))
        if st != 0:
            raise TomoError(st, "tomo_get_counts")
        return ne.value, nn.value, nl.value

    def launch_count(self) -> int:
        n = ctypes.c_int64()
        st = lib().tomo_get_launch_count(self._h, ctypes.byref(n))
        if st != 0:
            raise TomoError(st, "tomo_get_launch_count")
        return n.value

    def profile_enable(self, on=True, phases=False):
        lib().tomo_profile_enable(self._h, (1 if on else 0) | (2 if phases else 0))

    def profile_levels(self, n=16):
        """(ms, launches) per multigrid level, accumulated by profile_read()."""
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_int64 * n)()
        st = lib().tomo_profile_levels(self._h, ms, cnt, n)
        if st != 0:
            raise TomoError(st, "tomo_profile_levels")
        return list(ms), list(cnt)

    def profile_phases(self):
        """Accumulated ms per phase since the last call: filter, levels, cg, sensitivity,
        adjoints, oc; and the number of gradient calls."""
        ms = (ctypes.c_double * 7)()
        n = ctypes.c_int64()
        st = lib().tomo_profile_phases(self._h, ms, ctypes.byref(n))
        if st != 0:
            raise TomoError(st, "tomo_profile_phases")
        names = ["filter", "levels", "cg", "sensitivity", "adjoints", "unused", "oc"]
        out = {k: ms[i] for i, k in enumerate(names) if k != "unused"}
        return out, n.value

    def profile_read(self):
        n, ms, b = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
        st = lib().tomo_profile_read(self._h, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(b))
        if st != 0:
            raise TomoError(st, lib().tomo_last_error(self._h).decode())
        return n.value, ms.value, b.value

    def close(self):
        if getattr(self, "_h", None):
            lib().tomo_destroy_grid(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Batch:
    """A set of FP32 grids evaluated together (``tomo_batch_*``): ``workers`` host threads,
    one CUDA stream each, for the per-grid steps; with ``lockstep`` (the default) one CG
    loop for all grids, each phase one launch for every grid.  The batch does not own its
    grids."""

    def __init__(self, workers=8, lockstep=True, persistent=False):
        h = ctypes.c_void_p()
        st = lib().tomo_batch_create(int(workers), ctypes.byref(h))
        if st != 0:
            raise TomoError(st, lib().tomo_batch_last_error(None).decode())
        self._h = h
        self.grids = []
        lib().tomo_batch_set_lockstep(self._h, int(bool(lockstep)))
        lib().tomo_batch_set_persistent(self._h, int(bool(persistent)))

    def set_tiles(self, tile_rows=8, waves=4):
        """Tiles of the batched products (tomo_batch_set_tiles): thread rows per CTA (8 or
        4) and waves of resident CTAs for the z-chunking."""
        st = lib().tomo_batch_set_tiles(self._h, int(tile_rows), int(waves))
        if st != 0:
            raise TomoError(st, "tile rows must be 8 or 4 and waves 1..16")

    def tiles(self):
        r, w = ctypes.c_int32(), ctypes.c_int32()
        lib().tomo_batch_get_tiles(self._h, ctypes.byref(r), ctypes.byref(w))
        return r.value, w.value

    def autotune_tiles(self, zs, dcdzs, reps=2):
        """tomo_batch_autotune_tiles: returns (best (tile_rows, waves), list of dicts with
        rows, waves, status, ms per candidate); the best becomes the batch's setting."""
        n = len(self.grids)
        if len(zs) != n or len(dcdzs) != n:
            raise ValueError("one array per grid")
        arr = ctypes.c_void_p * n
        z = arr(*[g._e(a, "z") for g, a in zip(self.grids, zs)])
        dc = arr(*[g._e(a, "dcdz") for g, a in zip(self.grids, dcdzs)])
        res = (BatchTuneResult * 6)()
        best = ctypes.c_int32(-1)
        st = lib().tomo_batch_autotune_tiles(self._h, ctypes.cast(z, ctypes.c_void_p),
                                             ctypes.cast(dc, ctypes.c_void_p), int(reps),
                                             ctypes.cast(res, ctypes.c_void_p),
                                             ctypes.byref(best))
        if st != 0:
            raise TomoError(st, lib().tomo_batch_last_error(self._h).decode())
        rows = [dict(rows=r.tile_rows, waves=r.waves, status=r.status, ms=r.ms) for r in res]
        b = rows[best.value]
        return (b["rows"], b["waves"]), rows

    def set_persistent(self, on=True):
        """Each lockstep CG iteration as one cooperative launch (tomo_batch_set_persistent);
        on = 2 also times the phases (persistent_phase_times)."""
        st = lib().tomo_batch_set_persistent(self._h, int(on))
        if st != 0:
            raise TomoError(st, "persistent mode must be 0, 1 or 2")

    def set_wait_limit(self, ns):
        """Barrier wait limit of the persistent iteration in ns (tomo_batch_set_wait_limit)."""
        if int(ns) < 0:
            raise ValueError("wait limit must be >= 0")
        st = lib().tomo_batch_set_wait_limit(self._h, int(ns))
        if st != 0:
            raise TomoError(st, "wait limit rejected")

    PHASE_KINDS = ("product", "product+pTq", "residual", "chebyshev", "chebyshev+bTx",
                   "fp64 residual replacement", "jacobi start", "restriction",
                   "prolongation", "coarsest solve", "cg x/r", "cg p")

    def persistent_phase_times(self):
        """([(kind, total microseconds)], launches) of the latest call's persistent
        iterations (tomo_batch_persistent_phase_ns; needs set_persistent(2)); ([], 0)
        without timing or when the loop in use is the launched one."""
        cnt, nl = ctypes.c_int32(), ctypes.c_int64()
        lib().tomo_batch_persistent_phase_ns(self._h, None, None, 0, ctypes.byref(cnt), None)
        n = cnt.value
        if n == 0:
            return [], 0
        ns = (ctypes.c_int64 * n)()
        kinds = (ctypes.c_int32 * n)()
        st = lib().tomo_batch_persistent_phase_ns(self._h, ctypes.cast(ns, ctypes.c_void_p),
                                                  ctypes.cast(kinds, ctypes.c_void_p), n,
                                                  ctypes.byref(cnt), ctypes.byref(nl))
        if st != 0:
            raise TomoError(st, lib().tomo_batch_last_error(self._h).decode())
        return [(self.PHASE_KINDS[k], t / 1e3) for k, t in zip(kinds, ns)], nl.value

    @property
    def persistent_info(self):
        """(ctas, phases, runs) of the persistent iteration (tomo_batch_persistent_info);
        ctas = phases = 0 when the captured loop is the launched one."""
        c, p, r = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        lib().tomo_batch_persistent_info(self._h, ctypes.byref(c), ctypes.byref(p),
                                         ctypes.byref(r))
        return c.value, p.value, r.value

    def phase_times(self):
        """Phases of the last lockstep call in ms (tomo_batch_phase_times): issue of the
        per-grid steps before the loop, first V-cycle, CG loop, scalar read-back, per-grid
        steps after the loop."""
        ms = (ctypes.c_double * 5)()
        lib().tomo_batch_phase_times(self._h, ctypes.cast(ms, ctypes.c_void_p))
        return dict(zip(("issue_before", "first_vcycle", "loop", "readback", "after"), ms))

    @property
    def lockstep_runs(self):
        """Number of gradient calls that ran in lockstep."""
        n = ctypes.c_int64()
        lib().tomo_batch_lockstep_runs(self._h, ctypes.byref(n))
        return n.value

    def append(self, grid):
        st = lib().tomo_batch_append(self._h, grid._h)
        if st != 0:
            raise TomoError(st, lib().tomo_batch_last_error(self._h).decode())
        self.grids.append(grid)

    def __len__(self):
        n = ctypes.c_int32()
        lib().tomo_batch_size(self._h, ctypes.byref(n))
        return n.value

    def gradient(self, zs, dcdzs, dvdzs=None):
        """tomo_gradient on every grid; returns (compliances, infos)."""
        n = len(self.grids)
        if len(zs) != n or len(dcdzs) != n or (dvdzs is not None and len(dvdzs) != n):
            raise ValueError("one array per grid")
        arr = ctypes.c_void_p * n
        z = arr(*[g._e(a, "z") for g, a in zip(self.grids, zs)])
        dc = arr(*[g._e(a, "dcdz") for g, a in zip(self.grids, dcdzs)])
        dv = arr(*[g._e(a, "dvdz") for g, a in zip(self.grids, dvdzs)]) if dvdzs else None
        c = (ctypes.c_double * n)()
        info = (SolveInfo * n)()
        st = lib().tomo_batch_gradient(self._h, ctypes.cast(z, ctypes.c_void_p), c,
                                       ctypes.cast(dc, ctypes.c_void_p),
                                       ctypes.cast(dv, ctypes.c_void_p) if dv else None, info)
        if st != 0:
            raise TomoError(st, lib().tomo_batch_last_error(self._h).decode())
        return list(c), [Info(i.iters, i.rel_res, i.status, i.mg_levels) for i in info]

    def close(self):
        if getattr(self, "_h", None):
            lib().tomo_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def _problem_desc(p, precision=FP32, **kw):
    """A filled GridDesc for problem p (arrays referenced, not copied: keep p alive)."""
    L = lib()
    d = GridDesc()
    L.tomo_default_desc(ctypes.byref(d))
    dims = p.dims
    d.nx, d.ny, d.nz = dims.nx, dims.ny, dims.nz
    d.h, d.E0, d.Emin, d.nu, d.penal, d.rmin = p.h, p.E0, p.Emin, p.nu, p.penal, p.rmin
    fixed = np.ascontiguousarray(p.fixed.astype(np.uint8))
    f = np.ascontiguousarray(p.f.astype(np.float64))
    d.fixed_dof = fixed.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    d.f = f.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    d.precision = precision
    for k, v in kw.items():
        setattr(d, k, v)
    return d, (fixed, f)


def estimate_device_bytes(p, precision=FP32):
    d, keep = _problem_desc(p, precision)
    n = ctypes.c_size_t()
    st = lib().tomo_estimate_device_bytes(ctypes.byref(d), ctypes.byref(n))
    if st != 0:
        raise TomoError(st, "tomo_estimate_device_bytes")
    return n.value


class Server:
    """The request loop (``tomo_server_*``): gradient requests on grids of different sizes,
    ``workers`` threads with a stream each, grids resident per session, admission under a
    device-memory budget (bytes)."""

    def __init__(self, workers=8, budget_bytes=8 << 30, max_batch=1, batch_workers=4):
        h = ctypes.c_void_p()
        st = lib().tomo_server_create(int(workers), int(budget_bytes), ctypes.byref(h))
        if st != 0:
            raise TomoError(st, "tomo_server_create")
        self._h = h
        self._pending = {}
        if max_batch > 1:
            self.set_batching(max_batch, batch_workers)

    def set_batching(self, max_batch, batch_workers=4):
        """Lockstep batching of queued gradient requests (tomo_server_set_batching)."""
        st = lib().tomo_server_set_batching(self._h, int(max_batch), int(batch_workers))
        if st != 0:
            raise TomoError(st, "tomo_server_set_batching")

    def submit(self, p, z=None, session=-1, dvdz=True):
        """Queue tomo_gradient for problem p (FP32) with design z (default p.z0); returns a
        ticket.  Outputs are host arrays held until ``wait``."""
        d, keep = _problem_desc(p, FP32)
        zz = np.ascontiguousarray(np.asarray(p.z0 if z is None else z, np.float32))
        dc = np.empty(p.n_el, np.float32)
        dv = np.empty(p.n_el, np.float32) if dvdz else None
        t = ctypes.c_int64()
        st = lib().tomo_server_submit(self._h, ctypes.byref(d), int(session),
                                      zz.ctypes.data_as(ctypes.c_void_p),
                                      dc.ctypes.data_as(ctypes.c_void_p),
                                      dv.ctypes.data_as(ctypes.c_void_p) if dv is not None
                                      else None, ctypes.byref(t))
        if st != 0:
            raise TomoError(st, lib().tomo_server_last_error(self._h).decode())
        self._pending[t.value] = (dc, dv, keep, zz)
        return t.value

    def submit_optimize(self, p, iters, z=None, session=-1, volfrac=None, move=None):
        """Queue an optimisation request: `iters` OC iterations of problem p from design z
        (default p.z0) with p's volume fraction and move limit unless given; ``wait``
        returns (Result, final design, None)."""
        d, keep = _problem_desc(p, FP32)
        zz = np.ascontiguousarray(np.asarray(p.z0 if z is None else z, np.float32))
        zo = np.empty(p.n_el, np.float32)
        t = ctypes.c_int64()
        st = lib().tomo_server_submit_optimize(
            self._h, ctypes.byref(d), int(session), zz.ctypes.data_as(ctypes.c_void_p),
            int(iters), float(p.volfrac if volfrac is None else volfrac),
            float(p.move if move is None else move), zo.ctypes.data_as(ctypes.c_void_p),
            ctypes.byref(t))
        if st != 0:
            raise TomoError(st, lib().tomo_server_last_error(self._h).decode())
        self._pending[t.value] = (zo, None, keep, zz)
        return t.value

    def wait(self, ticket):
        """Returns (Result, dcdz, dvdz) for a gradient ticket, (Result, final design, None)
        for an optimisation ticket."""
        r = Result()
        st = lib().tomo_server_wait(self._h, int(ticket), ctypes.byref(r))
        if st != 0:
            raise TomoError(st, lib().tomo_server_last_error(self._h).decode())
        dc, dv, _, _ = self._pending.pop(ticket)
        return r, dc, dv

    def stats(self):
        s = ServerStats()
        lib().tomo_server_get_stats(self._h, ctypes.byref(s))
        return {k: getattr(s, k) for k, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            lib().tomo_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
