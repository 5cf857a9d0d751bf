"""ctypes binding of the C ABI in include/csem.h (argument marshalling only).

Every function here has the name of the C entry point without its `csem_`
prefix and forwards plain pointers and sizes; all arithmetic runs in the
CUDA library.  A missing library is an error: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcsemfw.so")

OK, ERR_INVALID_ARG, ERR_OUT_OF_DOMAIN, ERR_CFL, ERR_OOM, ERR_NONFINITE, ERR_TIMEOUT, ERR_CUDA = 0, -1, -2, -3, -4, -5, -6, -7

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_V = ctypes.c_void_p


class CsemError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"csem error {code}: {msg}")
        self.code = code


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("xn", _D), ("yn", _D), ("zn", _D), ("npml", ctypes.c_int)]


class PointsC(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("x", _D), ("y", _D), ("z", _D), ("comp", _I)]


class Opts(ctypes.Structure):
    _fields_ = [("f0", ctypes.c_double), ("rho_max", ctypes.c_double), ("dt", ctypes.c_double),
                ("nt", ctypes.c_int), ("cfl_safety", ctypes.c_double), ("precision", ctypes.c_int),
                ("kahan", ctypes.c_int), ("n_freq", ctypes.c_int), ("freqs", _D),
                ("max_src", ctypes.c_int), ("max_rec", ctypes.c_int), ("anisotropy", ctypes.c_int),
                ("order", ctypes.c_int), ("ring_slots", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("npml", ctypes.c_int),
                ("pitch", ctypes.c_int), ("vol_elems", ctypes.c_longlong), ("dt", ctypes.c_double),
                ("nt", ctypes.c_int), ("precision", ctypes.c_int), ("kahan", ctypes.c_int),
                ("n_freq", ctypes.c_int), ("max_src", ctypes.c_int), ("max_rec", ctypes.c_int),
                ("workspace_bytes", ctypes.c_longlong), ("transform_block", ctypes.c_int),
                ("anisotropy", ctypes.c_int), ("order", ctypes.c_int)]


# name -> (restype, argtypes)
SIGNATURES = {
    "csem_create": (ctypes.c_int, [ctypes.POINTER(_V), ctypes.POINTER(Grid), ctypes.POINTER(Opts)]),
    "csem_destroy": (None, [_V]),
    "csem_get_info": (ctypes.c_int, [_V, ctypes.POINTER(Info)]),
    "csem_fwd_model": (ctypes.c_int, [_V, _V, ctypes.POINTER(PointsC), ctypes.POINTER(PointsC), _V, _V, _V]),
    "csem_estimate_adjoint_basis": (ctypes.c_int, [ctypes.c_double, ctypes.c_int, _D, ctypes.c_int, ctypes.c_double,
                                                   ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                                   _V, _D, _I, _V]),
    "csem_estimate_adjoint_basis_noalloc": (ctypes.c_int, [ctypes.c_double, ctypes.c_int, _D, ctypes.c_int,
                                                           ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                                           ctypes.c_int, ctypes.c_double, _V, _D, _I, _V]),
    "csem_misfit": (ctypes.c_int, [ctypes.c_int, _V, _V, _V, _V, _V, _V]),
    "csem_adjoint_model": (ctypes.c_int, [_V, _V, ctypes.POINTER(PointsC), ctypes.c_int, _V, _V, _V, _V]),
    "csem_gradient": (ctypes.c_int, [_V, _V, _V, _V, ctypes.c_int, ctypes.c_int, _V, _V]),
    "csem_td_plan": (ctypes.c_int, [_V, ctypes.c_int, ctypes.c_int, ctypes.c_longlong, _I,
                                    ctypes.POINTER(ctypes.c_longlong)]),
    "csem_gradient_td": (ctypes.c_int, [_V, _V, ctypes.POINTER(PointsC), ctypes.POINTER(PointsC), _V, ctypes.c_int,
                                        ctypes.c_int, _V, _V, ctypes.c_longlong, _V]),
    "csem_set_early_stop": (ctypes.c_int, [_V, ctypes.c_double]),
    "csem_last_run_steps": (ctypes.c_int, [_V, _V, _I]),
    "csem_set_early_stop_volumes": (ctypes.c_int, [_V, ctypes.c_double, ctypes.c_double]),
    "csem_autotune": (ctypes.c_int, [_V, ctypes.c_int, _I, _V]),
    "csem_set_launch": (ctypes.c_int, [_V, _I]),
    "csem_set_wavelet": (ctypes.c_int, [_V, _D]),
    "csem_set_trace": (ctypes.c_int, [_V, _V]),
    "csem_set_copy_fault": (ctypes.c_int, [_V, ctypes.c_int]),
    "csem_check": (ctypes.c_int, [_V, _V]),
    "csem_launch_count": (ctypes.c_longlong, []),
    "csem_time_step_kernels": (ctypes.c_int, [_V, ctypes.c_int, _V, ctypes.c_int, _D, _V]),
    "csem_last_error": (ctypes.c_char_p, []),
}

_lib = None


def lib():
    """Loads libcsemfw.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                               "(there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc: int):
    if rc != OK:
        raise CsemError(rc, lib().csem_last_error().decode())


def _dptr(a):
    return a.ctypes.data_as(_D)


def make_points(pts, keep: list) -> PointsC:
    import numpy as np
    x = np.ascontiguousarray(pts.x, np.float64)
    y = np.ascontiguousarray(pts.y, np.float64)
    z = np.ascontiguousarray(pts.z, np.float64)
    c = np.ascontiguousarray(pts.comp, np.int32)
    keep += [x, y, z, c]
    return PointsC(int(x.size), _dptr(x), _dptr(y), _dptr(z), c.ctypes.data_as(_I))


def create(xn, yn, zn, npml, freqs, f0=1.0, rho_max=1.0, dt=0.0, nt=0, precision=32, kahan=1,
           max_src=1, max_rec=0, cfl_safety=0.0, anisotropy=0, order=2, ring_slots=0):
    import numpy as np
    keep = [np.ascontiguousarray(v, np.float64) for v in (xn, yn, zn, freqs)]
    g = Grid(keep[0].size - 1, keep[1].size - 1, keep[2].size - 1, _dptr(keep[0]), _dptr(keep[1]), _dptr(keep[2]),
             int(npml))
    o = Opts(float(f0), float(rho_max), float(dt), int(nt), float(cfl_safety), int(precision), int(kahan),
             int(keep[3].size), _dptr(keep[3]), int(max_src), int(max_rec), int(anisotropy), int(order),
             int(ring_slots))
    ctx = _V()
    _check(lib().csem_create(ctypes.byref(ctx), ctypes.byref(g), ctypes.byref(o)))
    return ctx


def destroy(ctx):
    lib().csem_destroy(ctx)


def get_info(ctx) -> Info:
    info = Info()
    _check(lib().csem_get_info(ctx, ctypes.byref(info)))
    return info


def fwd_model(ctx, rho_ptr, src, rec, d_syn_ptr, evol_ptr, stream):
    keep = []
    _check(lib().csem_fwd_model(ctx, rho_ptr, ctypes.byref(make_points(src, keep)),
                                ctypes.byref(make_points(rec, keep)), d_syn_ptr, evol_ptr, stream))


def estimate_adjoint_basis(dt, nt, freqs, f0, gamma, gamma_is_relative, max_iter, tol, basis_ptr, stream):
    import numpy as np
    fr = np.ascontiguousarray(freqs, np.float64)
    fit = ctypes.c_double(0.0)
    its = ctypes.c_int(0)
    _check(lib().csem_estimate_adjoint_basis(float(dt), int(nt), _dptr(fr), int(fr.size), float(f0), float(gamma),
                                             int(gamma_is_relative), int(max_iter), float(tol), basis_ptr,
                                             ctypes.byref(fit), ctypes.byref(its), stream))
    return fit.value, its.value


def estimate_adjoint_basis_noalloc(dt, nt, freqs, f0, gamma, gamma_is_relative, max_iter, tol, basis_ptr, stream):
    """As estimate_adjoint_basis, with the scratch in the library's static device array (no allocation)."""
    import numpy as np
    fr = np.ascontiguousarray(freqs, np.float64)
    fit = ctypes.c_double(0.0)
    its = ctypes.c_int(0)
    _check(lib().csem_estimate_adjoint_basis_noalloc(float(dt), int(nt), _dptr(fr), int(fr.size), float(f0),
                                                     float(gamma), int(gamma_is_relative), int(max_iter), float(tol),
                                                     basis_ptr, ctypes.byref(fit), ctypes.byref(its), stream))
    return fit.value, its.value


def misfit(n, d_obs_ptr, d_syn_ptr, w_ptr, resid_ptr, phi_ptr, stream):
    _check(lib().csem_misfit(int(n), d_obs_ptr, d_syn_ptr, w_ptr, resid_ptr, phi_ptr, stream))


def adjoint_model(ctx, rho_ptr, rec, n_src, resid_ptr, basis_ptr, vvol_ptr, stream):
    keep = []
    _check(lib().csem_adjoint_model(ctx, rho_ptr, ctypes.byref(make_points(rec, keep)), int(n_src), resid_ptr,
                                    basis_ptr, vvol_ptr, stream))


def gradient(ctx, rho_ptr, evol_ptr, vvol_ptr, n_src, wrt, grad_ptr, stream):
    _check(lib().csem_gradient(ctx, rho_ptr, evol_ptr, vvol_ptr, int(n_src), int(wrt), grad_ptr, stream))


def td_plan(ctx, n_src, n_rec, budget_bytes=0, segment=0):
    """(segment, workspace bytes) of the time-domain adjoint gradient."""
    seg = ctypes.c_int(int(segment))
    nb = ctypes.c_longlong(0)
    _check(lib().csem_td_plan(ctx, int(n_src), int(n_rec), int(budget_bytes), ctypes.byref(seg), ctypes.byref(nb)))
    return seg.value, nb.value


def gradient_td(ctx, rho_ptr, src, rec, resid_ptr, segment, wrt, grad_ptr, work_ptr, work_bytes, stream):
    keep = []
    _check(lib().csem_gradient_td(ctx, rho_ptr, ctypes.byref(make_points(src, keep)),
                                  ctypes.byref(make_points(rec, keep)), resid_ptr, int(segment), int(wrt), grad_ptr,
                                  work_ptr, int(work_bytes), stream))


def set_early_stop(ctx, tol):
    _check(lib().csem_set_early_stop(ctx, float(tol)))


def set_early_stop_volumes(ctx, tol, floor_frac):
    _check(lib().csem_set_early_stop_volumes(ctx, float(tol), float(floor_frac)))


def last_run_steps(ctx, stream) -> int:
    v = ctypes.c_int(0)
    _check(lib().csem_last_run_steps(ctx, stream, ctypes.byref(v)))
    return v.value


def autotune(ctx, n_src, stream):
    """Times the launch candidates; returns (H, E, flush) codes (see csem_autotune)."""
    out = (ctypes.c_int * 4)()
    _check(lib().csem_autotune(ctx, int(n_src), out, stream))
    return int(out[0]), int(out[1]), int(out[2]), int(out[3])


def set_launch(ctx, kz_h, mb_h, kz_e, mb_e, fused_kz, flush_mode, block, vec_h=0, vec_e=0, tma_h=0, tma_e=0,
               lean_h=0, lean_e=0):
    cfg = (ctypes.c_int * 13)(kz_h, mb_h, kz_e, mb_e, fused_kz, flush_mode, block, vec_h, vec_e, tma_h, tma_e,
                              lean_h, lean_e)
    _check(lib().csem_set_launch(ctx, cfg))


def set_wavelet(ctx, wavelet=None):
    import numpy as np
    if wavelet is None:
        _check(lib().csem_set_wavelet(ctx, None))
    else:
        w = np.ascontiguousarray(wavelet, np.float64)
        _check(lib().csem_set_wavelet(ctx, _dptr(w)))


def set_trace(ctx, trace_ptr):
    _check(lib().csem_set_trace(ctx, trace_ptr))


def set_copy_fault(ctx, extra_bytes):
    _check(lib().csem_set_copy_fault(ctx, int(extra_bytes)))


def check(ctx, stream):
    _check(lib().csem_check(ctx, stream))


def launch_count() -> int:
    return int(lib().csem_launch_count())


def time_step_kernels(ctx, n_src, vol_ptr, launches, stream):
    """Mean ms per launch of (H half-step, injection, E step, transform flush of 16 snapshots)."""
    out = (ctypes.c_double * 4)()
    _check(lib().csem_time_step_kernels(ctx, int(n_src), vol_ptr, int(launches), out, stream))
    return list(out)


def last_error() -> str:
    return lib().csem_last_error().decode()
