"""ctypes binding of the C ABI declared in include/mg.h and include/mg_box.h.

The functions below carry the C names and only marshal arguments; every step
of the solve runs in libmg.so.  Arrays may be torch tensors (CUDA or CPU),
numpy arrays or raw integer addresses; they must be contiguous float64.
There is no fallback: if libmg.so is missing or fails to load, importing this
module raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

MG_MAX_LEVELS = 8
MG_OK, MG_EINVAL, MG_ENOMEM, MG_ECUDA, MG_ESTATE, MG_ENOCONV, MG_EDIVERGED, MG_ETIMEOUT = range(8)
MG_FP64, MG_MIXED = 0, 1
MG_GUESS_INTERP, MG_GUESS_ZERO, MG_GUESS_USER, MG_GUESS_LEARNED = 0, 1, 2, 3
MG_FORCE_EQ2, MG_FORCE_CD2 = 0, 1
MG_IFACE_BUFFER, MG_IFACE_FROZEN = 0, 1
MG_STOP_RESIDUAL, MG_STOP_FORCE = 0, 1


class mg_hierarchy_desc(C.Structure):
    _fields_ = [("dim", C.c_int), ("num_levels", C.c_int), ("n", C.c_int * MG_MAX_LEVELS),
                ("lo", (C.c_double * 3) * MG_MAX_LEVELS), ("h0", C.c_double), ("G", C.c_double),
                ("tree", C.c_int), ("parent", C.c_int * MG_MAX_LEVELS)]


class mg_options(C.Structure):
    _fields_ = [("nu_pre", C.c_int), ("nu_post", C.c_int), ("max_cycles", C.c_int), ("rel_tol", C.c_double),
                ("precision", C.c_int), ("inner_cycles", C.c_int), ("guess", C.c_int),
                ("force_stencil", C.c_int), ("interface", C.c_int),
                ("stop", C.c_int), ("stream", C.c_void_p), ("inner_max", C.c_int)]


class mg_level_stats(C.Structure):
    _fields_ = [("cycles", C.c_int), ("outer_steps", C.c_int), ("rel_res", C.c_double), ("b_norm", C.c_double),
                ("status", C.c_int)]


class mg_box_desc(C.Structure):
    _fields_ = [("dim", C.c_int), ("num_patches", C.c_int), ("n", (C.c_int * 3) * MG_MAX_LEVELS),
                ("lo", (C.c_double * 3) * MG_MAX_LEVELS), ("h0", C.c_double), ("G", C.c_double),
                ("tree", C.c_int), ("parent", C.c_int * MG_MAX_LEVELS)]


class mg_kernel_stat(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_long), ("ms", C.c_double), ("bytes", C.c_double)]


_vp = C.c_void_p
_SIGS = {
    "mg_default_options": (C.c_int, [C.POINTER(mg_options)]),
    "mg_create_hierarchy": (C.c_int, [C.POINTER(mg_hierarchy_desc), C.c_int, C.POINTER(mg_options), C.POINTER(_vp)]),
    "mg_set_density": (C.c_int, [_vp, C.c_int, C.c_int, _vp, _vp, _vp]),
    "mg_set_guess": (C.c_int, [_vp, C.c_int, C.c_int, _vp]),
    "mg_solve": (C.c_int, [_vp, C.POINTER(mg_level_stats)]),
    "mg_forces": (C.c_int, [_vp, C.c_int, C.c_int, _vp, _vp]),
    "mg_set_outputs": (C.c_int, [_vp, C.c_int, C.c_int, _vp, _vp]),
    "mg_destroy": (C.c_int, [_vp]),
    "mg_status_str": (C.c_char_p, [C.c_int]),
    "mg_error_message": (C.c_char_p, [_vp]),
    "mg_level_sizes": (C.c_int, [C.c_int, C.POINTER(C.c_int), C.c_int]),
    "mg_profile": (C.c_int, [_vp, C.c_int]),
    "mg_autotune": (C.c_int, [_vp, C.c_char_p]),
    "mg_tuning": (C.c_int, [_vp, C.c_int, C.c_int, C.POINTER(C.c_int), C.c_int]),
    "mg_time_smoothing": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double),
                                    C.POINTER(C.c_double)]),
    "mg_solve_level_noalloc": (C.c_int, [C.c_int, C.c_int, C.c_double, C.c_double, _vp, _vp,
                                         C.POINTER(mg_options), C.POINTER(mg_level_stats)]),
    "mg_profile_read": (C.c_int, [_vp, C.POINTER(mg_kernel_stat), C.c_int]),
    "mg_persistent_count": (C.c_int, [_vp]),
    "mg_box_create": (C.c_int, [C.POINTER(mg_box_desc), C.POINTER(mg_options), C.POINTER(_vp)]),
    "mg_box_set_density": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp]),
    "mg_box_solve": (C.c_int, [_vp, C.POINTER(mg_level_stats)]),
    "mg_box_forces": (C.c_int, [_vp, C.c_int, _vp, _vp]),
    "mg_box_level_sizes": (C.c_int, [_vp, C.c_int, C.POINTER(C.c_int), C.c_int]),
    "mg_box_time_smoothing": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double),
                                        C.POINTER(C.c_double)]),
    "mg_box_error_message": (C.c_char_p, [_vp]),
    "mg_box_destroy": (C.c_int, [_vp]),
}


def _load():
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


LIB = _load()
LIB_PATH = _build.LIB


class MGError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{LIB.mg_status_str(status).decode()}: {msg}")
        self.status = status


def _addr(a):
    """Address of a contiguous float64 buffer (torch tensor, numpy array, int or None)."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if isinstance(a, np.ndarray):
        assert a.dtype == np.float64 and a.flags.c_contiguous, "need contiguous float64"
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        import torch
        assert a.dtype == torch.float64 and a.is_contiguous(), "need contiguous float64"
        return a.data_ptr()
    raise TypeError(type(a))


# ---------------------------------------------------------------------------
# the C entry points, same names
# ---------------------------------------------------------------------------
def mg_default_options():
    o = mg_options()
    LIB.mg_default_options(C.byref(o))
    return o


def mg_level_sizes(M):
    buf = (C.c_int * 64)()
    k = LIB.mg_level_sizes(int(M), buf, 64)
    return [buf[i] for i in range(k)]


def mg_status_str(s):
    return LIB.mg_status_str(int(s)).decode()


def mg_error_message(h=None):
    return LIB.mg_error_message(h).decode()


def mg_create_hierarchy(descs, opt=None):
    """descs: sequence of mg_hierarchy_desc; returns the opaque handle (int)."""
    arr = (mg_hierarchy_desc * len(descs))(*descs)
    h = _vp()
    s = LIB.mg_create_hierarchy(arr, len(descs), C.byref(opt) if opt is not None else None, C.byref(h))
    if s != MG_OK:
        raise MGError(s, mg_error_message(None))
    return h.value


def _check(h, s, ok=(MG_OK,)):
    if s not in ok:
        raise MGError(s, mg_error_message(h))
    return s


def mg_set_density(h, b, level, rho, bc_rho=None, bc_phi=None):
    return _check(h, LIB.mg_set_density(h, b, level, _addr(rho), _addr(bc_rho), _addr(bc_phi)))


def mg_set_guess(h, b, level, phi0):
    return _check(h, LIB.mg_set_guess(h, b, level, _addr(phi0)))


def mg_solve(h, batch, allow_noconv=False):
    """Returns (status, stats) with stats a (batch, MG_MAX_LEVELS) list of dicts."""
    st = (mg_level_stats * (batch * MG_MAX_LEVELS))()
    s = LIB.mg_solve(h, st)
    _check(h, s, (MG_OK, MG_ENOCONV) if allow_noconv else (MG_OK,))
    out = [[{"cycles": st[b * MG_MAX_LEVELS + l].cycles, "outer_steps": st[b * MG_MAX_LEVELS + l].outer_steps,
             "rel_res": st[b * MG_MAX_LEVELS + l].rel_res, "b_norm": st[b * MG_MAX_LEVELS + l].b_norm,
             "status": st[b * MG_MAX_LEVELS + l].status} for l in range(MG_MAX_LEVELS)] for b in range(batch)]
    return s, out


def mg_forces(h, b, level, phi_out=None, F_out=None):
    return _check(h, LIB.mg_forces(h, b, level, _addr(phi_out), _addr(F_out)))


def mg_set_outputs(h, b, level, phi_out=None, F_out=None):
    """Arrays (device or page-locked host) that mg_solve fills with the
    level's potential and forces; None, None unregisters."""
    return _check(h, LIB.mg_set_outputs(h, b, level, _addr(phi_out), _addr(F_out)))


def mg_profile(h, enable):
    return _check(h, LIB.mg_profile(h, 1 if enable else 0))


def mg_profile_read(h):
    """{kernel name: (launches, ms, algorithmic bytes)}."""
    buf = (mg_kernel_stat * 32)()
    k = LIB.mg_profile_read(h, buf, 32)
    if k < 0:
        raise MGError(MG_ESTATE, mg_error_message(h))
    return {buf[i].name.decode(): (buf[i].launches, buf[i].ms, buf[i].bytes) for i in range(k)}


def mg_solve_level_noalloc(dim, n, h, G, rho, phi, opt=None):
    """Allocation-free single-level solve (device (n+4)^d blocks); returns (status, stats dict)."""
    st = mg_level_stats()
    s = LIB.mg_solve_level_noalloc(dim, n, h, G, _addr(rho), _addr(phi),
                                   C.byref(opt) if opt is not None else None, C.byref(st))
    return s, {"cycles": st.cycles, "rel_res": st.rel_res, "b_norm": st.b_norm, "status": st.status}


def mg_autotune(h, cache_path=None):
    return _check(h, LIB.mg_autotune(h, cache_path.encode() if cache_path else None))


def mg_tuning(h, b, level):
    """(tiles per multigrid level, edge of the first one-block level)."""
    buf = (C.c_int * 16)()
    nb = LIB.mg_tuning(h, b, level, buf, 16)
    return [buf[i] for i in range(16)], nb


def mg_time_smoothing(h, b, level, L, launches):
    """(microseconds per launch, algorithmic bytes per launch) of multigrid
    level L's smoothing, timed as the solve graph launches it."""
    us, by = C.c_double(), C.c_double()
    _check(h, LIB.mg_time_smoothing(h, b, level, L, launches, C.byref(us), C.byref(by)))
    return us.value, by.value


def mg_persistent_count(h):
    """Hierarchies the solve graph gives to the persistent launch (-1: no graph yet)."""
    return LIB.mg_persistent_count(h)


def mg_destroy(h):
    return LIB.mg_destroy(h)


# box (non-cubic) patches, include/mg_box.h
def mg_box_error_message(b=None):
    return LIB.mg_box_error_message(b).decode()


def _bcheck(b, s, ok=(MG_OK,)):
    if s not in ok:
        raise MGError(s, mg_box_error_message(b))
    return s


def mg_box_create(desc, opt=None):
    """desc: mg_box_desc; returns the opaque handle (int)."""
    b = _vp()
    s = LIB.mg_box_create(C.byref(desc), C.byref(opt) if opt is not None else None, C.byref(b))
    if s != MG_OK:
        raise MGError(s, mg_box_error_message(None))
    return b.value


def mg_box_set_density(b, patch, rho, bc_rho=None, bc_phi=None):
    return _bcheck(b, LIB.mg_box_set_density(b, patch, _addr(rho), _addr(bc_rho), _addr(bc_phi)))


def mg_box_solve(b, num_patches, allow_noconv=False):
    """Returns (status, stats) with stats a list of one dict per patch."""
    st = (mg_level_stats * num_patches)()
    s = LIB.mg_box_solve(b, st)
    _bcheck(b, s, (MG_OK, MG_ENOCONV) if allow_noconv else (MG_OK,))
    return s, [{"cycles": st[l].cycles, "outer_steps": st[l].outer_steps, "rel_res": st[l].rel_res,
                "b_norm": st[l].b_norm, "status": st[l].status} for l in range(num_patches)]


def mg_box_forces(b, patch, phi_out=None, F_out=None):
    return _bcheck(b, LIB.mg_box_forces(b, patch, _addr(phi_out), _addr(F_out)))


def mg_box_level_sizes(b, patch):
    """[(N_x, N_y, N_z)] per multigrid level of the patch."""
    buf = (C.c_int * (3 * 64))()
    k = LIB.mg_box_level_sizes(b, patch, buf, 64)
    if k < 0:
        raise MGError(MG_EINVAL, "mg_box_level_sizes")
    return [tuple(buf[3 * L + a] for a in range(3)) for L in range(k)]


def mg_box_time_smoothing(b, patch, L, launches):
    """(microseconds per colour pass, algorithmic bytes per pass) on multigrid level L."""
    us, by = C.c_double(), C.c_double()
    _bcheck(b, LIB.mg_box_time_smoothing(b, patch, L, launches, C.byref(us), C.byref(by)))
    return us.value, by.value


def mg_box_destroy(b):
    return LIB.mg_box_destroy(b)


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------
def desc_from(H):
    """mg_hierarchy_desc from an inputs.Hierarchy."""
    d = mg_hierarchy_desc()
    d.dim = H.dim
    d.num_levels = H.num_levels
    for l in range(H.num_levels):
        d.n[l] = H.n[l]
        for a in range(H.dim):
            d.lo[l][a] = H.lo[l][a]
    d.h0 = H.h0
    d.G = H.G
    if getattr(H, "parents", None) is not None:
        d.tree = 1
        for l in range(1, H.num_levels):
            d.parent[l] = H.parent(l)
    return d


def box_desc_from(H):
    """mg_box_desc from an inputs.BoxHierarchy."""
    d = mg_box_desc()
    d.dim = H.dim
    d.num_patches = H.num_levels
    for l in range(H.num_levels):
        for a in range(H.dim):
            d.n[l][a] = H.n[l][a]
            d.lo[l][a] = H.lo[l][a]
    d.h0 = H.h0
    d.G = H.G
    if getattr(H, "parents", None) is not None:
        d.tree = 1
        for l in range(1, H.num_levels):
            d.parent[l] = H.parent(l)
    return d


def options(**kw):
    o = mg_default_options()
    for k, v in kw.items():
        if k == "stream" and v is not None and not isinstance(v, int):
            v = v.cuda_stream  # torch.cuda.Stream
        setattr(o, k, v)
    return o
