"""ctypes binding of include/unet.h (the learned initial guess) and of the
solver calls that use it (mg_set_unet, mg_interp_guess).  Same names as the C
entry points; arguments are marshalled, every step runs in libmg.so."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import mg as _mg

LIB = _mg.LIB
_vp = C.c_void_p
_SIGS = {
    "mg_unet_param_count": (C.c_long, []),
    "mg_unet_create": (C.c_int, [C.c_int, C.c_int, C.c_ulonglong, _vp, C.POINTER(_vp)]),
    "mg_unet_destroy": (C.c_int, [_vp]),
    "mg_unet_get_params": (C.c_int, [_vp, _vp]),
    "mg_unet_set_params": (C.c_int, [_vp, _vp]),
    "mg_unet_get_grad": (C.c_int, [_vp, _vp]),
    "mg_unet_pack": (C.c_int, [_vp]),
    "mg_unet_forward": (C.c_int, [_vp, C.c_int, C.c_int, _vp, _vp, _vp, _vp, _vp]),
    "mg_unet_train_step": (C.c_int, [_vp, C.c_int, C.c_int, _vp, _vp, _vp, _vp, _vp, C.c_float, C.c_float,
                                     C.c_int, C.POINTER(C.c_float)]),
    "mg_unet_predict_dev": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int, _vp, _vp, _vp, _vp, C.c_int, _vp]),
    "mg_set_unet": (C.c_int, [_vp, _vp]),
    "mg_interp_guess": (C.c_int, [_vp, C.c_int, C.c_int, _vp, _vp]),
}
for _name, (_res, _args) in _SIGS.items():
    _fn = getattr(LIB, _name)
    _fn.restype = _res
    _fn.argtypes = _args


class UNetError(RuntimeError):
    pass


def _ok(r, what):
    if r != 0:
        raise UNetError(f"{what} failed with code {r}")


def mg_unet_param_count():
    return int(LIB.mg_unet_param_count())


def mg_unet_create(nmax, bmax, seed=0, stream=None):
    h = _vp()
    st = stream.cuda_stream if (stream is not None and not isinstance(stream, int)) else stream
    _ok(LIB.mg_unet_create(int(nmax), int(bmax), int(seed), st, C.byref(h)), "mg_unet_create")
    return h.value


def mg_unet_destroy(u):
    return LIB.mg_unet_destroy(u)


def mg_unet_get_params(u):
    out = np.zeros(mg_unet_param_count(), dtype=np.float32)
    _ok(LIB.mg_unet_get_params(u, out.ctypes.data), "mg_unet_get_params")
    return out


def mg_unet_set_params(u, p):
    p = np.ascontiguousarray(p, dtype=np.float32)
    assert p.size == mg_unet_param_count()
    _ok(LIB.mg_unet_set_params(u, p.ctypes.data), "mg_unet_set_params")


def mg_unet_get_grad(u):
    out = np.zeros(mg_unet_param_count(), dtype=np.float32)
    _ok(LIB.mg_unet_get_grad(u, out.ctypes.data), "mg_unet_get_grad")
    return out


def mg_unet_pack(u):
    _ok(LIB.mg_unet_pack(u), "mg_unet_pack")


def mg_unet_forward(u, B, n, rho, phi_interp, resid, frho):
    """rho, phi_interp, resid: contiguous float64 CUDA tensors (B, n, n, n);
    frho: B floats.  Returns y (B, n, n, n)."""
    fr = np.ascontiguousarray(frho, dtype=np.float64)
    y = np.zeros(B * n ** 3, dtype=np.float32)
    _ok(LIB.mg_unet_forward(u, B, n, _mg._addr(rho), _mg._addr(phi_interp), _mg._addr(resid), fr.ctypes.data,
                            y.ctypes.data), "mg_unet_forward")
    return y.reshape((B, n, n, n))


def mg_unet_train_step(u, B, n, rho, phi_interp, resid, phi_true, frho, lr=1e-3, wd=0.0, update=True):
    fr = np.ascontiguousarray(frho, dtype=np.float64)
    loss = C.c_float(0.0)
    _ok(LIB.mg_unet_train_step(u, B, n, _mg._addr(rho), _mg._addr(phi_interp), _mg._addr(resid),
                               _mg._addr(phi_true),
                               fr.ctypes.data, float(lr), float(wd), 1 if update else 0, C.byref(loss)),
        "mg_unet_train_step")
    return float(loss.value)


def mg_set_unet(h, u):
    return _mg._check(h, LIB.mg_set_unet(h, u))


def mg_interp_guess(h, b, level, out, resid_out=None):
    return _mg._check(h, LIB.mg_interp_guess(h, b, level, _mg._addr(out), _mg._addr(resid_out)))


def mg_unet_predict_dev(u, B, n, blk, rho, phi, frho_dev, resid=None, apply=True, stream=None):
    """Solver-hook form: device arrays only (phi updated in place when apply;
    resid needed for dense layouts, blk = 0)."""
    st = stream.cuda_stream if (stream is not None and not isinstance(stream, int)) else stream
    _ok(LIB.mg_unet_predict_dev(u, B, n, blk, _mg._addr(rho), _mg._addr(phi), _mg._addr(resid), _mg._addr(frho_dev),
                                1 if apply else 0, st), "mg_unet_predict_dev")
