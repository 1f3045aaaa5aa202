"""Error norms of Sec. 3 (TEST INFRASTRUCTURE ONLY).

||F||_p = (integral over Omega of |F|^p)^(1/p), ||F||_inf = sup |F|
(Sec. 3, first equations), evaluated as cell sums weighted by the cell volume
h_l^d.  "The entire calculation domain" is read as the composite grid: the
cells of each level not covered by the next finer level; the all-cells
variant is available for comparison.
"""
from __future__ import annotations

import numpy as np


def covered_mask(H, l):
    """True on the cells of Omega^l (n^d) that a child patch covers."""
    n = H.n[l]
    mask = np.zeros((n,) * H.dim, dtype=bool)
    for c in H.children(l):
        o = H.offset(c)
        w = H.n[c] // 2
        sl = tuple(slice(o[a], o[a] + w) for a in reversed(range(H.dim)))  # C order (z,y,x)
        mask[sl] = True
    return mask


def force_errors(H, l, F):
    """Per-cell |f_x,num - f_x| and |f_R,num - f_R| with f_R = |grad Phi| (Sec. 3.1)."""
    X = H.centres(l, 0)
    Fa = H.force(X)                       # (..., dim), F = -grad Phi
    Fn = np.moveaxis(F, 0, -1)
    ex = np.abs(Fn[..., 0] - Fa[..., 0])
    eR = np.abs(np.sqrt(np.sum(Fn * Fn, axis=-1)) - np.sqrt(np.sum(Fa * Fa, axis=-1)))
    return ex, eR


def potential_error(H, l, phi_block):
    n = H.n[l]
    inner = tuple(slice(2, n + 2) for _ in range(H.dim))
    return np.abs(phi_block[inner] - H.potential(H.centres(l, 0)))


def norms(H, per_level_err, composite=True):
    """(L1, L2, Linf) of a per-level list of cellwise error arrays."""
    s1 = s2 = 0.0
    sinf = 0.0
    for l, e in enumerate(per_level_err):
        keep = ~covered_mask(H, l) if composite else np.ones_like(e, dtype=bool)
        v = H.h(l) ** H.dim
        ek = e[keep]
        s1 += np.sum(ek) * v
        s2 += np.sum(ek * ek) * v
        if ek.size:
            sinf = max(sinf, float(np.max(ek)))
    return s1, np.sqrt(s2), sinf


def hierarchy_norms(H, result, composite=True):
    """Table-1/2 style norms: dict with L1/L2/Linf of f_x, f_R and Phi errors."""
    ex, eR, ep = [], [], []
    for l, lev in enumerate(result):
        a, b = force_errors(H, l, lev["F"])
        ex.append(a)
        eR.append(b)
        ep.append(potential_error(H, l, lev["phi"]))
    out = {}
    for name, errs in (("x", ex), ("R", eR), ("phi", ep)):
        n1, n2, ni = norms(H, errs, composite)
        out[name] = (n1, n2, ni)
    return out
