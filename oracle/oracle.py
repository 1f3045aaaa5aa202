"""Python driver of the CPU FP64 oracle (TEST INFRASTRUCTURE ONLY).

Only the tests, the package smoke check and the benchmark's CPU-baseline /
reference arm may import this module.  It loads ``liboracle.so`` (compiled
from ``mg_oracle.c`` with ``-O2 -ffp-contract=off``) and strings its pieces
together in the order the paper gives:

  levels are solved coarse to fine (one-way scheme, Sec. 2.1); level 0 takes
  its buffer data from the caller; every finer level takes its outer-ring
  potential and inner-ring density from its parent by linear interpolation,
  and its initial potential likewise (Sec. 2.4); each level is solved by
  multigrid V-cycles (Sec. 2.3); forces follow from Eq. 2.

It shares no code with the CUDA path.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from math import pi

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "mg_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

_lib = None


def build(force=False):
    """Compile the oracle (plain C, no FMA contraction)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-std=c99", "-shared", "-fPIC",
                               "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
        ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
        L.or_mg_sizes.argtypes = [C.c_int, ip, C.c_int]
        L.or_mg_sizes.restype = C.c_int
        L.or_level_solve.argtypes = [C.c_int, C.c_int, C.c_double, dp, dp, C.c_double,
                                     C.c_int, C.c_int, C.c_int, C.c_double, dp, C.c_int, C.c_int]
        L.or_level_solve.restype = C.c_int
        L.or_residual_norm.argtypes = [C.c_int, C.c_int, C.c_double, dp, dp, C.c_double]
        L.or_residual_norm.restype = C.c_double
        L.or_interface_fill.argtypes = [C.c_int, C.c_int, dp, dp, C.c_int, ip, dp, dp, C.c_int]
        L.or_interface_fill.restype = None
        L.or_forces.argtypes = [C.c_int, C.c_int, C.c_double, dp, dp, C.c_int]
        L.or_forces.restype = None
        L.or_fill_ghosts.argtypes = [C.c_int, C.c_int, C.c_int, dp]
        L.or_fill_ghosts.restype = C.c_int
        L.or_mg_residual.argtypes = [C.c_int, C.c_int, C.c_int, dp, dp, dp]
        L.or_mg_residual.restype = C.c_int
        L.or_mg_restrict.argtypes = [C.c_int, C.c_int, C.c_int, dp, dp]
        L.or_mg_restrict.restype = C.c_int
        L.or_mg_prolong.argtypes = [C.c_int, C.c_int, C.c_int, dp, dp]
        L.or_mg_prolong.restype = C.c_int
        _lib = L
    return _lib


def mg_sizes(M):
    """Multigrid level sizes N^L for a Gamma of M cells per edge (Sec. 2.2)."""
    buf = np.zeros(64, dtype=np.int32)
    k = lib().or_mg_sizes(int(M), buf, 64)
    return [int(v) for v in buf[:k]]


def mg_restrict(dim, M, L, rf):
    """The restriction of Sec. 2.3 step 5 from multigrid level L to L+1 of a
    Gamma of M cells (test hook): returns the (N^{L+1}+2)^d coarse array."""
    Nc = mg_sizes(M)[L + 1]
    fc = np.zeros((Nc + 2,) * dim)
    assert lib().or_mg_restrict(dim, M, L, np.ascontiguousarray(rf, dtype=np.float64), fc) == Nc
    return fc


def mg_prolong(dim, M, L, phic, phif):
    """Prolongation and correction of Sec. 2.3 step 10 from level L+1 to L
    (test hook): phic's ghost layer is filled by the rule of Sec. 2.4, then
    phif (modified in place) += P(phic) on its active cells."""
    assert lib().or_mg_prolong(dim, M, L, phic, phif) == phic.shape[0] - 2


def level_solve(dim, n, h, phi, rho, fourpiG, nu_pre=2, nu_post=1, max_cycles=50, rel_tol=1e-10, stop=0,
                stencil=0):
    """Solve one refinement level in place; returns (cycles, history of the
    stopping quantity).  stop=0: relative residual over Gamma; stop=1: the
    largest change of the acceleration on Omega between cycles (Sec. 3)."""
    assert phi.shape == (n + 4,) * dim and rho.shape == (n + 4,) * dim
    hist = np.zeros(max_cycles + 1, dtype=np.float64)
    c = lib().or_level_solve(dim, n, h, phi, rho, fourpiG, nu_pre, nu_post, max_cycles, rel_tol, hist, stop,
                             stencil)
    return c, hist[:c + 1]


def residual_norm(dim, n, h, phi, rho, fourpiG):
    return lib().or_residual_norm(dim, n, h, phi, rho, fourpiG)


def interface_fill(dim, n_p, phi_p, rho_p, n_c, off, phi_c, rho_c, guess=True):
    off = np.ascontiguousarray(off, dtype=np.int32)
    lib().or_interface_fill(dim, n_p, phi_p, rho_p, n_c, off, phi_c, rho_c, 1 if guess else 0)


def forces(dim, n, h, phi, stencil=0):
    F = np.zeros((dim,) + (n,) * dim, dtype=np.float64)
    lib().or_forces(dim, n, h, phi, F, stencil)
    return F


def fill_ghosts(dim, M, L, phi):
    """Apply the multigrid ghost rule of Sec. 2.4 to an (N^L+2)^d array in place."""
    return lib().or_fill_ghosts(dim, M, L, phi)


def mg_residual(dim, M, L, phi, f):
    """f - lap(Phi) on multigrid level L (unit fine cell size), (N^L+2)^d arrays."""
    r = np.zeros_like(phi)
    lib().or_mg_residual(dim, M, L, phi, f, r)
    return r


def pad_into(block, interior, width):
    """Write `interior` into the centre of `block`, leaving `width` cells per side."""
    sl = tuple(slice(width, width + s) for s in interior.shape)
    block[sl] = interior


def solve_hierarchy(H, inputs, nu_pre=2, nu_post=1, max_cycles=50, rel_tol=1e-10, guess="interp",
                    force_stencil=0, interface="buffer", stop="residual"):
    """Solve a nested hierarchy coarse to fine.

    ``inputs`` is the per-level list from ``inputs.level_inputs``.  Returns a
    list of dicts with ``phi`` ((n+4)^d block after the solve), ``rho``
    ((n+4)^d block actually used), ``F`` ((dim, n^d)), ``cycles``, ``hist``.

    ``interface="buffer"`` is the method of Sec. 2.1: the inner buffer ring is
    solved with the patch.  ``interface="frozen"`` is the scheme Sec. 4 and
    Fig. 4 compare against: on levels l > 0 both buffer rings hold potential
    linearly interpolated from level l-1, and multigrid solves Omega alone
    with the inner ring as its Dirichlet boundary (M = n active cells).

    ``stop="residual"`` ends a level when ||b - A Phi|| / ||b|| < rel_tol;
    ``stop="force"`` when the acceleration on Omega changes by less than
    rel_tol between cycles (the test of Sec. 3.1 and 3.2).
    """
    assert interface in ("buffer", "frozen") and stop in ("residual", "force")
    assert not (interface == "frozen" and stop == "force")
    sflag = 1 if stop == "force" else 0
    dim = H.dim
    fourpiG = 4.0 * pi * H.G
    out = []
    for l in range(H.num_levels):
        n, h = H.n[l], H.h(l)
        phi = np.zeros((n + 4,) * dim)
        rho = np.zeros((n + 4,) * dim)
        if l == 0:
            # caller-owned buffer data of the base level: outer-ring potential
            # and inner-ring density (Gamma gets a zero initial guess)
            phi[...] = inputs[0]["bc_phi"]
            pad_into(rho, inputs[0]["bc_rho"], 1)
            inner = tuple(slice(1, n + 3) for _ in range(dim))
            phi[inner] = 0.0
        else:
            P = out[H.parent(l)]
            interface_fill(dim, H.n[H.parent(l)], P["phi"], P["rho"], n, H.offset(l), phi, rho,
                           guess=(guess == "interp"))
        pad_into(rho, inputs[l]["rho"], 2)
        if l > 0 and interface == "frozen":
            # inner-ring potential by the same linear interpolation as the outer ring
            ring_phi, ring_rho = np.zeros_like(phi), np.zeros_like(rho)
            interface_fill(dim, H.n[H.parent(l)], P["phi"], P["rho"], n, H.offset(l), ring_phi, ring_rho, guess=True)
            gam = tuple(slice(1, n + 3) for _ in range(dim))
            om = tuple(slice(2, n + 2) for _ in range(dim))
            keep = phi[om].copy()
            phi[gam] = ring_phi[gam]
            phi[om] = keep
            sub_phi, sub_rho = phi[gam].copy(), rho[gam].copy()
            cyc, hist = level_solve(dim, n - 2, h, sub_phi, sub_rho, fourpiG, nu_pre, nu_post, max_cycles, rel_tol)
            phi[gam] = sub_phi
        else:
            cyc, hist = level_solve(dim, n, h, phi, rho, fourpiG, nu_pre, nu_post, max_cycles, rel_tol, sflag,
                                    force_stencil)
        F = forces(dim, n, h, phi, force_stencil)
        out.append({"phi": phi, "rho": rho, "F": F, "cycles": cyc, "hist": hist})
    return out
