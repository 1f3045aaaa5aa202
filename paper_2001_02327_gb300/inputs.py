"""Seeded synthetic inputs for the nested-grid Poisson solver.

This module builds the *inputs* of the method and the analytic references
its results are checked against; it holds none of the method's own arithmetic
(no smoother, transfer, interface or force stencil).  Both the CUDA path and
the CPU oracle are fed from here.

Geometry (Sec. 2.1): level l is a square/cubic patch Omega^l of n_l cells per
edge with lower corner lo_l and cell size h_l = h0 / 2^l; each patch is
immersed in its parent and aligned to the parent's cell faces.  Densities are
point values at cell centres (Sec. 2.1, last sentence).

Analytic density/potential pairs, all with  lap(Phi) = 4 pi G rho  (Eq. 1):
  * ``PolySphere`` -- rho = rho0 (1 - r^2/R^2)^m inside R (3D).  For m = 2,
    rho0 = 1, R = 0.25, G = 1 this is the paper's 3D model (Sec. 3.2).
  * ``PolyDisk``   -- the same profile in 2D (logarithmic potential).
  * ``SoftDisk2D`` -- the paper's 2D model (Sec. 3.1): sigma =
    4 R0^2/(R^2+R0^2)^2 with G = 1/(4 pi), Phi = ln((R/R0)^2 + 1).
Forces are F = -grad(Phi) (Eq. 1 and the sentence after it).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from math import comb, pi

import numpy as np

BASE_SEED = 2001023270


# --------------------------------------------------------------------------
# analytic sources
# --------------------------------------------------------------------------
@dataclass
class PolySphere:
    """rho = rho0 (1-u^2)^m for u = |x-c|/R < 1 (3D).

    Enclosed mass M(r) = 4 pi rho0 R^3 sum_j C(m,j) (-1)^j u^(2j+3)/(2j+3);
    Phi = -G M(r)/r - 4 pi G rho0 R^2 (1-u^2)^(m+1) / (2(m+1)) inside,
    -G M/r outside;  F = -G M(r) (x-c)/r^3.
    """
    centre: tuple
    R: float
    rho0: float = 1.0
    m: int = 2

    @staticmethod
    def mass_factor(m: int) -> float:
        """M_total / (4 pi rho0 R^3)."""
        return sum(comb(m, j) * (-1) ** j / (2 * j + 3) for j in range(m + 1))

    @classmethod
    def from_mass(cls, centre, R, mass, m=3):
        return cls(tuple(centre), R, mass / (4 * pi * R ** 3 * cls.mass_factor(m)), m)

    @property
    def mass(self) -> float:
        return 4 * pi * self.rho0 * self.R ** 3 * self.mass_factor(self.m)

    def _r(self, X):
        d = X - np.asarray(self.centre, dtype=np.float64)
        return d, np.sqrt(np.sum(d * d, axis=-1))

    def density(self, X):
        _, r = self._r(X)
        u2 = (r / self.R) ** 2
        return np.where(u2 < 1.0, self.rho0 * np.clip(1.0 - u2, 0, None) ** self.m, 0.0)

    def _m_over_r3(self, r):
        """G-free M(r)/r^3, regular at r = 0."""
        R, m = self.R, self.m
        u = np.minimum(r / R, 1.0)
        s = sum(comb(m, j) * (-1) ** j * u ** (2 * j) / (2 * j + 3) for j in range(m + 1))
        inside = 4 * pi * self.rho0 * s
        outside = self.mass / np.maximum(r, 1e-100) ** 3
        return np.where(r < R, inside, outside)

    def potential(self, X, G):
        _, r = self._r(X)
        R, m = self.R, self.m
        u = np.minimum(r / R, 1.0)
        s = sum(comb(m, j) * (-1) ** j * u ** (2 * j + 2) / (2 * j + 3) for j in range(m + 1))
        m_over_r_in = 4 * pi * self.rho0 * R ** 2 * s
        inside = -G * m_over_r_in - 4 * pi * G * self.rho0 * R ** 2 * (1 - u * u) ** (m + 1) / (2 * (m + 1))
        outside = -G * self.mass / np.maximum(r, 1e-300)
        return np.where(r < R, inside, outside)

    def force(self, X, G):
        d, r = self._r(X)
        return -G * self._m_over_r3(r)[..., None] * d


@dataclass
class PolyDisk:
    """2D analogue: rho = rho0 (1-u^2)^m, m(r) = int_0^r rho r' dr',
    grad Phi = 4 pi G m(r) (x-c)/r^2, Phi = 4 pi G m(R) ln r outside."""
    centre: tuple
    R: float
    rho0: float = 1.0
    m: int = 4

    def _r(self, X):
        d = X - np.asarray(self.centre, dtype=np.float64)
        return d, np.sqrt(np.sum(d * d, axis=-1))

    def density(self, X):
        _, r = self._r(X)
        u2 = (r / self.R) ** 2
        return np.where(u2 < 1.0, self.rho0 * np.clip(1.0 - u2, 0, None) ** self.m, 0.0)

    def _mR(self):
        return self.rho0 * self.R ** 2 / (2 * (self.m + 1))

    def potential(self, X, G):
        _, r = self._r(X)
        R, m = self.R, self.m
        u = np.minimum(r / R, 1.0)
        s = sum(comb(m + 1, j) * (-1) ** (j + 1) * (1 - u ** (2 * j)) / j for j in range(1, m + 2))
        inside = 4 * pi * G * (self._mR() * np.log(R) - self.rho0 * R ** 2 / (4 * (m + 1)) * s)
        outside = 4 * pi * G * self._mR() * np.log(np.maximum(r, 1e-300))
        return np.where(r < R, inside, outside)

    def force(self, X, G):
        d, r = self._r(X)
        R, m = self.R, self.m
        u2 = np.minimum((r / R) ** 2, 1.0)
        # m(r)/r^2 regular at 0: m(r) = rho0 R^2 (1-(1-u^2)^(m+1)) / (2(m+1))
        #   (1-(1-v)^(m+1))/v = sum_{j>=1} C(m+1,j)(-1)^(j+1) v^(j-1)
        s = sum(comb(m + 1, j) * (-1) ** (j + 1) * u2 ** (j - 1) for j in range(1, m + 2))
        m_over_r2_in = self.rho0 / (2 * (m + 1)) * s
        m_over_r2_out = self._mR() / np.maximum(r, 1e-100) ** 2
        m_over_r2 = np.where(r < R, m_over_r2_in, m_over_r2_out)
        return -4 * pi * G * m_over_r2[..., None] * d


@dataclass
class SoftDisk2D:
    """The paper's 2D model (Sec. 3.1); valid with G = 1/(4 pi)."""
    R0: float = 0.3

    def density(self, X):
        R2 = np.sum(X * X, axis=-1)
        return 4 * self.R0 ** 2 / (R2 + self.R0 ** 2) ** 2

    def potential(self, X, G):
        R2 = np.sum(X * X, axis=-1)
        return np.log(R2 / self.R0 ** 2 + 1.0) * (4 * pi * G)

    def force(self, X, G):
        R2 = np.sum(X * X, axis=-1)
        return -(4 * pi * G) * (2.0 / (R2 + self.R0 ** 2))[..., None] * X


# --------------------------------------------------------------------------
# nested hierarchy description
# --------------------------------------------------------------------------
@dataclass
class Hierarchy:
    dim: int
    n: list
    lo: list          # per level, tuple of length dim
    h0: float
    G: float
    sources: list = field(default_factory=list)
    name: str = ""
    parents: list = None   # parent patch of each patch (None: a chain, parent of l is l-1)

    @property
    def num_levels(self):
        """Number of patches (in a chain: refinement levels)."""
        return len(self.n)

    def parent(self, l):
        return l - 1 if self.parents is None else self.parents[l]

    def children(self, l):
        return [c for c in range(1, self.num_levels) if self.parent(c) == l]

    def depth(self, l):
        k = 0
        while l > 0:
            l = self.parent(l)
            k += 1
        return k

    def h(self, l):
        return self.h0 / 2.0 ** self.depth(l)

    def offset(self, l):
        """Lower corner of patch l in parent cells (integer, Sec. 2.1 nesting)."""
        p = self.parent(l)
        off = [(self.lo[l][a] - self.lo[p][a]) / self.h(p) for a in range(self.dim)]
        ioff = [int(round(o)) for o in off]
        assert all(abs(o - i) < 1e-9 for o, i in zip(off, ioff)), "patch not aligned to parent faces"
        return ioff

    def zones(self):
        return sum(n ** self.dim for n in self.n)

    def validate(self):
        for l in range(1, self.num_levels):
            assert 0 <= self.parent(l) < l, l
            o = self.offset(l)
            nl, np_ = self.n[l], self.n[self.parent(l)]
            assert nl % 2 == 0
            for a in range(self.dim):
                assert 1 <= o[a] <= np_ - nl // 2 - 1, (l, a, o[a])

    # field evaluation ------------------------------------------------------
    def centres(self, l, pad):
        """Cell centres of level l over a (n+2*pad)^d block; shape (...,dim), C order (z,y,x)."""
        n, h = self.n[l], self.h(l)
        ax = [self.lo[l][a] + (np.arange(-pad, n + pad) + 0.5) * h for a in range(self.dim)]
        grids = np.meshgrid(*ax[::-1], indexing="ij")  # z,y,x order
        return np.stack(grids[::-1], axis=-1)          # last axis = (x,y,z)

    def density(self, X):
        return sum(s.density(X) for s in self.sources)

    def potential(self, X):
        return sum(s.potential(X, self.G) for s in self.sources)

    def force(self, X):
        return sum(s.force(X, self.G) for s in self.sources)


class BoxHierarchy(Hierarchy):
    """A hierarchy of box (non-cubic) patches: n[l] is a tuple of cells per
    axis (x, y[, z]); everything else as in Hierarchy."""

    def centres(self, l, pad):
        """Cell centres of patch l over a block of n_a + 2 pad cells per axis;
        shape (..., dim), C order (z, y, x)."""
        h = self.h(l)
        ax = [self.lo[l][a] + (np.arange(-pad, self.n[l][a] + pad) + 0.5) * h for a in range(self.dim)]
        grids = np.meshgrid(*ax[::-1], indexing="ij")
        return np.stack(grids[::-1], axis=-1)

    def zones(self):
        return sum(int(np.prod(n)) for n in self.n)

    def validate(self):
        for l in range(1, self.num_levels):
            assert 0 <= self.parent(l) < l, l
            o = self.offset(l)
            nl, np_ = self.n[l], self.n[self.parent(l)]
            for a in range(self.dim):
                assert nl[a] % 2 == 0
                assert 1 <= o[a] <= np_[a] - nl[a] // 2 - 1, (l, a, o[a])


def nested_boxes(dim, n_levels, n, half_widths, G, sources, name="", centre=0.0):
    """Base box [c - w_a, c + w_a] with n = (n_x, n_y[, n_z]) cells of one size;
    each finer patch halves the box about the centre (same cell counts)."""
    h0 = 2.0 * half_widths[0] / n[0]
    assert all(abs(2.0 * half_widths[a] / n[a] - h0) < 1e-12 * h0 for a in range(dim)), "cells must be cubes"
    lo = []
    for l in range(n_levels):
        hl = h0 / 2 ** l
        lo.append(tuple(centre - n[a] * hl / 2.0 for a in range(dim)))
    H = BoxHierarchy(dim, [tuple(n)] * n_levels, lo, h0, G, list(sources), name)
    H.validate()
    return H


def box_3d_sphere(n=(24, 32, 16), levels=3):
    """3D box patches: base of n cells (one cell size) centred on an offset
    compact sphere rho = (1 - r^2/R^2)^3, R = 0.3 at (0.05, 0.03, 0.02); G = 1;
    each finer patch halves the box."""
    h0 = 2.0 / max(n)
    hw = [0.5 * na * h0 for na in n]
    return nested_boxes(3, levels, n, hw, 1.0, [PolySphere((0.05, 0.03, 0.02), 0.3, 1.0, 3)],
                        f"box3d_{levels}x{'x'.join(map(str, n))}")


def box_2d_disk(n=(48, 24), levels=3):
    """2D box patches around the compact disk rho = (1 - r^2/R^2)^4, R = 0.5."""
    h0 = 2.0 / max(n)
    hw = [0.5 * na * h0 for na in n]
    return nested_boxes(2, levels, n, hw, 1.0, [PolyDisk((0.0, 0.0), 0.5, 1.0, 4)],
                        f"box2d_{levels}x{'x'.join(map(str, n))}")


def nested_centred(dim, n_levels, n, half_width, G, sources, name="", centre=0.0):
    """Base [c-w, c+w]^d with n cells; each finer level halves the box (same n)."""
    ns = [n] * n_levels if np.isscalar(n) else list(n)
    h0 = 2.0 * half_width / ns[0]
    lo = []
    for l in range(n_levels):
        hl = h0 / 2 ** l
        lo.append(tuple([centre - ns[l] * hl / 2.0] * dim))
    H = Hierarchy(dim, ns, lo, h0, G, list(sources), name)
    H.validate()
    return H


# --------------------------------------------------------------------------
# the workloads
# --------------------------------------------------------------------------
def paper_2d(N, levels=4):
    """Sec. 3.1: G=1/(4pi), R0=0.3, Omega^0=[-0.5,0.5]^2, levels 0..3, N per level."""
    return nested_centred(2, levels, N, 0.5, 1.0 / (4 * pi), [SoftDisk2D(0.3)], f"paper2d_N{N}")


def paper_3d(N, levels=3):
    """Sec. 3.2: G=1, rho=(1-r^2/r0^2)^2, r0=0.25, Omega^0=[-0.5,0.5]^3, levels 0..2."""
    return nested_centred(3, levels, N, 0.5, 1.0, [PolySphere((0.0, 0.0, 0.0), 0.25, 1.0, 2)], f"paper3d_N{N}")


def config_2d_disk(n=64, levels=3):
    """2D: base 64^2 on [-1,1]^2 + 2 nested levels; rho=(1-r^2/R^2)^4, R=0.5, G=1."""
    return nested_centred(2, levels, n, 1.0, 1.0, [PolyDisk((0.0, 0.0), 0.5, 1.0, 4)], f"disk2d_{levels}x{n}")


def config_3d_offset_sphere(n=64, levels=4):
    """3D: base n^3 on [-1,1]^3 + 3 nested levels; rho=(1-r^2/R^2)^3, R=0.3,
    centred at (0.05,0.03,0.02); G=1."""
    return nested_centred(3, levels, n, 1.0, 1.0, [PolySphere((0.05, 0.03, 0.02), 0.3, 1.0, 3)],
                          f"sphere3d_{levels}x{n}")


def random_spheres(rng, count, box_lo, box_hi, r_frac=(0.02, 0.1), edge=2.0, mass=(0.5, 2.0), m=3):
    out = []
    for _ in range(count):
        c = tuple(rng.uniform(box_lo, box_hi, size=3))
        R = rng.uniform(*r_frac) * edge
        M = rng.uniform(*mass)
        out.append(PolySphere.from_mass(c, R, M, m))
    return out


def config_3d_spheres(n=256, levels=4, count=8, seed=BASE_SEED):
    """3D at scale: n^3 per level, 4 nested levels on [-1,1]^3; sum of `count`
    compact spheres, centres uniform in the finest box, radii U[0.02,0.1] of
    the base edge, masses U[0.5,2]."""
    rng = np.random.default_rng(seed)
    w = 2.0 ** (-(levels - 1))
    sph = random_spheres(rng, count, -w, w)
    return nested_centred(3, levels, n, 1.0, 1.0, sph, f"spheres3d_{levels}x{n}_s{seed}")


def config_3d_patches(n=64, m=32, seed=BASE_SEED):
    """Patch-based refinement: base n^3 on [-1,1]^3, two disjoint m^3 patches
    on level 1 (one per compact sphere), and an m^3 patch inside the first.
    Patches are listed parents first."""
    h0 = 2.0 / n
    w = m // 2                               # patch width in parent cells
    o1 = (n // 8, n // 2 - w // 2, n // 2 - w // 2)
    o2 = (n - n // 8 - w, n // 2 - w // 2, n // 2 - w // 2)
    lo1 = tuple(-1.0 + o * h0 for o in o1)
    lo2 = tuple(-1.0 + o * h0 for o in o2)
    h1 = h0 / 2
    o3 = (m // 4,) * 3
    lo3 = tuple(l + o * h1 for l, o in zip(lo1, o3))
    c1 = tuple(l + (w * h0) / 2 for l in lo1)
    c2 = tuple(l + (w * h0) / 2 for l in lo2)
    sph = [PolySphere(c1, 0.2, 1.0, 3), PolySphere(c2, 0.18, 1.5, 3)]
    H = Hierarchy(3, [n, m, m, m], [(-1.0,) * 3, lo1, lo2, lo3], h0, 1.0, sph, f"patches3d_{n}_{m}",
                  parents=[-1, 0, 0, 1])
    H.validate()
    return H


EDGES = (32, 48, 64, 96, 128)


def random_hierarchy(seed, edges=EDGES):
    """One hierarchy of the uneven batch: 2-4 levels, edges from `edges`
    (rejected against the nesting constraint), 1-4 spheres in the finest box."""
    rng = np.random.default_rng(seed)
    nl = int(rng.integers(2, 5))
    while True:
        ns = [int(rng.choice(edges)) for _ in range(nl)]
        # centred child: offset (n_p - n_c/2)/2 parent cells must be a whole
        # number in [1, n_p - n_c/2 - 1]  <=>  n_p - n_c/2 even and >= 2
        if all((ns[l - 1] - ns[l] // 2) % 2 == 0 and ns[l - 1] - ns[l] // 2 >= 2 for l in range(1, nl)):
            break
    h0 = 2.0 / ns[0]
    lo = [tuple([-1.0] * 3)]
    for l in range(1, nl):
        hp = h0 / 2 ** (l - 1)
        off = (ns[l - 1] - ns[l] // 2) // 2
        lo.append(tuple([lo[l - 1][0] + off * hp] * 3))
    w_lo = lo[-1][0]
    w_hi = w_lo + ns[-1] * h0 / 2 ** (nl - 1)
    sph = random_spheres(rng, int(rng.integers(1, 5)), w_lo, w_hi)
    H = Hierarchy(3, ns, lo, h0, 1.0, sph, f"rand_s{seed}")
    H.validate()
    return H


# --------------------------------------------------------------------------
# arrays handed to a solver
# --------------------------------------------------------------------------
def level_inputs(H: Hierarchy):
    """Per level: rho on Omega^l (n^d, C order), and for level 0 the boundary
    data the caller owns: rho at the centres of Gamma^0 ((n+2)^d; only its
    inner ring is read) and Phi at the centres of the (n+4)^d block (only its
    outer ring is read)."""
    out = []
    for l in range(H.num_levels):
        d = {"rho": np.ascontiguousarray(H.density(H.centres(l, 0)))}
        if l == 0:
            d["bc_rho"] = np.ascontiguousarray(H.density(H.centres(0, 1)))
            d["bc_phi"] = np.ascontiguousarray(H.potential(H.centres(0, 2)))
        out.append(d)
    return out
