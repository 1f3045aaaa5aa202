"""Per-axis (non-cubic) multigrid of one refinement level: plain numpy FP64.

TEST INFRASTRUCTURE ONLY: imported by tests, never by the product path, and
sharing no code with the CUDA path.

A patch of n_x x n_y [x n_z] cells (Sec. 2.1) is solved on its region Gamma of
M_a = n_a + 2 cells per axis.  Sec. 2.2 builds the multigrid sizes along one
axis (normalise Gamma to [0, 1], h^0 = 1/M, h^L = 2 h^{L-1}, N^L = round(1/h^L),
stop once N^L = 1), and the paper applies it "in x direction" and the others
alike.  Readings for a patch whose axes differ (each applied where used):

  A1  each axis follows its own sequence; once it reaches one cell it stops
      coarsening while the others go on (semi-coarsening), so a multigrid level
      L has N_a = seq_a[min(L, stop_a)] cells and cell size h 2^min(L, stop_a)
      along axis a; the hierarchy ends when every axis has one cell.
  A2  the Laplacian of a level is the sum over axes of the second differences
      divided by that axis's squared cell size; each Gauss-Seidel update solves
      the cell's own equation with the ghost rule of Sec. 2.4 folded in per axis,
      using that axis's normalised geometry (x_N of the axis).
  A3  restriction averages the children: two along an axis that coarsened from
      the finer level, one along an axis that did not (weight 1 / 2^k, k the
      coarsened axes); children beyond the fine N count zero.
  A4  prolongation uses the 3/4 - 1/4 weights along coarsened axes (the coarse
      ghosts by the rule of Sec. 2.4) and copies along the others.

With every axis equal these are the cubic method (the same sizes, stencil,
transfers and order of phases); the tests pin that case to the cubic oracle
and the non-cubic fixed point to a direct solve of the level's 5/7-point system.
"""
import numpy as np


def axis_sizes(M):
    """N^L along one axis of M cells (Sec. 2.2 items 1-4; halves rounded up)."""
    N = [M]
    L = 0
    while N[-1] > 1:
        L += 1
        N.append(int(np.floor(M / 2.0 ** L + 0.5)))
    return N


class Level:
    """Geometry of multigrid level L of a patch: per axis the cell count N, the
    cell size h, the axis's own level index la = min(L, stop), whether the
    right-most centre sits exactly at x_MG = 1 (tie) and the right-ghost
    factor cR (Sec. 2.4, linear extrapolation through zero at x_MG = 1)."""

    def __init__(self, M, h0, L):
        self.L = L
        self.N, self.h, self.la, self.tie, self.cR = [], [], [], [], []
        for Ma in M:
            seq = axis_sizes(Ma)
            la = min(L, len(seq) - 1)
            Na = seq[la]
            twoM = 2.0 * Ma
            xN2 = (2.0 * Na - 1.0) * 2.0 ** la        # x_N in units of 1/(2M)
            hL2 = 2.0 * 2.0 ** la
            tie = xN2 == twoM
            self.N.append(Na)
            self.h.append(h0 * 2.0 ** la)
            self.la.append(la)
            self.tie.append(tie)
            self.cR.append(0.0 if tie else (twoM - xN2 - hL2) / (twoM - xN2))
        self.dim = len(M)

    def shape(self):
        """storage shape, one ghost layer per side, axis order (z,) y, x"""
        return tuple(n + 2 for n in reversed(self.N))


def levels(M, h0):
    """Multigrid levels of a patch with Gamma of M = (M_x, M_y[, M_z]) cells (A1)."""
    depth = max(len(axis_sizes(Ma)) for Ma in M)
    return [Level(M, h0, L) for L in range(depth)]


def _axis_terms(lv, phi, a):
    """Along axis a (0 = x), for every active cell: the neighbour values the
    ghost rule leaves as other cells, and the coefficient of the cell itself
    that the folded ghosts add (Sec. 2.4; at L = 0 the outer ring holds data)."""
    dim = lv.dim
    ax = dim - 1 - a                                   # array axis of x_a
    N = lv.N[a]
    act = tuple(slice(1, n + 1) for n in reversed(lv.N))
    c = phi[act]

    def shifted(d):
        sl = list(act)
        sl[ax] = slice(1 + d, N + 1 + d)
        return phi[tuple(sl)]

    left, right = shifted(-1), shifted(+1)
    if lv.L == 0:
        return left + right, np.zeros_like(c)
    idx = np.arange(1, N + 1).reshape([-1 if k == ax else 1 for k in range(dim)])
    lo, hi = idx == 1, idx == N
    self_ = np.zeros_like(c)
    other = np.zeros_like(c)
    other = other + np.where(lo, 0.0, left)            # left ghost -Phi_1: on the diagonal
    self_ = self_ + np.where(lo, -1.0, 0.0)
    if lv.tie[a]:
        if N >= 2:                                     # right ghost -Phi_{N-1}
            sl = list(act)
            sl[ax] = slice(N - 1, N)
            other = other + np.where(hi, -phi[tuple(sl)], right)
        else:                                          # -Phi_0 = +Phi_1
            self_ = self_ + np.where(hi, 1.0, 0.0)
            other = other + np.where(hi, 0.0, right)
    else:                                              # right ghost cR Phi_N
        self_ = self_ + np.where(hi, lv.cR[a], 0.0)
        other = other + np.where(hi, 0.0, right)
    return other, self_


def _operator(lv, phi):
    """sum over axes of (other_a, self_a) / h_a^2 (A2)"""
    other = 0.0
    diag = 0.0
    for a in range(lv.dim):
        o, s = _axis_terms(lv, phi, a)
        h2 = lv.h[a] ** 2
        other = other + o / h2
        diag = diag + (s - 2.0) / h2
    return other, diag


def _colour_mask(lv, colour):
    idx = np.indices(tuple(lv.N[::-1])).sum(axis=0) + lv.dim   # 1-based (i + j [+ k])
    return (idx & 1) == colour


def smooth(lv, phi, f, sweeps):
    """Red-black Gauss-Seidel (Sec. 2.3 steps 2, 6, 11; red = (i+j[+k]) even
    first); each update solves the cell's own equation."""
    act = tuple(slice(1, n + 1) for n in reversed(lv.N))
    masks = [_colour_mask(lv, 0), _colour_mask(lv, 1)]
    for _ in range(sweeps):
        for m in masks:
            other, diag = _operator(lv, phi)
            new = (f[act] - other) / diag
            phi[act] = np.where(m, new, phi[act])


def residual(lv, phi, f):
    """r = f - lap(Phi) on the active cells (Sec. 2.3 step 4, defect form)"""
    act = tuple(slice(1, n + 1) for n in reversed(lv.N))
    other, diag = _operator(lv, phi)
    r = np.zeros_like(phi)
    r[act] = f[act] - (other + diag * phi[act])
    return r


def restrict(fine, r, coarse):
    """f of the coarse level from the fine residual (A3): along a coarsened
    axis coarse cell I sums fine cells 2I-1 and 2I (cells beyond the fine N
    count zero, a fine cell beyond 2 N_coarse has no parent), along the others
    it takes cell I; the sum is divided by 2^k, k the coarsened axes."""
    dim = fine.dim
    act = tuple(slice(1, n + 1) for n in reversed(fine.N))
    v = r[act]
    k = 0
    for a in range(dim):
        if coarse.la[a] <= fine.la[a]:
            continue
        k += 1
        ax = dim - 1 - a
        Nc, Nf = coarse.N[a], fine.N[a]
        if 2 * Nc > Nf:
            pad = [(0, 0)] * dim
            pad[ax] = (0, 2 * Nc - Nf)
            v = np.pad(v, pad)
        else:
            sl = [slice(None)] * dim
            sl[ax] = slice(0, 2 * Nc)
            v = v[tuple(sl)]
        shp = list(v.shape)
        shp[ax:ax + 1] = [Nc, 2]
        v = v.reshape(shp).sum(axis=ax + 1)
    fc = np.zeros(coarse.shape())
    fc[tuple(slice(1, n + 1) for n in reversed(coarse.N))] = v / 2.0 ** k
    return fc


def fill_ghosts(lv, phi):
    """Ghost layer of a coarse level by the rule of Sec. 2.4, axis after axis."""
    dim = lv.dim
    for a in range(dim):
        ax = dim - 1 - a
        N = lv.N[a]

        def at(i):
            sl = [slice(None)] * dim
            sl[ax] = i
            return tuple(sl)

        phi[at(0)] = -phi[at(1)]
        if lv.tie[a]:
            phi[at(N + 1)] = -phi[at(N - 1)] if N >= 2 else -phi[at(0)]
        else:
            phi[at(N + 1)] = lv.cR[a] * phi[at(N)]


def prolong_add(coarse, phic, fine, phif):
    """Phi_fine += P(Phi_coarse) (A4; Sec. 2.3 step 10): axis after axis, the
    fine centre of cell i a quarter coarse cell from coarse cell ceil(i/2)
    towards cell ceil(i/2) - 1 (i odd) or + 1 (i even), weights 3/4 and 1/4,
    along coarsened axes (coarse ghosts by the rule of Sec. 2.4); the coarse
    value of cell i along the others."""
    dim = fine.dim
    fill_ghosts(coarse, phic)
    v = phic
    for a in range(dim):
        ax = dim - 1 - a
        i = np.arange(1, fine.N[a] + 1)
        if coarse.la[a] > fine.la[a]:
            near = (i + 1) // 2
            far = np.where(i & 1, near - 1, near + 1)
            v = 0.75 * np.take(v, near, axis=ax) + 0.25 * np.take(v, far, axis=ax)
        else:
            v = np.take(v, i, axis=ax)
    phif[tuple(slice(1, n + 1) for n in reversed(fine.N))] += v


def vcycle(lvs, phi, f, nu_pre, nu_post):
    """One multigrid iteration (Sec. 2.3 steps 2-13) over the levels of A1."""
    smooth(lvs[0], phi[0], f[0], nu_pre)
    L = 0
    while True:
        r = residual(lvs[L], phi[L], f[L])
        f[L + 1] = restrict(lvs[L], r, lvs[L + 1])
        phi[L + 1] = np.zeros(lvs[L + 1].shape())
        smooth(lvs[L + 1], phi[L + 1], f[L + 1], nu_pre)
        L += 1
        if all(n == 1 for n in lvs[L].N) or L + 1 == len(lvs):
            break
    while L > 0:
        prolong_add(lvs[L], phi[L], lvs[L - 1], phi[L - 1])
        smooth(lvs[L - 1], phi[L - 1], f[L - 1], nu_post)
        L -= 1


def level_solve(n, h, phi, rho, fourpiG, nu_pre=2, nu_post=1, max_cycles=50, rel_tol=1e-10):
    """Solve one refinement level of n = (n_x, n_y[, n_z]) cells in place.
    phi, rho: arrays of n_a + 4 cells per axis (axis order (z,) y, x): the
    outer ring of phi holds the Dirichlet potential, Gamma (n_a + 2 cells)
    the initial guess on entry and the solution on exit; rho is read on
    Gamma.  Stops when ||f - lap Phi||_2 / ||f - lap Phi_zero||_2 < rel_tol
    (Phi_zero zero on Gamma, same outer ring) or after max_cycles; returns
    (cycles, history of that ratio)."""
    dim = len(n)
    M = [na + 2 for na in n]
    lvs = levels(M, h)
    # multigrid level 0 is the whole block: Gamma (storage 1..n_a+2) and the
    # outer ring as its ghost layer (storage 0 and n_a+3)
    phis = [np.array(phi, dtype=np.float64)] + [None] * (len(lvs) - 1)
    fs = [np.zeros_like(phis[0])] + [None] * (len(lvs) - 1)
    act = tuple(slice(1, m + 1) for m in reversed(M))
    fs[0][act] = fourpiG * rho[act]
    zero = phis[0].copy()
    zero[act] = 0.0
    bnorm = np.linalg.norm(residual(lvs[0], zero, fs[0])[act])
    rel = lambda: np.linalg.norm(residual(lvs[0], phis[0], fs[0])[act]) / bnorm if bnorm > 0 else 0.0
    hist = [rel()]
    c = 0
    while c < max_cycles and not (hist[-1] < rel_tol):
        if len(lvs) > 1:
            vcycle(lvs, phis, fs, nu_pre, nu_post)
        else:
            smooth(lvs[0], phis[0], fs[0], nu_pre)
        c += 1
        hist.append(rel())
    phi[act] = phis[0][act]
    return c, np.array(hist)


# ---------------------------------------------------------------------------
# A hierarchy of box patches (Sec. 2.1): interface, forces, the coarse-to-fine solve
# ---------------------------------------------------------------------------
def interface_fill(n_p, phi_p, rho_p, n_c, off, phi_c, rho_c, guess=True):
    """Buffer rings of a child patch from its parent (Sec. 2.1; Appendix A
    weights): bi/trilinear interpolation from the 2^d parent centres around
    each child centre -- potential into the outer ring, density into the
    inner ring, and (guess) the interpolated potential as the initial value
    of Gamma; the parent's centre of storage index p sits at coordinate p,
    the child's storage index s at off + 1.5 + (s - 1.5) / 2."""
    dim = len(n_c)
    shape_c = tuple(m + 4 for m in reversed(n_c))
    p0, t = [], []
    for a in range(dim):
        s = np.arange(n_c[a] + 4)
        q = off[a] + 1.5 + (s - 1.5) * 0.5
        f = np.floor(q).astype(int)
        p0.append(f)
        t.append(q - f)

    def interp(src):
        v = np.zeros(shape_c)
        for corner in np.ndindex(*([2] * dim)):
            w = np.ones(shape_c)
            idx = []
            for a in range(dim):
                ax = dim - 1 - a
                wa = t[a] if corner[a] else 1.0 - t[a]
                w = w * wa.reshape([-1 if k == ax else 1 for k in range(dim)])
                idx.append(p0[a] + corner[a])
            v += w * src[np.ix_(*reversed(idx))]
        return v

    outer = np.zeros(shape_c, dtype=bool)
    inner = np.zeros(shape_c, dtype=bool)
    for a in range(dim):
        ax = dim - 1 - a
        s = np.arange(n_c[a] + 4).reshape([-1 if k == ax else 1 for k in range(dim)])
        outer |= (s == 0) | (s == n_c[a] + 3)
        inner |= (s == 1) | (s == n_c[a] + 2)
    inner &= ~outer
    vphi = interp(phi_p)
    vrho = interp(rho_p)
    phi_c[outer] = vphi[outer]
    rho_c[inner] = vrho[inner]
    phi_c[~outer] = vphi[~outer] if guess else 0.0


def forces(n, h, phi, stencil=0):
    """F = -grad(Phi) on the patch cells by Eq. 2 (stencil 0) or the two-point
    central difference (stencil 1); shape (dim,) + patch shape ((z,) y, x)."""
    dim = len(n)
    om = [slice(2, m + 2) for m in reversed(n)]
    F = np.zeros((dim,) + tuple(reversed(n)))
    for a in range(dim):
        ax = dim - 1 - a

        def sh(d):
            sl = list(om)
            sl[ax] = slice(2 + d, n[a] + 2 + d)
            return phi[tuple(sl)]

        d1 = sh(1) - sh(-1)
        d2 = sh(2) - sh(-2)
        g = (4.0 / 3.0) * d1 / (2.0 * h) - (1.0 / 3.0) * d2 / (4.0 * h) if stencil == 0 else d1 / (2.0 * h)
        F[a] = -g
    return F


def solve_hierarchy(H, inputs, nu_pre=2, nu_post=1, max_cycles=50, rel_tol=1e-10, force_stencil=0):
    """Solve a nested hierarchy of box patches coarse to fine (Sec. 2.1 one-way
    scheme): the base level from the caller's boundary data (outer-ring
    potential, inner-ring density) and a zero start, every finer patch from
    its parent's converged solution (interpolated rings and initial guess).
    Returns per patch dicts with phi (the n_a + 4 block), rho, F, cycles, hist."""
    from math import pi
    dim = H.dim
    fourpiG = 4.0 * pi * H.G
    out = []
    for l in range(H.num_levels):
        n, h = tuple(H.n[l]), H.h(l)
        shape = tuple(m + 4 for m in reversed(n))
        phi = np.zeros(shape)
        rho = np.zeros(shape)
        gam = tuple(slice(1, m + 3) for m in reversed(n))
        om = tuple(slice(2, m + 2) for m in reversed(n))
        if l == 0:
            phi[...] = inputs[0]["bc_phi"]
            rho[gam] = inputs[0]["bc_rho"]
            phi[gam] = 0.0
        else:
            P = out[H.parent(l)]
            interface_fill(tuple(H.n[H.parent(l)]), P["phi"], P["rho"], n, H.offset(l), phi, rho, guess=True)
        rho[om] = inputs[l]["rho"]
        cyc, hist = level_solve(n, h, phi, rho, fourpiG, nu_pre, nu_post, max_cycles, rel_tol)
        out.append({"phi": phi, "rho": rho, "F": forces(n, h, phi, force_stencil), "cycles": cyc, "hist": hist})
    return out
