"""The per-axis (non-cubic) multigrid of one refinement level in the oracle
(oracle/aniso.py), pinned by what fixes it independently of its own code:

- the per-axis sizes of Sec. 2.2 (halves rounded up, each axis stopping at one
  cell) on hand-worked cases, including the M = 10 sequence the paper prints;
- with every axis equal, the iterates of the cubic oracle (compiled C, pinned
  by its own tests) after a fixed number of V-cycles;
- for patches whose axes differ, the fixed point: the direct solution of the
  level's 5/7-point system with the Dirichlet outer ring;
- the contraction of a working multigrid cycle on those patches;
- for hierarchies of box patches: the cubic case equals the cubic oracle's
  hierarchy solve, the buffer fill is exact on multilinear fields, Eq. 2 is
  exact on quartics, and the error against the closed forms falls at second
  order.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import aniso as A
from paper_2001_02327_gb300 import inputs as I


def test_axis_sizes_and_semi_coarsening():
    assert A.axis_sizes(10) == [10, 5, 3, 1]          # Sec. 2.2's example, round(2.5) = 3
    assert A.axis_sizes(66) == [66, 33, 17, 8, 4, 2, 1]
    assert A.axis_sizes(6) == [6, 3, 2, 1]
    assert A.axis_sizes(18) == [18, 9, 5, 2, 1]
    lv = A.levels([10, 6, 18], 1.0)
    assert [l.N for l in lv] == [[10, 6, 18], [5, 3, 9], [3, 2, 5], [1, 1, 2], [1, 1, 1]]
    # cell sizes double only along axes that still coarsen
    assert [l.h for l in lv][-1] == [8.0, 8.0, 16.0]
    # x_N = 1 exactly for M = 10 at L = 2 (three cells of width 4/10 end at 1.1): the tie case
    assert lv[2].tie[0] and not lv[1].tie[0]


def test_restriction_averages_on_a_semi_coarsened_level():
    """A3: the restriction is an average -- a constant residual restricts to
    the same constant where every child exists, also where one axis no longer
    coarsens (M = (4, 34), levels 2 -> 3: x stays at one cell, y halves)."""
    lv = A.levels([4, 34], 1.0)
    fine, coarse = lv[2], lv[3]
    assert fine.N == [1, 9] and coarse.N == [1, 4]
    r = np.zeros(fine.shape())
    r[1:-1, 1:-1] = 1.0
    fc = A.restrict(fine, r, coarse)
    assert np.allclose(fc[1:5, 1], 1.0)                 # coarse cells J = 1..4 (children 1..8)


def test_operator_on_a_semi_coarsened_level():
    """A2 on level 3 of M = (4, 34) (h0 = 1): one cell along x of size 4
    (its left ghost -Phi_1 and its right ghost -Phi_1, since x_N + h/2 = 1),
    four cells along y of size 8.  For Phi = y^2 the interior cells give
    r = 0 - (x part + y part) = -((-1 - 1 - 2) Phi / 16 + 2) = Phi / 4 - 2."""
    lv = A.levels([4, 34], 1.0)[3]
    assert lv.N == [1, 4] and lv.h == [4.0, 8.0]
    y = (np.arange(6) - 0.5) * 8.0                      # storage 0..5 along y
    phi = np.zeros(lv.shape())
    phi[:, 1] = y ** 2
    r = A.residual(lv, phi, np.zeros_like(phi))
    for j in (2, 3):
        assert r[j, 1] == pytest.approx(phi[j, 1] / 4.0 - 2.0, rel=1e-14), j


def test_right_ghost_rule_per_axis():
    """Sec. 2.4 per axis on level 2 of M = (9, 11): x has 2 cells with right
    ghost -Phi_2 / 3, y 3 cells with right ghost -3 Phi_3 (linear
    extrapolation through zero at x_MG = 1 on each axis's own grid).  A field
    linear in y vanishing at y_MG = 1 has no y part at j = 2, 3, so the
    residual there is minus the x part: Phi / 8 at i = 1 and Phi / 12 at
    i = 2 (cell size 4)."""
    lv = A.levels([9, 11], 1.0)[2]
    assert lv.N == [2, 3] and lv.cR == pytest.approx([-1.0 / 3.0, -3.0])
    yn = (np.arange(5) - 0.5) * 4.0 / 11.0               # normalised centres, storage 0..4
    phi = np.zeros(lv.shape())
    phi[:, 1:3] = (1.0 - yn)[:, None]
    r = A.residual(lv, phi, np.zeros_like(phi))
    for j in (2, 3):
        assert r[j, 1] == pytest.approx(phi[j, 1] / 8.0, rel=1e-13), j
        assert r[j, 2] == pytest.approx(phi[j, 2] / 12.0, rel=1e-13), j


@pytest.mark.parametrize("dim,n", [(3, 12), (3, 8), (3, 9), (2, 20), (2, 8), (2, 13)])
def test_cubic_case_equals_the_cubic_oracle(oracle, dim, n):
    rng = np.random.default_rng(100 + 10 * dim + n)
    phi = rng.standard_normal((n + 4,) * dim)
    rho = rng.standard_normal((n + 4,) * dim)
    a, b = phi.copy(), phi.copy()
    ca, ha = A.level_solve((n,) * dim, 1.0 / n, a, rho, 0.7, 2, 1, 3, 0.0)
    cb, hb = oracle.level_solve(dim, n, 1.0 / n, b, rho, 0.7, 2, 1, 3, 0.0)
    assert ca == cb == 3
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))
    assert np.allclose(ha, hb, rtol=1e-9, atol=0.0)


def _direct(n, h, phi, rho, fourpiG):
    """Gamma values of the direct solution of the level's 5/7-point system
    (Dirichlet outer ring from phi), by a sparse LU factorisation."""
    dim = len(n)
    M = [na + 2 for na in n]
    act = tuple(slice(1, m + 1) for m in reversed(M))
    ring = phi.copy()
    ring[act] = 0.0
    # the ring's contribution to the Laplacian on Gamma
    lap_ring = np.zeros_like(ring)
    for ax in range(dim):
        lap_ring += np.roll(ring, 1, axis=ax) + np.roll(ring, -1, axis=ax)
    b = fourpiG * rho[act] - lap_ring[act] / h ** 2
    ops = []
    for a in range(dim):
        m = M[a]
        D = sp.diags([np.ones(m - 1), -2.0 * np.ones(m), np.ones(m - 1)], [-1, 0, 1])
        mats = [sp.identity(M[k]) if k != a else D for k in reversed(range(dim))]   # (z,) y, x order
        K = mats[0]
        for X in mats[1:]:
            K = sp.kron(K, X)
        ops.append(K)
    Amat = sum(ops).tocsc() / h ** 2
    x = spla.spsolve(Amat, b.ravel())
    return x.reshape(b.shape)


@pytest.mark.parametrize("n", [(8, 12, 6), (5, 9, 14), (14, 9), (30, 7), (3, 17)])
def test_non_cubic_fixed_point_is_the_direct_solution(n):
    dim = len(n)
    rng = np.random.default_rng(sum(n))
    shape = tuple(na + 4 for na in reversed(n))
    phi = rng.standard_normal(shape)
    rho = rng.standard_normal(shape)
    h = 1.0 / max(n)
    ref = _direct(n, h, phi, rho, 0.9)
    c, hist = A.level_solve(n, h, phi, rho, 0.9, 2, 2, 60, 1e-13)
    act = tuple(slice(1, na + 3) for na in reversed(n))
    assert hist[-1] < 1e-13, hist[-6:]
    assert np.max(np.abs(phi[act] - ref)) <= 1e-10 * np.max(np.abs(ref))


@pytest.mark.parametrize("n", [(16, 8, 12), (24, 10), (12, 30)])
def test_non_cubic_cycles_contract(n):
    """A working V(2,1) cycle: the residual falls by well over a factor of
    three per cycle once the first cycles have passed."""
    rng = np.random.default_rng(7 * sum(n))
    shape = tuple(na + 4 for na in reversed(n))
    phi = rng.standard_normal(shape)
    rho = rng.standard_normal(shape)
    c, hist = A.level_solve(n, 1.0 / max(n), phi, rho, 1.0, 2, 1, 10, 0.0)
    rates = hist[4:] / hist[3:-1]
    assert np.all(rates < 0.3), rates


# --------------------------------------------------------------------------
# hierarchies of box patches: interface, forces, the coarse-to-fine solve
# --------------------------------------------------------------------------


@pytest.mark.parametrize("dim,n", [(3, 16), (2, 32)])
def test_box_hierarchy_cubic_case_equals_cubic_oracle(oracle, dim, n):
    Hc = I.config_3d_offset_sphere(n, 3) if dim == 3 else I.config_2d_disk(n, 3)
    Hb = I.nested_boxes(dim, 3, (n,) * dim, [1.0] * dim, Hc.G, Hc.sources)
    ic, ib = I.level_inputs(Hc), I.level_inputs(Hb)
    rc = oracle.solve_hierarchy(Hc, ic, 2, 1, 3, 0.0)
    rb = A.solve_hierarchy(Hb, ib, 2, 1, 3, 0.0)
    for l in range(3):
        for key in ("phi", "F"):
            ref = rc[l][key]
            assert np.max(np.abs(rb[l][key] - ref)) <= 1e-12 * np.max(np.abs(ref)), (l, key)


@pytest.mark.parametrize("dim", [2, 3])
def test_box_interface_exact_on_multilinear_fields(dim):
    """Appendix A: the bi/trilinear buffer fill reproduces any multilinear
    field; parent centre of storage index p at coordinate p, child storage
    index s at off + 1.5 + (s - 1.5) / 2, per axis."""
    rng = np.random.default_rng(dim)
    n_p = (20, 14, 18)[:dim]
    n_c = (12, 8, 10)[:dim]
    off = (3, 2, 5)[:dim]
    coef = rng.standard_normal(2 ** dim)

    def field(coords):                                   # sum over subsets of the product of coordinates
        v = 0.0
        for m, c in zip(np.ndindex(*([2] * dim)), coef):
            term = c
            for a in range(dim):
                if m[a]:
                    term = term * coords[a]
            v = v + term
        return v

    def grid(n, to_coord):
        ax = [to_coord(a, np.arange(n[a] + 4)) for a in range(dim)]
        g = np.meshgrid(*ax[::-1], indexing="ij")
        return g[::-1]                                   # x, y[, z] arrays in (z,) y, x order

    phi_p = field(grid(n_p, lambda a, p: p.astype(float)))
    rho_p = 2.0 * phi_p + 1.0
    phi_c = np.full(tuple(m + 4 for m in reversed(n_c)), np.nan)
    rho_c = np.full_like(phi_c, np.nan)
    A.interface_fill(n_p, phi_p, rho_p, n_c, off, phi_c, rho_c, guess=True)
    want = field(grid(n_c, lambda a, s: off[a] + 1.5 + (s - 1.5) * 0.5))
    assert np.allclose(phi_c, want, rtol=0, atol=1e-12 * np.max(np.abs(want)))
    inner = np.zeros(phi_c.shape, dtype=bool)
    outer = np.zeros(phi_c.shape, dtype=bool)
    for a in range(dim):
        ax = dim - 1 - a
        s = np.arange(n_c[a] + 4).reshape([-1 if k == ax else 1 for k in range(dim)])
        outer |= (s == 0) | (s == n_c[a] + 3)
        inner |= (s == 1) | (s == n_c[a] + 2)
    inner &= ~outer
    assert np.allclose(rho_c[inner], 2.0 * want[inner] + 1.0, rtol=0, atol=1e-12 * np.max(np.abs(want)))
    assert np.all(np.isnan(rho_c[~inner]))              # density only into the inner ring


@pytest.mark.parametrize("n", [(10, 7, 12), (9, 15)])
def test_box_forces_exact_on_quartics(n):
    """Eq. 2 is exact for polynomials of degree four along each axis."""
    dim = len(n)
    h = 0.37
    ax = [(np.arange(n[a] + 4) - 1.5) * h for a in range(dim)]
    g = np.meshgrid(*ax[::-1], indexing="ij")[::-1]
    polys = [(0.3, -1.1, 0.7, 2.0, -0.4), (1.5, 0.2, -0.9, 0.1, 0.8), (-0.6, 0.5, 0.3, -1.2, 0.05)][:dim]
    phi = sum(np.polyval(p, g[a]) for a, p in enumerate(polys))
    F = A.forces(n, h, phi, 0)
    for a, p in enumerate(polys):
        om = tuple(slice(2, m + 2) for m in reversed(n))
        want = -np.polyval(np.polyder(p), g[a][om])
        assert np.allclose(F[a], want, rtol=0, atol=1e-10 * np.max(np.abs(want))), a


def _errors(H, res):
    ep = ef = 0.0
    for l in range(H.num_levels):
        X = H.centres(l, 0)
        om = tuple(slice(2, m + 2) for m in reversed(H.n[l]))
        pa, fa = H.potential(X), H.force(X)
        ep = max(ep, np.max(np.abs(res[l]["phi"][om] - pa)) / np.max(np.abs(pa)))
        ef = max(ef, np.max(np.abs(np.moveaxis(res[l]["F"], 0, -1) - fa)) / np.max(np.abs(fa)))
    return ep, ef


@pytest.mark.parametrize("make", [lambda k: I.box_3d_sphere((12 * k, 16 * k, 8 * k), 3),
                                  lambda k: I.box_2d_disk((24 * k, 12 * k), 3)])
def test_box_hierarchy_second_order(make):
    """Potential and forces of a nested box hierarchy against the closed form:
    the largest error over all patches falls by more than 3 when the cells
    halve (second order across the refinement interfaces)."""
    e = []
    for k in (1, 2):
        H = make(k)
        res = A.solve_hierarchy(H, I.level_inputs(H), 2, 2, 40, 1e-10)
        assert all(r["hist"][-1] < 1e-10 for r in res)
        e.append(_errors(H, res))
    assert e[0][0] / e[1][0] > 3.0 and e[0][1] / e[1][1] > 3.0, e
