"""The per-axis (non-cubic) multigrid of one refinement level in the oracle
(oracle/aniso.py), pinned by what fixes it independently of its own code:

- the per-axis sizes of Sec. 2.2 (halves rounded up, each axis stopping at one
  cell) on hand-worked cases, including the M = 10 sequence the paper prints;
- with every axis equal, the iterates of the cubic oracle (compiled C, pinned
  by its own tests) after a fixed number of V-cycles;
- for patches whose axes differ, the fixed point: the direct solution of the
  level's 5/7-point system with the Dirichlet outer ring;
- the contraction of a working multigrid cycle on those patches.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import aniso as A


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
