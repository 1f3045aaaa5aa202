"""Parity of the box-patch (non-cubic) CUDA path (include/mg_box.h) with the
per-axis FP64 oracle (oracle/aniso.py), through the C ABI.

After the same number of V-cycles on the same seeded inputs the FP64 path
must match the oracle to 1e-12 in the relative max-norm on potential and
force, on hierarchies whose axes stop coarsening at different multigrid
levels (semi-coarsening), at tie and non-tie sizes per axis; converged it must
take the same cycle counts.  With every axis equal it must equal the cubic
path (include/mg.h).  The mixed FP32-in-FP64 form must reach the same residual
tolerance and differ from the FP64 solution by less than 1e-2 of the
discretisation error.
"""
import numpy as np
import pytest

from oracle import aniso as A
from paper_2001_02327_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def mg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2001_02327_gb300 import build
    build.build()
    from paper_2001_02327_gb300 import mg as M
    return M


def relmax(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def box_solve(mg, H, inp, host_io=False, **kw):
    """(status, stats, [(phi, F)] per patch) from the CUDA path."""
    import torch
    b = mg.mg_box_create(mg.box_desc_from(H), mg.options(**kw))
    try:
        conv = (lambda a: np.ascontiguousarray(a)) if host_io else \
            (lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda())
        for l in range(H.num_levels):
            if l == 0:
                mg.mg_box_set_density(b, 0, conv(inp[0]["rho"]), conv(inp[0]["bc_rho"]), conv(inp[0]["bc_phi"]))
            else:
                mg.mg_box_set_density(b, l, conv(inp[l]["rho"]))
        status, stats = mg.mg_box_solve(b, H.num_levels, allow_noconv=True)
        out = []
        for l in range(H.num_levels):
            shape = tuple(reversed(H.n[l]))
            if host_io:
                phi, F = np.zeros(shape), np.zeros((H.dim,) + shape)
            else:
                phi = torch.zeros(shape, dtype=torch.float64, device="cuda")
                F = torch.zeros((H.dim,) + shape, dtype=torch.float64, device="cuda")
            mg.mg_box_forces(b, l, phi, F)
            if not host_io:
                phi, F = phi.cpu().numpy(), F.cpu().numpy()
            out.append((phi, F))
        return status, stats, out
    finally:
        mg.mg_box_destroy(b)


def oracle_solve(H, inp, nu=(2, 1), cycles=50, tol=1e-10, stencil=0):
    ref = A.solve_hierarchy(H, inp, nu[0], nu[1], cycles, tol, stencil)
    om = lambda l: tuple(slice(2, m + 2) for m in reversed(H.n[l]))
    return [(r["phi"][om(l)], r["F"], r["cycles"]) for l, r in enumerate(ref)]


# hierarchies: the box test cases of the oracle, and shapes whose axes stop
# coarsening at three different multigrid levels (3D M = 42, 14, 10: x at 5,
# y at 4, z at 3, with x_N = 1 exactly on z's level 2) and at two (2D)
CASES = {
    "box3d_24x32x16": lambda: I.box_3d_sphere(n=(24, 32, 16), levels=3),
    "box2d_48x24": lambda: I.box_2d_disk(n=(48, 24), levels=3),
    "box3d_40x12x8": lambda: I.box_3d_sphere(n=(40, 12, 8), levels=2),
    "box2d_44x12": lambda: I.box_2d_disk(n=(44, 12), levels=3),
}


def _stopped_axis_level(sizes, dim):
    """a multigrid level where one axis has one cell and another more"""
    return any(min(N[:dim]) == 1 and max(N[:dim]) > 1 for N in sizes)


@pytest.mark.parametrize("name", sorted(CASES))
def test_level_sizes_match_oracle(mg, name):
    H = CASES[name]()
    b = mg.mg_box_create(mg.box_desc_from(H), mg.options())
    try:
        for l in range(H.num_levels):
            got = mg.mg_box_level_sizes(b, l)
            want = [tuple(lv.N) + (1,) * (3 - H.dim) for lv in A.levels([n + 2 for n in H.n[l]], H.h(l))]
            assert got == want, (l, got, want)
            assert _stopped_axis_level(got, H.dim), got
    finally:
        mg.mg_box_destroy(b)


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("nu", [(2, 1), (1, 1), (2, 2)])
def test_fixed_cycles_match_oracle(mg, name, nu):
    H = CASES[name]()
    inp = I.level_inputs(H)
    cyc = 3
    status, stats, got = box_solve(mg, H, inp, nu_pre=nu[0], nu_post=nu[1], max_cycles=cyc, rel_tol=0.0)
    ref = oracle_solve(H, inp, nu, cyc, 0.0)
    for l, ((phi, F), (rphi, rF, rc)) in enumerate(zip(got, ref)):
        assert stats[l]["cycles"] == cyc == rc
        assert relmax(phi, rphi) < TOL, (l, relmax(phi, rphi))
        assert relmax(F, rF) < TOL, (l, relmax(F, rF))


@pytest.mark.parametrize("name", sorted(CASES))
def test_converged_matches_oracle(mg, name):
    H = CASES[name]()
    inp = I.level_inputs(H)
    status, stats, got = box_solve(mg, H, inp, rel_tol=1e-10, max_cycles=50)
    assert status == mg.MG_OK
    ref = oracle_solve(H, inp)
    for l, ((phi, F), (rphi, rF, rc)) in enumerate(zip(got, ref)):
        assert stats[l]["cycles"] == rc, (l, stats[l], rc)
        assert stats[l]["rel_res"] < 1e-10
        assert relmax(phi, rphi) < TOL, (l, relmax(phi, rphi))
        assert relmax(F, rF) < TOL, (l, relmax(F, rF))


def test_two_point_force_stencil(mg):
    H = CASES["box3d_40x12x8"]()
    inp = I.level_inputs(H)
    _, _, got = box_solve(mg, H, inp, max_cycles=2, rel_tol=0.0, force_stencil=mg.MG_FORCE_CD2)
    ref = oracle_solve(H, inp, cycles=2, tol=0.0, stencil=1)
    for (phi, F), (rphi, rF, _) in zip(got, ref):
        assert relmax(F, rF) < TOL


def test_host_arrays_equal_device_arrays(mg):
    H = CASES["box2d_44x12"]()
    inp = I.level_inputs(H)
    _, s1, d = box_solve(mg, H, inp, max_cycles=4, rel_tol=0.0)
    _, s2, h = box_solve(mg, H, inp, host_io=True, max_cycles=4, rel_tol=0.0)
    for (p1, F1), (p2, F2) in zip(d, h):
        assert np.array_equal(p1, p2) and np.array_equal(F1, F2)


def test_tree_of_box_patches(mg):
    """Two children of the base patch and a grandchild (Sec. 2.1 nesting with
    several patches per level), each solved from its own parent."""
    H0 = I.box_3d_sphere(n=(24, 32, 16), levels=1)
    h0 = H0.h0
    lo0 = H0.lo[0]
    n = [(24, 32, 16), (8, 12, 8), (12, 8, 8), (8, 8, 8)]
    off = [None, (2, 3, 2), (11, 15, 3), (1, 2, 2)]      # in parent cells
    parents = [None, 0, 0, 1]
    lo = [tuple(lo0)]
    for l in range(1, 4):
        p = parents[l]
        hp = h0 / 2 ** (0 if p == 0 else 1)
        lo.append(tuple(lo[p][a] + off[l][a] * hp for a in range(3)))
    H = I.BoxHierarchy(3, n, lo, h0, H0.G, H0.sources, "box_tree", parents=[-1, 0, 0, 1])
    H.validate()
    inp = I.level_inputs(H)
    status, stats, got = box_solve(mg, H, inp, max_cycles=3, rel_tol=0.0)
    ref = oracle_solve(H, inp, cycles=3, tol=0.0)
    for l, ((phi, F), (rphi, rF, _)) in enumerate(zip(got, ref)):
        assert relmax(phi, rphi) < TOL, l
        assert relmax(F, rF) < TOL, l


def test_equal_axes_equal_the_cubic_path(mg):
    """With n_x = n_y = n_z the box path solves the cubic method."""
    import torch
    Hc = I.config_3d_offset_sphere(n=16, levels=3)
    Hb = I.BoxHierarchy(3, [(16, 16, 16)] * 3, Hc.lo, Hc.h0, Hc.G, Hc.sources, "box_cube")
    inp = I.level_inputs(Hc)
    _, sb, gb = box_solve(mg, Hb, inp, rel_tol=1e-10)
    h = mg.mg_create_hierarchy([mg.desc_from(Hc)], mg.options(rel_tol=1e-10))
    try:
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        mg.mg_set_density(h, 0, 0, dev(inp[0]["rho"]), dev(inp[0]["bc_rho"]), dev(inp[0]["bc_phi"]))
        for l in range(1, 3):
            mg.mg_set_density(h, 0, l, dev(inp[l]["rho"]))
        _, sc = mg.mg_solve(h, 1)
        for l in range(3):
            phi = torch.zeros((16,) * 3, dtype=torch.float64, device="cuda")
            F = torch.zeros((3, 16, 16, 16), dtype=torch.float64, device="cuda")
            mg.mg_forces(h, 0, l, phi, F)
            assert sb[l]["cycles"] == sc[0][l]["cycles"]
            assert relmax(gb[l][0], phi.cpu().numpy()) < TOL
            assert relmax(gb[l][1], F.cpu().numpy()) < TOL
    finally:
        mg.mg_destroy(h)


@pytest.mark.parametrize("name", ["box3d_24x32x16", "box2d_48x24"])
@pytest.mark.parametrize("inner_max", [0, 8])
def test_mixed_precision_error_budget(mg, name, inner_max):
    H = CASES[name]()
    inp = I.level_inputs(H)
    status, stats, got = box_solve(mg, H, inp, rel_tol=1e-10, precision=mg.MG_MIXED, inner_max=inner_max)
    assert status == mg.MG_OK
    ref = oracle_solve(H, inp)
    for l, ((phi, F), (rphi, rF, _)) in enumerate(zip(got, ref)):
        assert stats[l]["rel_res"] < 1e-10
        exact = H.potential(H.centres(l, 0))
        disc = np.max(np.abs(rphi - exact))
        assert np.max(np.abs(phi - rphi)) < 1e-2 * disc, (l, np.max(np.abs(phi - rphi)), disc)


def test_time_smoothing_reports_bytes(mg):
    H = CASES["box3d_24x32x16"]()
    inp = I.level_inputs(H)
    b = mg.mg_box_create(mg.box_desc_from(H), mg.options(precision=mg.MG_MIXED))
    try:
        us, by = mg.mg_box_time_smoothing(b, 0, 0, 10)
        assert us > 0 and by == 1.5 * 26 * 34 * 18 * 4
    finally:
        mg.mg_box_destroy(b)
