"""Parity of the CUDA path with the CPU FP64 oracle, through the C ABI.

The FP64 path must match the oracle to 1e-12 in the relative max-norm
(max|gpu - oracle| / max|oracle|) on potential and force after the same
number of V-cycles on the same seeded inputs.  The mixed FP32-in-FP64 form
must reach the same residual tolerance and differ from the FP64 solution by
less than 1e-2 of the discretisation error (the closed-form error at the
same grid).
"""
import numpy as np
import pytest

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


def gpu_solve(mg, H, inp, host_io=False, allow_noconv=True, batch_copies=1, **kw):
    import torch
    opt = mg.options(**kw)
    h = mg.mg_create_hierarchy([mg.desc_from(H)] * batch_copies, opt)
    try:
        conv = (lambda a: np.ascontiguousarray(a)) if host_io else (lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda())
        for b in range(batch_copies):
            for l in range(H.num_levels):
                if l == 0:
                    mg.mg_set_density(h, b, 0, conv(inp[0]["rho"]), conv(inp[0]["bc_rho"]), conv(inp[0]["bc_phi"]))
                else:
                    mg.mg_set_density(h, b, l, conv(inp[l]["rho"]))
        status, stats = mg.mg_solve(h, batch_copies, allow_noconv=allow_noconv)
        out = []
        for b in range(batch_copies):
            lev = []
            for l in range(H.num_levels):
                n = H.n[l]
                if host_io:
                    phi = np.zeros((n,) * H.dim)
                    F = np.zeros((H.dim,) + (n,) * H.dim)
                    mg.mg_forces(h, b, l, phi, F)
                else:
                    phi = torch.zeros((n,) * H.dim, dtype=torch.float64, device="cuda")
                    F = torch.zeros((H.dim,) + (n,) * H.dim, dtype=torch.float64, device="cuda")
                    mg.mg_forces(h, b, l, phi, F)
                    torch.cuda.synchronize()
                    phi, F = phi.cpu().numpy(), F.cpu().numpy()
                lev.append({"phi": phi, "F": F, **stats[b][l]})
            out.append(lev)
        return status, out if batch_copies > 1 else out[0]
    finally:
        mg.mg_destroy(h)


def omega(block, n, dim):
    return block[(slice(2, n + 2),) * dim]


def check_parity(H, gpu, ref, tol=TOL):
    for l in range(H.num_levels):
        n = H.n[l]
        e_phi = relmax(gpu[l]["phi"], omega(ref[l]["phi"], n, H.dim))
        e_F = relmax(gpu[l]["F"], ref[l]["F"])
        assert e_phi < tol and e_F < tol, (l, e_phi, e_F)


def random_single_level(dim, n, seed, h=None):
    rng = np.random.default_rng(I.BASE_SEED + seed)
    hh = h or 1.0 / n
    H = I.Hierarchy(dim, [n], [tuple([0.0] * dim)], hh, 0.9, [], f"rand{dim}d{n}")
    inp = [{"rho": rng.standard_normal((n,) * dim), "bc_rho": rng.standard_normal((n + 2,) * dim),
            "bc_phi": rng.standard_normal((n + 4,) * dim)}]
    return H, inp


# --------------------------------------------------------------------------
# one level, random data, fixed cycle count: sizes spanning tiles, odd
# sizes, the smallest level, ragged tails
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dim,n", [(2, 2), (2, 5), (2, 30), (2, 62), (2, 126), (2, 255),
                                   (3, 2), (3, 3), (3, 5), (3, 14), (3, 30), (3, 47), (3, 62)])
@pytest.mark.parametrize("nu", [(2, 1), (2, 2)])
def test_single_level_fixed_cycles(mg, oracle, dim, n, nu):
    H, inp = random_single_level(dim, n, 100 * dim + n)
    _, g = gpu_solve(mg, H, inp, nu_pre=nu[0], nu_post=nu[1], max_cycles=3, rel_tol=0.0)
    ref = oracle.solve_hierarchy(H, inp, nu[0], nu[1], 3, 0.0)
    assert g[0]["cycles"] == 3
    check_parity(H, g, ref)


@pytest.mark.parametrize("dim,n", [(2, 62), (3, 30)])
def test_single_level_to_stagnation(mg, oracle, dim, n):
    """Both sides iterated to round-off agree with each other (and so with
    the direct solves the oracle is pinned to)."""
    H, inp = random_single_level(dim, n, 7)
    _, g = gpu_solve(mg, H, inp, max_cycles=40, rel_tol=0.0)
    ref = oracle.solve_hierarchy(H, inp, 2, 1, 40, 0.0)
    check_parity(H, g, ref)


def test_force_stencil_cd2(mg, oracle):
    H, inp = random_single_level(3, 14, 3)
    _, g = gpu_solve(mg, H, inp, max_cycles=2, rel_tol=0.0, force_stencil=mg.MG_FORCE_CD2)
    ref = oracle.solve_hierarchy(H, inp, 2, 1, 2, 0.0, force_stencil=1)
    check_parity(H, g, ref)


# --------------------------------------------------------------------------
# nested hierarchies (interface + per-level solves), fixed cycles per level
# --------------------------------------------------------------------------
@pytest.mark.parametrize("make", [lambda: I.config_2d_disk(64, 3), lambda: I.config_3d_offset_sphere(32, 4),
                                  lambda: I.paper_3d(16), lambda: I.paper_2d(32), lambda: I.random_hierarchy(3)])
def test_hierarchy_fixed_cycles(mg, oracle, make):
    H = make()
    inp = I.level_inputs(H)
    _, g = gpu_solve(mg, H, inp, max_cycles=3, rel_tol=0.0)
    ref = oracle.solve_hierarchy(H, inp, 2, 1, 3, 0.0)
    check_parity(H, g, ref)


@pytest.mark.parametrize("guess", ["zero"])
def test_hierarchy_zero_guess(mg, oracle, guess):
    H = I.config_3d_offset_sphere(16, 3)
    inp = I.level_inputs(H)
    _, g = gpu_solve(mg, H, inp, max_cycles=3, rel_tol=0.0, guess=mg.MG_GUESS_ZERO)
    ref = oracle.solve_hierarchy(H, inp, 2, 1, 3, 0.0, guess="zero")
    check_parity(H, g, ref)


# --------------------------------------------------------------------------
# frozen-interface ablation (the scheme Sec. 4 compares against)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("make", [lambda: I.config_2d_disk(64, 3), lambda: I.config_3d_offset_sphere(32, 4),
                                  lambda: I.random_hierarchy(5)])
def test_frozen_interface_fixed_cycles(mg, oracle, make):
    H = make()
    inp = I.level_inputs(H)
    _, g = gpu_solve(mg, H, inp, max_cycles=3, rel_tol=0.0, interface=mg.MG_IFACE_FROZEN)
    ref = oracle.solve_hierarchy(H, inp, 2, 1, 3, 0.0, interface="frozen")
    check_parity(H, g, ref)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_frozen_interface_converged(mg, oracle, precision):
    """Converged frozen-interface solve: same cycle counts (FP64) and results
    as the oracle, and really different from the buffer-ring method."""
    H = I.config_3d_offset_sphere(32, 3)
    inp = I.level_inputs(H)
    p = mg.MG_FP64 if precision == "fp64" else mg.MG_MIXED
    kw = dict(nu_pre=2, nu_post=2, max_cycles=60, rel_tol=1e-10, allow_noconv=False, precision=p)
    _, g = gpu_solve(mg, H, inp, interface=mg.MG_IFACE_FROZEN, **kw)
    _, gb = gpu_solve(mg, H, inp, **kw)
    ref = oracle.solve_hierarchy(H, inp, 2, 2, 60, 1e-10, interface="frozen")
    for l in range(H.num_levels):
        assert g[l]["rel_res"] < 1e-10
        if p == mg.MG_FP64:
            assert g[l]["cycles"] == ref[l]["cycles"], (l, g[l]["cycles"], ref[l]["cycles"])
    check_parity(H, g, ref, tol=TOL if p == mg.MG_FP64 else 1e-8)
    assert relmax(g[0]["phi"], gb[0]["phi"]) == 0.0          # level 0 has no interface
    for l in range(1, H.num_levels):
        assert relmax(g[l]["phi"], gb[l]["phi"]) > 1e-6


# --------------------------------------------------------------------------
# patch-based refinement: several patches per level (a tree of patches)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_patch_tree(mg, oracle, prec):
    H = I.config_3d_patches(64, 32)
    inp = I.level_inputs(H)
    p = mg.MG_FP64 if prec == "fp64" else mg.MG_MIXED
    _, g = gpu_solve(mg, H, inp, max_cycles=3, rel_tol=0.0, precision=mg.MG_FP64)
    check_parity(H, g, oracle.solve_hierarchy(H, inp, 2, 1, 3, 0.0))
    _, gc = gpu_solve(mg, H, inp, nu_pre=2, nu_post=2, max_cycles=60, rel_tol=1e-10, precision=p,
                      allow_noconv=False)
    ref = oracle.solve_hierarchy(H, inp, 2, 2, 60, 1e-10)
    for l in range(H.num_levels):
        assert gc[l]["rel_res"] < 1e-10
        if p == mg.MG_FP64:
            assert gc[l]["cycles"] == ref[l]["cycles"], l
    check_parity(H, gc, ref, tol=TOL if p == mg.MG_FP64 else 1e-8)


def test_patch_tree_equals_chains_on_gpu(mg):
    H = I.config_3d_patches(64, 32)
    _, g = gpu_solve(mg, H, I.level_inputs(H), max_cycles=4, rel_tol=0.0)
    for path in ([0, 1, 3], [0, 2]):
        Hc = I.Hierarchy(3, [H.n[l] for l in path], [H.lo[l] for l in path], H.h0, H.G, H.sources)
        _, gc = gpu_solve(mg, Hc, I.level_inputs(Hc), max_cycles=4, rel_tol=0.0)
        for k, l in enumerate(path):
            assert np.array_equal(gc[k]["phi"], g[l]["phi"]) and np.array_equal(gc[k]["F"], g[l]["F"]), (path, l)


# --------------------------------------------------------------------------
# the force-change stopping test of Sec. 3
# --------------------------------------------------------------------------
@pytest.mark.parametrize("make,stencil", [(lambda: I.paper_3d(16), 0), (lambda: I.paper_2d(64), 0),
                                          (lambda: I.config_3d_offset_sphere(32, 3), 1)])
def test_force_stop_rule(mg, oracle, make, stencil):
    H = make()
    inp = I.level_inputs(H)
    _, g = gpu_solve(mg, H, inp, max_cycles=60, rel_tol=1e-10, stop=mg.MG_STOP_FORCE, force_stencil=stencil,
                     allow_noconv=False)
    ref = oracle.solve_hierarchy(H, inp, 2, 1, 60, 1e-10, stop="force", force_stencil=stencil)
    for l in range(H.num_levels):
        assert g[l]["cycles"] == ref[l]["cycles"], (l, g[l]["cycles"], ref[l]["cycles"])
        assert g[l]["rel_res"] < 1e-10
        assert abs(g[l]["rel_res"] / ref[l]["hist"][-1] - 1) < 1e-3, (l, g[l]["rel_res"], ref[l]["hist"][-1])
    check_parity(H, g, ref)


def test_force_stop_mixed_and_invalid_combination(mg):
    H = I.paper_3d(16)
    inp = I.level_inputs(H)
    _, g = gpu_solve(mg, H, inp, max_cycles=60, rel_tol=1e-10, stop=mg.MG_STOP_FORCE, precision=mg.MG_MIXED,
                     allow_noconv=False)
    _, f = gpu_solve(mg, H, inp, max_cycles=60, rel_tol=1e-10, stop=mg.MG_STOP_FORCE, allow_noconv=False)
    for l in range(H.num_levels):
        assert g[l]["rel_res"] < 1e-10
        assert relmax(g[l]["F"], f[l]["F"]) < 1e-8
    with pytest.raises(mg.MGError):
        mg.mg_create_hierarchy([mg.desc_from(H)], mg.options(stop=mg.MG_STOP_FORCE, interface=mg.MG_IFACE_FROZEN))


def test_full_size_config_fixed_cycles(mg, oracle):
    """The benchmark workload (4 nested 64^3 levels), element by element."""
    H = I.config_3d_offset_sphere(64, 4)
    inp = I.level_inputs(H)
    _, g = gpu_solve(mg, H, inp, nu_pre=2, nu_post=2, max_cycles=2, rel_tol=0.0)
    ref = oracle.solve_hierarchy(H, inp, 2, 2, 2, 0.0)
    check_parity(H, g, ref)


def test_full_size_config_converged(mg, oracle):
    """The benchmark workload solved to 1e-10 exactly as the benchmark runs
    it: same cycle counts as the oracle and the same results."""
    H = I.config_3d_offset_sphere(64, 4)
    inp = I.level_inputs(H)
    st, g = gpu_solve(mg, H, inp, nu_pre=2, nu_post=2, max_cycles=50, rel_tol=1e-10, allow_noconv=False)
    ref = oracle.solve_hierarchy(H, inp, 2, 2, 50, 1e-10)
    for l in range(H.num_levels):
        assert g[l]["cycles"] == ref[l]["cycles"], (l, g[l]["cycles"], ref[l]["cycles"])
        assert g[l]["rel_res"] < 1e-10
        # ||r|| ~ 1e-10 ||b|| is a difference of O(||b||) terms: round-off of
        # 1e-16 in the operands is ~1e-6 of it
        assert abs(g[l]["rel_res"] / ref[l]["hist"][-1] - 1) < 1e-4
    check_parity(H, g, ref)


# --------------------------------------------------------------------------
# mixed FP32-in-FP64 defect correction
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n,levels", [(32, 4), (64, 4)])
def test_mixed_precision_error_budget(mg, n, levels):
    H = I.config_3d_offset_sphere(n, levels)
    inp = I.level_inputs(H)
    _, ref = gpu_solve(mg, H, inp, nu_pre=2, nu_post=2, max_cycles=60, rel_tol=1e-10, allow_noconv=False)
    _, mix = gpu_solve(mg, H, inp, nu_pre=2, nu_post=2, max_cycles=60, rel_tol=1e-10, allow_noconv=False,
                       precision=mg.MG_MIXED, inner_cycles=3)
    for l in range(H.num_levels):
        X = H.centres(l, 0)
        disc_phi = np.max(np.abs(ref[l]["phi"] - H.potential(X)))
        disc_F = np.max(np.abs(np.moveaxis(ref[l]["F"], 0, -1) - H.force(X)))
        assert mix[l]["rel_res"] < 1e-10
        assert np.max(np.abs(mix[l]["phi"] - ref[l]["phi"])) < 1e-2 * disc_phi
        assert np.max(np.abs(mix[l]["F"] - ref[l]["F"])) < 1e-2 * disc_F


# --------------------------------------------------------------------------
# API behaviour
# --------------------------------------------------------------------------
def test_host_buffers_equal_device_buffers(mg):
    H = I.config_3d_offset_sphere(16, 3)
    inp = I.level_inputs(H)
    _, a = gpu_solve(mg, H, inp, max_cycles=4, rel_tol=0.0)
    _, b = gpu_solve(mg, H, inp, host_io=True, max_cycles=4, rel_tol=0.0)
    for l in range(H.num_levels):
        assert np.array_equal(a[l]["phi"], b[l]["phi"]) and np.array_equal(a[l]["F"], b[l]["F"])


def test_page_locked_host_buffers_equal_device_buffers(mg):
    """Page-locked (pinned) host arrays are read and written by the kernels in
    place; the results equal those through device arrays, and the caller's
    host arrays are complete when each call returns."""
    import torch
    H = I.config_3d_offset_sphere(32, 3)
    inp = I.level_inputs(H)
    _, a = gpu_solve(mg, H, inp, max_cycles=4, rel_tol=0.0)
    pin = lambda x: torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
    h = mg.mg_create_hierarchy([mg.desc_from(H)], mg.options(max_cycles=4, rel_tol=0.0))
    try:
        for l in range(H.num_levels):
            if l == 0:
                mg.mg_set_density(h, 0, 0, pin(inp[0]["rho"]), pin(inp[0]["bc_rho"]), pin(inp[0]["bc_phi"]))
            else:
                mg.mg_set_density(h, 0, l, pin(inp[l]["rho"]))
        mg.mg_solve(h, 1, allow_noconv=True)
        for l in range(H.num_levels):
            n = H.n[l]
            phi = torch.zeros((n,) * 3, dtype=torch.float64).pin_memory()
            F = torch.zeros((3,) + (n,) * 3, dtype=torch.float64).pin_memory()
            mg.mg_forces(h, 0, l, phi, F)
            assert np.array_equal(phi.numpy(), a[l]["phi"]) and np.array_equal(F.numpy(), a[l]["F"]), l
    finally:
        mg.mg_destroy(h)


def test_deterministic(mg):
    H = I.config_3d_offset_sphere(32, 2)
    inp = I.level_inputs(H)
    _, a = gpu_solve(mg, H, inp)
    _, b = gpu_solve(mg, H, inp)
    for l in range(H.num_levels):
        assert np.array_equal(a[l]["phi"], b[l]["phi"]) and a[l]["cycles"] == b[l]["cycles"]


def test_batch_of_identical_hierarchies(mg):
    H = I.config_3d_offset_sphere(16, 3)
    inp = I.level_inputs(H)
    _, single = gpu_solve(mg, H, inp, max_cycles=3, rel_tol=0.0)
    _, many = gpu_solve(mg, H, inp, max_cycles=3, rel_tol=0.0, batch_copies=3)
    for b in range(3):
        for l in range(H.num_levels):
            assert np.array_equal(many[b][l]["phi"], single[l]["phi"])


def test_zero_problem(mg):
    H, inp = random_single_level(3, 8, 1)
    for k in inp[0]:
        inp[0][k][...] = 0.0
    _, g = gpu_solve(mg, H, inp)
    assert g[0]["cycles"] == 0 and np.all(g[0]["phi"] == 0) and np.all(g[0]["F"] == 0)


def test_state_errors(mg):
    import torch
    H = I.config_3d_offset_sphere(16, 2)
    h = mg.mg_create_hierarchy([mg.desc_from(H)])
    try:
        with pytest.raises(mg.MGError) as e:
            mg.mg_solve(h, 1)
        assert e.value.status == mg.MG_ESTATE
        with pytest.raises(mg.MGError) as e:
            mg.mg_forces(h, 0, 0, None, torch.zeros(3 * 16 ** 3, dtype=torch.float64, device="cuda"))
        assert e.value.status == mg.MG_ESTATE
        with pytest.raises(mg.MGError) as e:
            mg.mg_set_density(h, 0, 5, torch.zeros(16 ** 3, dtype=torch.float64, device="cuda"))
        assert e.value.status == mg.MG_EINVAL
    finally:
        mg.mg_destroy(h)


@pytest.mark.parametrize("graph", ["1", "0"])
def test_too_few_cycles_reports_enoconv(mg, graph, monkeypatch):
    monkeypatch.setenv("MG_SOLVE_GRAPH", graph)
    H = I.config_3d_offset_sphere(32, 3)
    status, g = gpu_solve(mg, H, I.level_inputs(H), max_cycles=2, rel_tol=1e-10)
    assert status == mg.MG_ENOCONV
    for l in range(H.num_levels):
        assert g[l]["cycles"] == 2 and g[l]["status"] == mg.MG_ENOCONV and g[l]["rel_res"] > 1e-10


@pytest.mark.parametrize("graph", ["1", "0"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_non_finite_density_reports_ediverged(mg, graph, prec, monkeypatch):
    """A NaN in the density is reported as MG_EDIVERGED (not as a converged
    level), and the handle solves the next, finite input normally."""
    import torch
    monkeypatch.setenv("MG_SOLVE_GRAPH", graph)
    H = I.config_3d_offset_sphere(16, 2)
    inp = I.level_inputs(H)
    p = mg.MG_FP64 if prec == "fp64" else mg.MG_MIXED
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    bad = inp[0]["rho"].copy()
    bad[3, 4, 5] = np.nan
    h = mg.mg_create_hierarchy([mg.desc_from(H)], mg.options(precision=p))
    try:
        mg.mg_set_density(h, 0, 0, dev(bad), dev(inp[0]["bc_rho"]), dev(inp[0]["bc_phi"]))
        mg.mg_set_density(h, 0, 1, dev(inp[1]["rho"]))
        with pytest.raises(mg.MGError) as e:
            mg.mg_solve(h, 1)
        assert e.value.status == mg.MG_EDIVERGED
        mg.mg_set_density(h, 0, 0, dev(inp[0]["rho"]), dev(inp[0]["bc_rho"]), dev(inp[0]["bc_phi"]))
        mg.mg_set_density(h, 0, 1, dev(inp[1]["rho"]))
        status, st = mg.mg_solve(h, 1)
        assert status == mg.MG_OK and all(st[0][l]["rel_res"] < 1e-10 for l in range(2))
    finally:
        mg.mg_destroy(h)


def test_second_order_on_gpu(mg):
    """Second order in L1, L2 and L-infinity for potential and force, from
    the GPU results (composite-grid norms as in Tables 1-2)."""
    from oracle import norms as NR
    prev = None
    for n in (16, 32, 64):
        H = I.config_3d_offset_sphere(n, 4)
        _, g = gpu_solve(mg, H, I.level_inputs(H), nu_pre=2, nu_post=2, allow_noconv=False)
        ex, ep = [], []
        for l in range(H.num_levels):
            X = H.centres(l, 0)
            ex.append(np.sqrt(np.sum((np.moveaxis(g[l]["F"], 0, -1) - H.force(X)) ** 2, axis=-1)))
            ep.append(np.abs(g[l]["phi"] - H.potential(X)))
        cur = np.array(NR.norms(H, ex) + NR.norms(H, ep))
        if prev is not None:
            order = np.log2(prev / cur)
            assert np.all(order > 1.7), order
        prev = cur


def test_graph_path_equals_host_loop(mg):
    """The solve graph (device-side loop control) and the host-driven loop
    (taken while per-kernel profiling is on) launch the same kernels in the
    same order: identical results and cycle counts."""
    import torch
    H = I.config_3d_offset_sphere(32, 3)
    inp = I.level_inputs(H)
    res = {}
    for prof in (False, True):
        h = mg.mg_create_hierarchy([mg.desc_from(H)], mg.options(nu_pre=2, nu_post=2))
        try:
            dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
            mg.mg_set_density(h, 0, 0, dev(inp[0]["rho"]), dev(inp[0]["bc_rho"]), dev(inp[0]["bc_phi"]))
            for l in range(1, H.num_levels):
                mg.mg_set_density(h, 0, l, dev(inp[l]["rho"]))
            mg.mg_profile(h, prof)
            _, st = mg.mg_solve(h, 1)
            if prof:
                k = mg.mg_profile_read(h)
                assert k["smooth_colour"][0] > 0 and k["resid_norm"][0] > 0
            out = []
            for l in range(H.num_levels):
                phi = torch.zeros((H.n[l],) * 3, dtype=torch.float64, device="cuda")
                mg.mg_forces(h, 0, l, phi, None)
                torch.cuda.synchronize()
                out.append((phi.cpu().numpy(), st[0][l]["cycles"]))
            res[prof] = out
        finally:
            mg.mg_destroy(h)
    for (a, ca), (b, cb) in zip(res[False], res[True]):
        assert ca == cb and np.array_equal(a, b)


def _solve_with(mg, H, inp, prof, **kw):
    """Solve on the GPU with the graph (prof False) or the host-driven loop
    (prof True); per level the potential, the stats and (host loop) the
    one-block kernel's launch count."""
    import torch
    h = mg.mg_create_hierarchy([mg.desc_from(H)], mg.options(**kw))
    try:
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        mg.mg_set_density(h, 0, 0, dev(inp[0]["rho"]), dev(inp[0]["bc_rho"]), dev(inp[0]["bc_phi"]))
        for l in range(1, H.num_levels):
            mg.mg_set_density(h, 0, l, dev(inp[l]["rho"]))
        mg.mg_profile(h, prof)
        status, st = mg.mg_solve(h, 1, allow_noconv=True)
        bottoms = mg.mg_profile_read(h).get("bottom", (0,))[0] if prof else None
        out = []
        for l in range(H.num_levels):
            phi = torch.zeros((H.n[l],) * H.dim, dtype=torch.float64, device="cuda")
            F = torch.zeros((H.dim,) + (H.n[l],) * H.dim, dtype=torch.float64, device="cuda")
            mg.mg_forces(h, 0, l, phi, F)
            torch.cuda.synchronize()
            out.append((phi.cpu().numpy(), F.cpu().numpy(), dict(st[0][l])))
        return status, out, bottoms
    finally:
        mg.mg_destroy(h)


@pytest.mark.parametrize("make", [lambda: I.config_3d_offset_sphere(64, 4), lambda: I.random_hierarchy(11),
                                  lambda: I.config_2d_disk(64, 3)])
def test_adaptive_inner_cycles(mg, make):
    """Mixed precision with each defect-correction step choosing its FP32
    V-cycles (inner_max > 0): converges to the tolerance, stays within the
    mixed form's bar against FP64, counts exactly the V-cycles it ran (one
    one-block launch per V-cycle), takes no more outer steps than fixed steps
    of inner_cycles, and the graph's device-side choices equal the host
    loop's."""
    H = make()
    inp = I.level_inputs(H)
    kw = dict(nu_pre=2, nu_post=2, max_cycles=60, rel_tol=1e-10, precision=mg.MG_MIXED, inner_cycles=3)
    s64, r64, _ = _solve_with(mg, H, inp, False, **dict(kw, precision=mg.MG_FP64))
    sfx, rfx, _ = _solve_with(mg, H, inp, False, **kw)
    sg, rg, _ = _solve_with(mg, H, inp, False, inner_max=6, **kw)
    sh, rh, bottoms = _solve_with(mg, H, inp, True, inner_max=6, **kw)
    assert s64 == sfx == sg == sh == mg.MG_OK
    X = [H.centres(l, 0) for l in range(H.num_levels)]
    for l in range(H.num_levels):
        phi, F, st = rg[l]
        assert st["rel_res"] < 1e-10, (l, st)
        assert st["outer_steps"] <= rfx[l][2]["outer_steps"], (l, st, rfx[l][2])
        disc = np.max(np.abs(r64[l][0] - H.potential(X[l])))
        assert np.max(np.abs(phi - r64[l][0])) < 1e-2 * disc, l
        assert relmax(phi, r64[l][0]) < 1e-7 and relmax(F, r64[l][1]) < 1e-7, l
        assert np.array_equal(phi, rh[l][0]) and np.array_equal(F, rh[l][1]), l
        assert st["cycles"] == rh[l][2]["cycles"] and st["outer_steps"] == rh[l][2]["outer_steps"], l
    assert bottoms == sum(rh[l][2]["cycles"] for l in range(H.num_levels))


@pytest.mark.parametrize("prof", [False, True])
def test_registered_outputs_equal_mg_forces(mg, prof):
    """mg_solve writes the registered outputs (device and page-locked host,
    potential with forces or forces alone) with the values mg_forces gives,
    in the solve graph (two hierarchies as branches) and in the host-driven
    loop; an unregistered level is left alone; pageable host memory and a
    potential without forces are refused."""
    import torch
    Hs = [I.config_3d_offset_sphere(32, 3), I.random_hierarchy(4)]
    h = mg.mg_create_hierarchy([mg.desc_from(H) for H in Hs], mg.options(nu_pre=2, nu_post=2))
    try:
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        for b, H in enumerate(Hs):
            inp = I.level_inputs(H)
            mg.mg_set_density(h, b, 0, dev(inp[0]["rho"]), dev(inp[0]["bc_rho"]), dev(inp[0]["bc_phi"]))
            for l in range(1, H.num_levels):
                mg.mg_set_density(h, b, l, dev(inp[l]["rho"]))
        shp = lambda H, l: ((H.n[l],) * 3, (3,) + (H.n[l],) * 3)
        outs = {}
        for b, H in enumerate(Hs):
            for l in range(H.num_levels):
                ps, fs = shp(H, l)
                if (b, l) == (0, 1):                      # page-locked host
                    P = torch.full(ps, 7.0, dtype=torch.float64).pin_memory()
                    F = torch.full(fs, 7.0, dtype=torch.float64).pin_memory()
                elif (b, l) == (0, 2):                    # forces alone
                    P, F = None, torch.full(fs, 7.0, dtype=torch.float64, device="cuda")
                else:
                    P, F = (torch.full(ps, 7.0, dtype=torch.float64, device="cuda"),
                            torch.full(fs, 7.0, dtype=torch.float64, device="cuda"))
                mg.mg_set_outputs(h, b, l, P, F)
                outs[(b, l)] = (P, F)
        # registered, then unregistered: stays untouched
        mg.mg_set_outputs(h, 1, 1, None, None)
        with pytest.raises(mg.MGError):
            mg.mg_set_outputs(h, 0, 0, np.zeros(shp(Hs[0], 0)[0]), np.zeros(shp(Hs[0], 0)[1]))
        with pytest.raises(mg.MGError):
            mg.mg_set_outputs(h, 0, 0, torch.zeros(shp(Hs[0], 0)[0], dtype=torch.float64, device="cuda"), None)
        mg.mg_profile(h, prof)
        mg.mg_solve(h, 2, allow_noconv=True)
        for (b, l), (P, F) in outs.items():
            ps, fs = shp(Hs[b], l)
            rp = torch.zeros(ps, dtype=torch.float64, device="cuda")
            rf = torch.zeros(fs, dtype=torch.float64, device="cuda")
            mg.mg_forces(h, b, l, rp, rf)
            torch.cuda.synchronize()
            if (b, l) == (1, 1):
                assert torch.all(P.cpu() == 7.0) and torch.all(F.cpu() == 7.0)
                continue
            assert np.array_equal(F.cpu().numpy(), rf.cpu().numpy()), (b, l)
            if P is not None:
                assert np.array_equal(P.cpu().numpy(), rp.cpu().numpy()), (b, l)
    finally:
        mg.mg_destroy(h)


def test_heterogeneous_batch(mg):
    """Uneven hierarchies solved together (parallel branches of the solve
    graph) give the same results as each solved alone."""
    Hs = [I.random_hierarchy(s) for s in range(5)]
    Hs = [H for H in Hs if max(H.n) <= 96][:3]
    import torch
    h = mg.mg_create_hierarchy([mg.desc_from(H) for H in Hs], mg.options())
    try:
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        for b, H in enumerate(Hs):
            inp = I.level_inputs(H)
            mg.mg_set_density(h, b, 0, dev(inp[0]["rho"]), dev(inp[0]["bc_rho"]), dev(inp[0]["bc_phi"]))
            for l in range(1, H.num_levels):
                mg.mg_set_density(h, b, l, dev(inp[l]["rho"]))
        _, st = mg.mg_solve(h, len(Hs))
        for b, H in enumerate(Hs):
            _, alone = gpu_solve(mg, H, I.level_inputs(H), allow_noconv=False)
            for l in range(H.num_levels):
                phi = torch.zeros((H.n[l],) * 3, dtype=torch.float64, device="cuda")
                mg.mg_forces(h, b, l, phi, None)
                torch.cuda.synchronize()
                assert st[b][l]["cycles"] == alone[l]["cycles"]
                assert np.array_equal(phi.cpu().numpy(), alone[l]["phi"])
    finally:
        mg.mg_destroy(h)


@pytest.mark.parametrize("n,levels,dim", [(64, 4, 3), (32, 3, 3), (64, 3, 2)])
def test_mixed_temporal_blocking_matches_one_kernel_per_phase(mg, n, levels, dim, monkeypatch):
    """The temporally blocked FP32 legs (tile + halo in shared memory) repeat
    the one-kernel-per-phase arithmetic; only FMA contraction may differ."""
    H = I.config_3d_offset_sphere(n, levels) if dim == 3 else I.config_2d_disk(n, levels)
    inp = I.level_inputs(H)
    res = {}
    for tile in ("0", None):
        if tile is None:
            monkeypatch.delenv("MG_TB_TILE", raising=False)
        else:
            monkeypatch.setenv("MG_TB_TILE", tile)
        _, res[tile] = gpu_solve(mg, H, inp, nu_pre=2, nu_post=2, precision=mg.MG_MIXED, allow_noconv=False)
    for l in range(H.num_levels):
        a, b = res["0"][l], res[None][l]
        assert abs(a["cycles"] - b["cycles"]) <= 3
        assert relmax(b["phi"], a["phi"]) < 1e-8 and relmax(b["F"], a["F"]) < 1e-7


def test_batched_mixed_equals_per_hierarchy_branches(mg, monkeypatch):
    """The batched mixed-precision solve (one launch per phase over every
    hierarchy of the batch, converged ones masked) gives the results of the
    per-hierarchy solve graph."""
    import torch
    Hs = [I.random_hierarchy(s) for s in range(12)]
    Hs = [H for H in Hs if max(H.n) <= 96][:5]
    res = {}
    monkeypatch.setenv("MG_SPLIT", "0")                 # the batched kernels run plain-layout levels
    for mode in ("0", "1"):
        monkeypatch.setenv("MG_BATCHED", mode)
        h = mg.mg_create_hierarchy([mg.desc_from(H) for H in Hs], mg.options(precision=mg.MG_MIXED, nu_pre=2,
                                                                             nu_post=2))
        try:
            dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
            for b, H in enumerate(Hs):
                inp = I.level_inputs(H)
                mg.mg_set_density(h, b, 0, dev(inp[0]["rho"]), dev(inp[0]["bc_rho"]), dev(inp[0]["bc_phi"]))
                for l in range(1, H.num_levels):
                    mg.mg_set_density(h, b, l, dev(inp[l]["rho"]))
            _, st = mg.mg_solve(h, len(Hs))
            out = []
            for b, H in enumerate(Hs):
                lev = []
                for l in range(H.num_levels):
                    phi = torch.zeros((H.n[l],) * 3, dtype=torch.float64, device="cuda")
                    mg.mg_forces(h, b, l, phi, None)
                    torch.cuda.synchronize()
                    lev.append((phi.cpu().numpy(), st[b][l]["cycles"], st[b][l]["rel_res"]))
                out.append(lev)
            res[mode] = out
        finally:
            mg.mg_destroy(h)
    for a_h, b_h in zip(res["0"], res["1"]):
        for (pa, ca, ra), (pb, cb, rb) in zip(a_h, b_h):
            assert ca == cb and rb < 1e-10
            assert relmax(pb, pa) < 1e-10


def test_autotune_keeps_results_and_caches(mg, tmp_path):
    """Autotuning only changes the launch plan: the mixed solve gives the
    same results; a second hierarchy takes the plan from the cache."""
    import torch
    H = I.config_3d_offset_sphere(64, 2)
    inp = I.level_inputs(H)
    _, plain = gpu_solve(mg, H, inp, nu_pre=2, nu_post=2, precision=mg.MG_MIXED, allow_noconv=False)
    cache = str(tmp_path / "tune.txt")
    plans = []
    for rep in range(2):
        h = mg.mg_create_hierarchy([mg.desc_from(H)], mg.options(nu_pre=2, nu_post=2, precision=mg.MG_MIXED))
        try:
            mg.mg_autotune(h, cache)
            plans.append(mg.mg_tuning(h, 0, 0))
            dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
            mg.mg_set_density(h, 0, 0, dev(inp[0]["rho"]), dev(inp[0]["bc_rho"]), dev(inp[0]["bc_phi"]))
            mg.mg_set_density(h, 0, 1, dev(inp[1]["rho"]))
            _, st = mg.mg_solve(h, 1)
            for l in range(H.num_levels):
                phi = torch.zeros((64,) * 3, dtype=torch.float64, device="cuda")
                mg.mg_forces(h, 0, l, phi, None)
                torch.cuda.synchronize()
                assert st[0][l]["rel_res"] < 1e-10
                assert relmax(phi.cpu().numpy(), plain[l]["phi"]) < 1e-8
        finally:
            mg.mg_destroy(h)
    assert plans[0] == plans[1]
    assert len(open(cache).read().strip().splitlines()) == 1


# --------------------------------------------------------------------------
# the cluster V-cycle (levels from Lc down in one thread-block cluster)
# --------------------------------------------------------------------------
def _solve_profiled(mg, H, inp, **kw):
    """gpu_solve plus the per-kernel launch counts of the same solve."""
    import torch
    h = mg.mg_create_hierarchy([mg.desc_from(H)], mg.options(**kw))
    try:
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        for l in range(H.num_levels):
            if l == 0:
                mg.mg_set_density(h, 0, 0, dev(inp[0]["rho"]), dev(inp[0]["bc_rho"]), dev(inp[0]["bc_phi"]))
            else:
                mg.mg_set_density(h, 0, l, dev(inp[l]["rho"]))
        mg.mg_profile(h, 1)
        mg.mg_solve(h, 1, allow_noconv=True)
        prof = mg.mg_profile_read(h)
        out = []
        for l in range(H.num_levels):
            n = H.n[l]
            phi = torch.zeros((n,) * H.dim, dtype=torch.float64, device="cuda")
            F = torch.zeros((H.dim,) + (n,) * H.dim, dtype=torch.float64, device="cuda")
            mg.mg_forces(h, 0, l, phi, F)
            torch.cuda.synchronize()
            out.append((phi.cpu().numpy(), F.cpu().numpy()))
        return out, prof
    finally:
        mg.mg_destroy(h)


@pytest.mark.parametrize("make,prec,lim", [
    (lambda: I.config_3d_offset_sphere(64, 4), "mixed", 33),
    (lambda: I.config_3d_offset_sphere(64, 4), "mixed", 17),
    (lambda: I.config_3d_offset_sphere(64, 4), "fp64", 17),
    (lambda: I.config_3d_offset_sphere(64, 4), "fp64", 33),
    (lambda: I.config_3d_offset_sphere(32, 3), "mixed", 34),
    (lambda: I.paper_3d(48), "fp64", 25),
    (lambda: I.random_hierarchy(7), "mixed", 50)])
def test_cluster_vcycle_matches_one_kernel_per_phase(mg, make, prec, lim, monkeypatch):
    """The V-cycle from a level down in one cluster with the levels in
    distributed shared memory gives bit-identical results."""
    H = make()
    inp = I.level_inputs(H)
    p = mg.MG_FP64 if prec == "fp64" else mg.MG_MIXED
    kw = dict(nu_pre=2, nu_post=2, max_cycles=4, rel_tol=0.0, precision=p, inner_cycles=2)
    var = "MG_CLUSTER_N64" if prec == "fp64" else "MG_CLUSTER_N32"
    monkeypatch.setenv("MG_SPLIT", "0")             # the cluster kernel runs plain-layout levels
    monkeypatch.setenv("MG_CLUSTER_N64", "0")
    monkeypatch.setenv("MG_CLUSTER_N32", "0")
    a, pa = _solve_profiled(mg, H, inp, **kw)
    monkeypatch.setenv(var, str(lim))
    b, pb = _solve_profiled(mg, H, inp, **kw)
    assert "cluster_vcycle" not in pa and pb["cluster_vcycle"][0] > 0, pb
    for l in range(H.num_levels):
        assert np.array_equal(a[l][0], b[l][0]), (l, relmax(b[l][0], a[l][0]))
        assert np.array_equal(a[l][1], b[l][1]), l


@pytest.mark.parametrize("make,prec,lim", [
    (lambda: I.config_3d_offset_sphere(64, 3), "fp64", 8),
    (lambda: I.config_3d_offset_sphere(64, 3), "mixed", 8),
    (lambda: I.config_3d_offset_sphere(32, 3), "fp64", 17),
    (lambda: I.paper_3d(48), "mixed", 13),
    (lambda: I.config_2d_disk(64, 3), "fp64", 33),
    (lambda: I.config_2d_disk(64, 3), "mixed", 17)])
def test_one_block_bottom_matches_one_kernel_per_phase(mg, make, prec, lim, monkeypatch):
    """The multigrid levels from N <= lim down in the one-block kernel (every
    array in shared memory, smoothing from its per-cell plan) give results
    bit-identical to one kernel per phase on every level but the last."""
    H = make()
    inp = I.level_inputs(H)
    p = mg.MG_FP64 if prec == "fp64" else mg.MG_MIXED
    kw = dict(nu_pre=2, nu_post=2, max_cycles=4, rel_tol=0.0, precision=p, inner_cycles=2)
    for v in ("MG_BOTTOM_N64", "MG_BOTTOM_N32", "MG_CLUSTER_N64", "MG_CLUSTER_N32", "MG_WAVE"):
        monkeypatch.setenv(v, "0")
    a, pa = _solve_profiled(mg, H, inp, **kw)
    monkeypatch.setenv("MG_BOTTOM_N64", str(lim))
    monkeypatch.setenv("MG_BOTTOM_N32", str(lim))
    b, pb = _solve_profiled(mg, H, inp, **kw)
    assert pb.get("smooth_colour", (0,))[0] < pa["smooth_colour"][0], (pa, pb)
    for l in range(H.num_levels):
        assert np.array_equal(a[l][0], b[l][0]), (l, relmax(b[l][0], a[l][0]))
        assert np.array_equal(a[l][1], b[l][1]), l


def test_cluster_vcycle_is_3d_only(mg, monkeypatch):
    H = I.config_2d_disk(64, 3)
    inp = I.level_inputs(H)
    monkeypatch.setenv("MG_CLUSTER_N64", "33")
    monkeypatch.setenv("MG_CLUSTER_N32", "33")
    b, pb = _solve_profiled(mg, H, inp, max_cycles=3, rel_tol=0.0)
    assert "cluster_vcycle" not in pb


# --------------------------------------------------------------------------
# plane-marching FP32 sweeps (all colour passes of a smoothing stint in one
# launch, out of place) against one launch per colour
# --------------------------------------------------------------------------
@pytest.mark.parametrize("make,nu", [
    (lambda: I.config_3d_offset_sphere(64, 3), (2, 2)),
    (lambda: I.config_3d_offset_sphere(64, 2), (2, 1)),
    (lambda: I.config_3d_offset_sphere(32, 3), (1, 1)),
    (lambda: I.paper_3d(48), (2, 2)),
    (lambda: I.paper_3d(48), (1, 2)),
    (lambda: I.random_hierarchy(7), (2, 2)),
    (lambda: I.random_hierarchy(3), (2, 1))])
def test_wave_sweeps_match_one_colour_kernels(mg, make, nu, monkeypatch):
    """Every multigrid level above the one-block kernel smoothed by the
    plane-marching kernel (tile ring recomputed per block, ping-pong arrays)
    gives potential and forces bit-identical to one launch per colour; the
    multigrid sizes include odd, tie (x_N = 1) and non-tie levels."""
    H = make()
    inp = I.level_inputs(H)
    kw = dict(nu_pre=nu[0], nu_post=nu[1], max_cycles=4, rel_tol=0.0, precision=mg.MG_MIXED, inner_cycles=2)
    monkeypatch.setenv("MG_WAVE", "0")
    a, pa = _solve_profiled(mg, H, inp, **kw)
    monkeypatch.setenv("MG_WAVE", "1")
    b, pb = _solve_profiled(mg, H, inp, **kw)
    assert "smooth_wave" not in pa and "smooth_wave_finest" not in pa
    assert pb["smooth_wave_finest"][0] > 0 and "smooth_colour_finest" not in pb, pb
    for l in range(H.num_levels):
        assert np.array_equal(a[l][0], b[l][0]), (l, relmax(b[l][0], a[l][0]))
        assert np.array_equal(a[l][1], b[l][1]), l


@pytest.mark.parametrize("zc", ["1", "5"])
def test_wave_converged_adaptive_equals_one_colour(mg, zc, monkeypatch):
    """Converged mixed solve with adaptive correction steps (the last sweep
    launch of each FP32 V-cycle counts it in the nested graph loop): same
    cycle counts and bit-identical results with and without the sweeps."""
    H = I.config_3d_offset_sphere(64, 4)
    inp = I.level_inputs(H)
    kw = dict(nu_pre=2, nu_post=2, precision=mg.MG_MIXED, inner_max=8, allow_noconv=False)
    monkeypatch.setenv("MG_WAVE", "0")
    _, a = gpu_solve(mg, H, inp, **kw)
    monkeypatch.setenv("MG_WAVE", "1")
    monkeypatch.setenv("MG_WAVE_PLAN", f"1,{zc}")
    _, b = gpu_solve(mg, H, inp, **kw)
    for l in range(H.num_levels):
        assert a[l]["cycles"] == b[l]["cycles"] and b[l]["rel_res"] < 1e-10
        assert np.array_equal(a[l]["phi"], b[l]["phi"]) and np.array_equal(a[l]["F"], b[l]["F"])


def test_time_smoothing_reports_plan_bytes(mg, monkeypatch):
    """mg_time_smoothing times the level's smoothing in its plan's launch
    form and states the algorithmic bytes of one launch (3 words per cell for
    a plane-marching launch, 1.5 for one colour)."""
    H = I.config_3d_offset_sphere(64, 2)
    for wave in ("1", "0"):
        monkeypatch.setenv("MG_WAVE", wave)
        h = mg.mg_create_hierarchy([mg.desc_from(H)], mg.options(nu_pre=2, nu_post=2, precision=mg.MG_MIXED))
        try:
            tiles, _ = mg.mg_tuning(h, 0, 0)
            us, by = mg.mg_time_smoothing(h, 0, 0, 0, 8)
            N = 66
            assert us > 0.0
            assert by == (3.0 if wave == "1" else 1.5) * 4 * N ** 3
            assert (tiles[0] < 0) == (wave == "1")
            with pytest.raises(mg.MGError):
                mg.mg_time_smoothing(h, 0, 0, 12, 8)   # the one-block kernel's levels are not per-level launches
        finally:
            mg.mg_destroy(h)


def test_wave_load_wait_timeout_reports_etimeout(mg, monkeypatch):
    """Every mbarrier wait of the plane-marching kernel has a clock budget.
    With MG_FAULT_WAVE_WAIT=1 one load group of every block is never issued
    (a wait nothing completes; budget about 1 ms): the blocks record the
    timeout and return, mg_solve reports MG_ETIMEOUT and the handle refuses
    further work; the GPU stays usable and a new handle solves normally."""
    H = I.config_3d_offset_sphere(32, 2)
    inp = I.level_inputs(H)
    kw = dict(nu_pre=2, nu_post=2, max_cycles=2, rel_tol=0.0, precision=mg.MG_MIXED, inner_cycles=1)
    monkeypatch.setenv("MG_WAVE", "1")
    monkeypatch.setenv("MG_FAULT_WAVE_WAIT", "1")
    with pytest.raises(mg.MGError) as ei:
        gpu_solve(mg, H, inp, **kw)
    assert ei.value.status == mg.MG_ETIMEOUT, ei.value
    monkeypatch.delenv("MG_FAULT_WAVE_WAIT")
    _, good = gpu_solve(mg, H, inp, **kw)
    monkeypatch.setenv("MG_WAVE", "0")
    _, plain = gpu_solve(mg, H, inp, **kw)
    for l in range(H.num_levels):
        assert np.array_equal(good[l]["phi"], plain[l]["phi"])


# --------------------------------------------------------------------------
# colour-split FP32 levels (mixed precision)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("make,split,want", [
    (lambda: I.config_3d_offset_sphere(64, 3), "1", 1),
    (lambda: I.config_3d_offset_sphere(128, 2), "2", 2),
    (lambda: I.config_3d_offset_sphere(64, 3), "9", None),       # every level above the one-block bottom
    (lambda: I.config_2d_disk(256, 2), "", 1),                   # default: levels of >= 192 cells per edge
    (lambda: I.config_2d_disk(64, 2), "9", None)])
def test_split_levels_match_plain_layout(mg, make, split, want, monkeypatch):
    """FP32 levels stored colour-split and run by the box-patch kernels
    reach the same tolerance as the plain layout, with cycle counts within
    one and potentials within 1e-8 of each other (only FP32 rounding
    differs); mg_tuning reports the split levels as 65536."""
    import torch
    H = make()
    inp = I.level_inputs(H)
    res, plans = {}, {}
    for mode in ("0", split):
        monkeypatch.setenv("MG_SPLIT", mode)
        h = mg.mg_create_hierarchy([mg.desc_from(H)], mg.options(nu_pre=2, nu_post=2, precision=mg.MG_MIXED,
                                                                 inner_max=8))
        try:
            plans[mode] = [mg.mg_tuning(h, 0, l) for l in range(H.num_levels)]
            dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
            mg.mg_set_density(h, 0, 0, dev(inp[0]["rho"]), dev(inp[0]["bc_rho"]), dev(inp[0]["bc_phi"]))
            for l in range(1, H.num_levels):
                mg.mg_set_density(h, 0, l, dev(inp[l]["rho"]))
            _, st = mg.mg_solve(h, 1)
            out = []
            for l in range(H.num_levels):
                phi = torch.zeros((H.n[l],) * H.dim, dtype=torch.float64, device="cuda")
                mg.mg_forces(h, 0, l, phi, None)
                torch.cuda.synchronize()
                out.append((phi.cpu().numpy(), st[0][l]["cycles"], st[0][l]["rel_res"]))
            res[mode] = out
        finally:
            mg.mg_destroy(h)
    for l in range(H.num_levels):
        tiles0, nb0 = plans["0"][l]
        tiles, nb = plans[split][l]
        assert 65536 not in tiles0
        nsplit = sum(1 for t in tiles if t == 65536)
        assert tiles[:nsplit] == [65536] * nsplit and 65536 not in tiles[nsplit:]
        if want is not None:
            assert nsplit == want, tiles
        else:
            # every level above the one-block kernel (edge nb) is split
            Ns = mg.mg_level_sizes(H.n[l] + 2)
            assert nsplit == Ns.index(nb), (tiles, nb)
        (pa, ca, ra), (pb, cb, rb) = res["0"][l], res[split][l]
        assert ra < 1e-10 and rb < 1e-10
        assert abs(ca - cb) <= 1, (ca, cb)
        assert relmax(pb, pa) < 1e-8, relmax(pb, pa)


def test_split_smoothing_timed_with_split_bytes(mg, monkeypatch):
    """mg_time_smoothing times the split colour pass where the plan has one
    (1.5 words per active cell)."""
    monkeypatch.setenv("MG_SPLIT", "1")
    H = I.config_3d_offset_sphere(64, 2)
    h = mg.mg_create_hierarchy([mg.desc_from(H)], mg.options(precision=mg.MG_MIXED))
    try:
        assert mg.mg_tuning(h, 0, 0)[0][0] == 65536
        us, by = mg.mg_time_smoothing(h, 0, 0, 0, 8)
        assert us > 0 and by == 1.5 * 4 * 66 ** 3
    finally:
        mg.mg_destroy(h)


# --------------------------------------------------------------------------
# the persistent batched solve (one launch for the whole batch)
# --------------------------------------------------------------------------
def _batch_solve(mg, Hs, outputs=False, **kw):
    import torch
    h = mg.mg_create_hierarchy([mg.desc_from(H) for H in Hs], mg.options(**kw))
    try:
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        outs = {}
        for b, H in enumerate(Hs):
            inp = I.level_inputs(H)
            mg.mg_set_density(h, b, 0, dev(inp[0]["rho"]), dev(inp[0]["bc_rho"]), dev(inp[0]["bc_phi"]))
            for l in range(1, H.num_levels):
                mg.mg_set_density(h, b, l, dev(inp[l]["rho"]))
            if outputs:
                for l in range(H.num_levels):
                    shp = (H.n[l],) * H.dim
                    P = torch.zeros(shp, dtype=torch.float64, device="cuda")
                    F = torch.zeros((H.dim,) + shp, dtype=torch.float64, device="cuda")
                    mg.mg_set_outputs(h, b, l, P, F)
                    outs[b, l] = (P, F)
        res = []
        for rep in range(2):                  # the second solve reuses the graph
            for b, H in enumerate(Hs):
                inp = I.level_inputs(H)
                mg.mg_set_density(h, b, 0, dev(inp[0]["rho"]), dev(inp[0]["bc_rho"]), dev(inp[0]["bc_phi"]))
                for l in range(1, H.num_levels):
                    mg.mg_set_density(h, b, l, dev(inp[l]["rho"]))
            _, st = mg.mg_solve(h, len(Hs))
        for b, H in enumerate(Hs):
            lev = []
            for l in range(H.num_levels):
                shp = (H.n[l],) * H.dim
                if outputs:
                    P, F = outs[b, l]
                else:
                    P = torch.zeros(shp, dtype=torch.float64, device="cuda")
                    F = torch.zeros((H.dim,) + shp, dtype=torch.float64, device="cuda")
                    mg.mg_forces(h, b, l, P, F)
                torch.cuda.synchronize()
                lev.append((P.cpu().numpy(), F.cpu().numpy(), st[b][l]))
            res.append(lev)
        return res
    finally:
        mg.mg_destroy(h)


@pytest.mark.parametrize("inner_max,outputs,guess", [(8, False, 0), (0, True, 0), (8, True, 1)])
def test_persistent_batch_equals_graph_branches(mg, monkeypatch, inner_max, outputs, guess):
    """One persistent launch over the batch (a block per hierarchy, levels in
    order) gives the cycle counts and results of the per-hierarchy graph
    branches: the same per-cell arithmetic, norms summed in another order."""
    Hs = [I.random_hierarchy(s) for s in range(14)]
    Hs = [H for H in Hs if max(H.n) <= 96][:6]
    monkeypatch.setenv("MG_SPLIT", "0")
    kw = dict(precision=mg.MG_MIXED, nu_pre=2, nu_post=2, inner_max=inner_max, guess=guess)
    monkeypatch.setenv("MG_PERSIST", "0")
    a = _batch_solve(mg, Hs, outputs, **kw)
    monkeypatch.setenv("MG_PERSIST", "1")
    b = _batch_solve(mg, Hs, outputs, **kw)
    for ha, hb in zip(a, b):
        for (pa, Fa, sa), (pb, Fb, sb) in zip(ha, hb):
            assert sb["status"] == 0 and sb["rel_res"] < 1e-10
            assert sa["cycles"] == sb["cycles"] and sa["outer_steps"] == sb["outer_steps"], (sa, sb)
            assert relmax(pb, pa) < 1e-10 and relmax(Fb, Fa) < 1e-9


def test_persistent_batch_2d(mg, monkeypatch):
    Hs = [I.config_2d_disk(n, 3) for n in (32, 64, 48, 64, 96)]
    monkeypatch.setenv("MG_SPLIT", "0")
    kw = dict(precision=mg.MG_MIXED, nu_pre=2, nu_post=2, inner_max=8)
    monkeypatch.setenv("MG_PERSIST", "0")
    a = _batch_solve(mg, Hs, **kw)
    monkeypatch.setenv("MG_PERSIST", "1")
    b = _batch_solve(mg, Hs, **kw)
    for ha, hb in zip(a, b):
        for (pa, Fa, sa), (pb, Fb, sb) in zip(ha, hb):
            assert sa["cycles"] == sb["cycles"] and sb["rel_res"] < 1e-10
            assert relmax(pb, pa) < 1e-10


def test_mixed_persistent_and_graph_branches(mg, monkeypatch):
    """The smallest hierarchies in the persistent launch, the others as graph
    branches beside it in the same graph, as the cost model splits a batch:
    results and cycle counts as with graph branches only."""
    Hs = [I.random_hierarchy(s, edges=(16, 24, 32)) for s in range(6)] + \
         [I.random_hierarchy(s) for s in range(20, 24)]
    monkeypatch.setenv("MG_SPLIT", "0")
    kw = dict(precision=mg.MG_MIXED, nu_pre=2, nu_post=2, inner_max=8)
    monkeypatch.setenv("MG_PERSIST", "0")
    a = _batch_solve(mg, Hs, True, **kw)
    monkeypatch.delenv("MG_PERSIST")
    monkeypatch.setenv("MG_PERSIST_COUNT", "6")
    b = _batch_solve(mg, Hs, True, **kw)
    monkeypatch.delenv("MG_PERSIST_COUNT")
    c = _batch_solve(mg, Hs, True, **kw)          # the cost model's own split
    for ha, hb, hc in zip(a, b, c):
        for (pa, Fa, sa), (pb, Fb, sb), (pc, Fc, sc) in zip(ha, hb, hc):
            assert sa["cycles"] == sb["cycles"] == sc["cycles"]
            assert relmax(pb, pa) < 1e-10 and relmax(pc, pa) < 1e-10 and relmax(Fb, Fa) < 1e-9
