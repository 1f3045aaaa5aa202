"""mg_solve_level_noalloc: the allocation-free single-level solve.

Some callers cannot allocate device memory (their own pool owns the GPU, or
the solve runs inside a time step where cudaMalloc/cudaFree and the
synchronisation they imply are not allowed).  For them the library has one
entry point whose working memory is a fixed device array inside the library.
These tests check, through the C ABI, that it returns what the allocating
entry point (mg_create_hierarchy / mg_set_density / mg_solve / mg_forces)
returns for the same single-level problem, on two calls in a row of
different sizes (the shared array keeps the first call's contents), and that
sizes beyond its limit are refused before any GPU work.

This file sorts last so that a run stopping at its first failure has already
run every other test.
"""
import numpy as np
import pytest

from paper_2001_02327_gb300 import inputs as I

TOL = 1e-12


def _problem(dim, n, seed):
    rng = np.random.default_rng(I.BASE_SEED + 900 + seed)
    return {"rho": rng.standard_normal((n,) * dim), "bc_rho": rng.standard_normal((n + 2,) * dim),
            "bc_phi": rng.standard_normal((n + 4,) * dim)}


def _blocks(dim, n, p):
    """(n+4)^d density block (solved region filled) and potential block
    (outer ring = Dirichlet data, zero initial guess inside)."""
    rho = np.zeros((n + 4,) * dim)
    rho[(slice(1, n + 3),) * dim] = p["bc_rho"]
    rho[(slice(2, n + 2),) * dim] = p["rho"]
    phi = p["bc_phi"].copy()
    phi[(slice(1, n + 3),) * dim] = 0.0
    return rho, phi


def _allocating(mg, dim, n, h, G, p, opt):
    import torch
    H = I.Hierarchy(dim, [n], [tuple([0.0] * dim)], h, G, [], "single")
    hd = mg.mg_create_hierarchy([mg.desc_from(H)], opt)
    try:
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        mg.mg_set_density(hd, 0, 0, dev(p["rho"]), dev(p["bc_rho"]), dev(p["bc_phi"]))
        _, st = mg.mg_solve(hd, 1, allow_noconv=True)
        phi = torch.zeros((n,) * dim, dtype=torch.float64, device="cuda")
        mg.mg_forces(hd, 0, 0, phi, None)
        torch.cuda.synchronize()
        return phi.cpu().numpy(), st[0][0]
    finally:
        mg.mg_destroy(hd)


@pytest.mark.gpu
def test_no_alloc_matches_allocating_entry_point():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2001_02327_gb300 import build
    build.build()
    from paper_2001_02327_gb300 import mg
    cases = [(3, 46, 0.021, 0.8, mg.options(max_cycles=4, rel_tol=0.0)),     # first call: larger
             (3, 14, 0.05, 1.1, mg.options(nu_pre=2, nu_post=2)),             # second call: smaller, to 1e-10
             (2, 62, 0.017, 0.5, mg.options(max_cycles=3, rel_tol=0.0)),
             (3, 69, 0.014, 1.0, mg.options(max_cycles=2, rel_tol=0.0))]     # the largest 3D size accepted
    prepared = []
    for k, (dim, n, h, G, opt) in enumerate(cases):
        p = _problem(dim, n, k)
        want, st_want = _allocating(mg, dim, n, h, G, p, opt)
        rho, phi = _blocks(dim, n, p)
        prepared.append((want, st_want, torch.from_numpy(rho).cuda(), torch.from_numpy(phi).cuda(), phi))
    # warm-up call (first use on the device looks the array's address up)
    w_rho, w_phi = _blocks(3, 8, _problem(3, 8, 99))
    mg.mg_solve_level_noalloc(3, 8, 0.1, 1.0, torch.from_numpy(w_rho).cuda(), torch.from_numpy(w_phi).cuda(),
                              mg.options(max_cycles=1, rel_tol=0.0))
    torch.cuda.synchronize()
    free0, reserved0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
    results = []
    for k, (dim, n, h, G, opt) in enumerate(cases):
        d_rho, d_phi = prepared[k][2], prepared[k][3]
        results.append(mg.mg_solve_level_noalloc(dim, n, h, G, d_rho, d_phi, opt))
    torch.cuda.synchronize()
    # the calls allocated nothing: the device's free memory and torch's pool are unchanged
    assert torch.cuda.mem_get_info()[0] == free0 and torch.cuda.memory_reserved() == reserved0
    for k, (dim, n, h, G, opt) in enumerate(cases):
        want, st_want, d_rho, d_phi, phi = prepared[k]
        s, st = results[k]
        assert s in (mg.MG_OK, mg.MG_ENOCONV)
        assert st["cycles"] == st_want["cycles"]
        got = d_phi.cpu().numpy()[(slice(2, n + 2),) * dim]
        err = np.max(np.abs(got - want)) / np.max(np.abs(want))
        assert err < TOL, (k, err)
        # the outer ring (Dirichlet data) is left as it was
        ring = np.ones((n + 4,) * dim, dtype=bool)
        ring[(slice(1, n + 3),) * dim] = False
        assert np.array_equal(d_phi.cpu().numpy()[ring], phi[ring])


def test_no_alloc_rejects_sizes_beyond_its_array():
    """Refused on the host, before any CUDA call, with MG_EINVAL."""
    from paper_2001_02327_gb300 import build
    build.build()
    from paper_2001_02327_gb300 import mg
    for dim, n in ((3, 70), (3, 80), (3, 200), (2, 555), (2, 2000)):   # 70 and 555: one past the limits
        s, _ = mg.mg_solve_level_noalloc(dim, n, 0.01, 1.0, 1 << 20, 1 << 20)
        assert s == mg.MG_EINVAL


@pytest.mark.gpu
def test_no_alloc_refuses_a_capturing_stream():
    """The call waits on the host for its norms; on a stream that is
    capturing a graph it returns MG_EINVAL before queuing anything, and the
    capture stays intact."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2001_02327_gb300 import build
    build.build()
    from paper_2001_02327_gb300 import mg
    rho, phi = _blocks(3, 8, _problem(3, 8, 5))
    d_rho, d_phi = torch.from_numpy(rho).cuda(), torch.from_numpy(phi).cuda()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        st, _ = mg.mg_solve_level_noalloc(3, 8, 0.1, 1.0, d_rho, d_phi, mg.options(stream=s))
        d_phi.add_(0.0)   # the capture goes on after the refusal
    assert st == mg.MG_EINVAL
    g.replay()
    torch.cuda.synchronize()
