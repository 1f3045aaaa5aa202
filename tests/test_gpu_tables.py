"""Tables 1 and 2 (Sec. 3.1, 3.2) reproduced on the GPU at every N the paper
prints, with the paper's stopping test (the acceleration changes by less than
1e-10 between cycles), and the frozen-interface comparison of Sec. 4 at the
same sizes.  Error norms are taken over the composite grid against the closed
forms; the printed values are the golden fixtures under tests/golden/.

Set MG_FIG3_OUT to a file name to also write the Fig. 3 data of the 2D
model (cell radius, radial-acceleration error and level of every cell of the
composite grid, N = 128) as an .npz archive.
"""
import os

import numpy as np
import pytest

from paper_2001_02327_gb300 import inputs as I

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def mg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2001_02327_gb300 import build
    build.build()
    from paper_2001_02327_gb300 import mg as M
    return M


def _table(name):
    rows = {}
    for line in open(os.path.join(GOLD, name)):
        if line.startswith("#") or not line.strip():
            continue
        v = line.split()
        rows[int(v[0])] = [float(t) for t in v[1:]]
    return rows


def _solve(mg, H, **kw):
    """Solve on the GPU; per level {"phi": (n+4)^d block with Omega filled, "F"}."""
    import torch
    inp = I.level_inputs(H)
    h = mg.mg_create_hierarchy([mg.desc_from(H)], mg.options(**kw))
    try:
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        for l in range(H.num_levels):
            if l == 0:
                mg.mg_set_density(h, 0, 0, dev(inp[0]["rho"]), dev(inp[0]["bc_rho"]), dev(inp[0]["bc_phi"]))
            else:
                mg.mg_set_density(h, 0, l, dev(inp[l]["rho"]))
        _, st = mg.mg_solve(h, 1)
        out = []
        for l in range(H.num_levels):
            n = H.n[l]
            phi = torch.zeros((n,) * H.dim, dtype=torch.float64, device="cuda")
            F = torch.zeros((H.dim,) + (n,) * H.dim, dtype=torch.float64, device="cuda")
            mg.mg_forces(h, 0, l, phi, F)
            torch.cuda.synchronize()
            blk = np.zeros((n + 4,) * H.dim)
            blk[(slice(2, n + 2),) * H.dim] = phi.cpu().numpy()
            out.append({"phi": blk, "F": F.cpu().numpy(), **st[0][l]})
        return out
    finally:
        mg.mg_destroy(h)


def _interface_error(H, res):
    from oracle import norms as NR
    worst = 0.0
    for l in range(1, H.num_levels):
        _, eR = NR.force_errors(H, l, res[l]["F"])
        m = np.ones(eR.shape, bool)
        m[(slice(1, -1),) * H.dim] = False
        worst = max(worst, float(eR[m].max()))
    return worst


@pytest.mark.parametrize("dim,name,Ns,band,band_inf", [
    (2, "table1_2d.txt", (8, 16, 32, 64, 128, 256, 512, 1024), 0.15, 0.05),
    (3, "table2_3d.txt", (8, 16, 32, 64, 128, 256), 0.22, 0.06)])
def test_tables_on_gpu(mg, dim, name, Ns, band, band_inf):
    from oracle import norms as NR
    ref = _table(name)
    prev = None
    for N in Ns:
        H = I.paper_2d(N) if dim == 2 else I.paper_3d(N)
        res = _solve(mg, H, nu_pre=2, nu_post=1, max_cycles=80, rel_tol=1e-10, stop=mg.MG_STOP_FORCE)
        for l, r in enumerate(res):
            assert r["status"] == mg.MG_OK and r["rel_res"] < 1e-10, (N, l, r["rel_res"])
        nm = NR.hierarchy_norms(H, res)
        got = np.array(list(nm["x"]) + list(nm["R"]))
        want = np.array(ref[N])
        assert np.all(np.abs(got / want - 1) <= band), (N, got, want)
        assert abs(got[2] / want[2] - 1) < band_inf and abs(got[5] / want[5] - 1) < band_inf, (N, got, want)
        if prev is not None and N >= 32:
            order = np.log2(prev / got)
            assert np.all(order > 1.8) and np.all(order < 2.2), (N, order)
        prev = got
        if dim == 2 and N == 128 and os.environ.get("MG_FIG3_OUT"):
            _write_fig3(H, res, os.environ["MG_FIG3_OUT"])


def _write_fig3(H, res, path):
    from oracle import norms as NR
    r, e, lev = [], [], []
    for l in range(H.num_levels):
        X = H.centres(l, 0)
        keep = ~NR.covered_mask(H, l)
        _, eR = NR.force_errors(H, l, res[l]["F"])
        r.append(np.sqrt((X ** 2).sum(axis=-1))[keep])
        e.append(eR[keep])
        lev.append(np.full(int(keep.sum()), l))
    np.savez(path, radius=np.concatenate(r), err_fr=np.concatenate(e), level=np.concatenate(lev))


@pytest.mark.parametrize("dim,Ns", [(2, (128, 256, 512, 1024)), (3, (32, 64, 128))])
def test_frozen_interface_ablation_on_gpu(mg, dim, Ns):
    """Sec. 4's comparison at the table sizes: on the first cells of each
    patch the frozen-ring scheme's force error is larger than the buffer
    method's, and with the interpolated ring as the fine solve's Dirichlet
    boundary it still falls at second order."""
    e = {}
    for N in Ns:
        H = I.paper_2d(N) if dim == 2 else I.paper_3d(N)
        for mode, iface in (("buffer", mg.MG_IFACE_BUFFER), ("frozen", mg.MG_IFACE_FROZEN)):
            res = _solve(mg, H, nu_pre=2, nu_post=1, max_cycles=80, rel_tol=1e-12, interface=iface)
            e[mode, N] = _interface_error(H, res)
    for N in Ns:
        assert e["frozen", N] > 1.2 * e["buffer", N], (N, e)
    for a, b in zip(Ns[:-1], Ns[1:]):
        for mode in ("buffer", "frozen"):
            assert np.log2(e[mode, a] / e[mode, b]) > 1.8, (mode, a, b, e)
