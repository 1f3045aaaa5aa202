"""The learned initial guess: the network's forward pass and gradients on the
GPU against the CPU float64 reference (oracle/unet_ref.py, itself checked by
finite differences), training, and its use inside the solver."""
import numpy as np
import pytest

from paper_2001_02327_gb300 import inputs as I


def _sample(B, n, seed):
    rng = np.random.default_rng(I.BASE_SEED + 500 + seed)
    z, y, x = np.meshgrid(*([np.linspace(-1, 1, n)] * 3), indexing="ij")
    rho = np.stack([np.exp(-((x - a) ** 2 + (y - b) ** 2 + z ** 2) * 6) * (1 + 0.3 * rng.standard_normal((n, n, n)))
                    for a, b in rng.uniform(-0.3, 0.3, size=(B, 2))])
    phi = np.stack([-1.0 / (1.0 + x ** 2 + y ** 2 + (z - c) ** 2) + 0.05 * rng.standard_normal((n, n, n))
                    for c in rng.uniform(-0.2, 0.2, size=B)])
    tru = phi + 0.02 * np.sin(3 * x) * np.cos(2 * y) + 0.01 * rng.standard_normal((B, n, n, n))
    frho = rng.uniform(0.5, 2.0, size=B) * 0.01
    import torch
    from oracle import unet_ref as R
    res = R.residual_h2(torch.from_numpy(phi), torch.from_numpy(rho), frho).numpy()
    return rho, phi, res, tru, frho


# --------------------------------------------------------------------------
# CPU: the reference is pinned by finite differences
# --------------------------------------------------------------------------
def test_reference_param_count():
    from oracle import unet_ref as R
    # nine 3x3x3 convolutions (3->16, 16->16, 16->32, 32->32, 32->64, 64->64,
    # 128->32, 64->16, 32->16) with biases, then a 1x1 16->1 output
    assert R.param_count() == 367937


def test_reference_gradient_by_finite_differences():
    torch = pytest.importorskip("torch")
    from oracle import unet_ref as R
    rng = np.random.default_rng(3)
    p = rng.standard_normal(R.param_count()) * 0.2
    rho, phi, res, tru, frho = _sample(1, 8, 0)
    T = lambda a: torch.from_numpy(a)
    L, g = R.loss_and_grad(p, T(rho), T(phi), T(res), T(tru), frho)
    # parameters spread over the layers, including biases and the output layer
    idx = [0, 100, 900, 1295, 9000, 30000, 60000, 150000, 250000, 330000, 367920, 367936]
    for i in idx:
        e = 1e-4      # the loss is O(1e3): smaller steps lose digits to round-off
        pp, pm = p.copy(), p.copy()
        pp[i] += e
        pm[i] -= e
        lp, _ = R.loss_and_grad(pp, T(rho), T(phi), T(res), T(tru), frho)
        lm, _ = R.loss_and_grad(pm, T(rho), T(phi), T(res), T(tru), frho)
        fd = (lp - lm) / (2 * e)
        assert abs(fd - g[i]) <= 1e-5 * max(1.0, abs(fd)) + 1e-7, (i, fd, g[i])


# --------------------------------------------------------------------------
# GPU
# --------------------------------------------------------------------------
@pytest.fixture(scope="module")
def un():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2001_02327_gb300 import build
    build.build()
    from paper_2001_02327_gb300 import unet as U
    return U


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.gpu
@pytest.mark.parametrize("n,B", [(8, 2), (16, 1)])
def test_forward_matches_reference(un, n, B):
    import torch
    from oracle import unet_ref as R
    u = un.mg_unet_create(16, 2, seed=7)
    try:
        p = un.mg_unet_get_params(u).astype(np.float64)
        rho, phi, res, tru, frho = _sample(B, n, 1)
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        y = un.mg_unet_forward(u, B, n, dev(rho), dev(phi), dev(res), frho)
        T = torch.from_numpy
        yr, _ = R.forward(T(p), T(rho), T(phi), T(res), frho)
        # BF16 operands with FP32 accumulation through nine layers
        assert _rel(y, yr.detach().numpy()) < 3e-2
    finally:
        un.mg_unet_destroy(u)


@pytest.mark.gpu
def test_gradient_matches_reference(un):
    import torch
    from oracle import unet_ref as R
    u = un.mg_unet_create(16, 2, seed=11)
    try:
        p = un.mg_unet_get_params(u).astype(np.float64)
        rho, phi, res, tru, frho = _sample(2, 16, 2)
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        loss = un.mg_unet_train_step(u, 2, 16, dev(rho), dev(phi), dev(res), dev(tru), frho, update=False)
        g = un.mg_unet_get_grad(u).astype(np.float64)
        T = lambda a: torch.from_numpy(a)
        lr, gr = R.loss_and_grad(p, T(rho), T(phi), T(res), T(tru), frho)
        assert abs(loss / lr - 1) < 3e-2
        off = 0
        for cin, cout in R.CONV_DIMS:
            nw = 27 * cin * cout
            assert _rel(g[off:off + nw], gr[off:off + nw]) < 8e-2, (cin, cout)
            assert _rel(g[off + nw:off + nw + cout], gr[off + nw:off + nw + cout]) < 8e-2, (cin, cout, "bias")
            off += nw + cout
        assert _rel(g[off:], gr[off:]) < 5e-2
    finally:
        un.mg_unet_destroy(u)


@pytest.mark.gpu
def test_training_reduces_loss(un):
    import torch
    u = un.mg_unet_create(16, 4, seed=5)
    try:
        rho, phi, res, tru, frho = _sample(4, 16, 4)
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        r, p_, q, t = dev(rho), dev(phi), dev(res), dev(tru)
        first = un.mg_unet_train_step(u, 4, 16, r, p_, q, t, frho, lr=2e-3, update=True)
        for _ in range(150):
            last = un.mg_unet_train_step(u, 4, 16, r, p_, q, t, frho, lr=2e-3, update=True)
        assert last < 0.5 * first, (first, last)
    finally:
        un.mg_unet_destroy(u)


@pytest.mark.gpu
def test_learned_guess_in_solver_keeps_accuracy(un):
    """The solver with the learned guess reaches the same residual and the
    same solution as with the interpolated guess (any network: the stopping
    rule decides)."""
    import torch
    from paper_2001_02327_gb300 import mg
    H = I.config_3d_offset_sphere(32, 3)
    inp = I.level_inputs(H)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    u = un.mg_unet_create(32, 1, seed=1)
    res = {}
    try:
        for mode in (mg.MG_GUESS_INTERP, mg.MG_GUESS_LEARNED):
            h = mg.mg_create_hierarchy([mg.desc_from(H)], mg.options(guess=mode, precision=mg.MG_MIXED))
            try:
                if mode == mg.MG_GUESS_LEARNED:
                    un.mg_set_unet(h, u)
                mg.mg_set_density(h, 0, 0, dev(inp[0]["rho"]), dev(inp[0]["bc_rho"]), dev(inp[0]["bc_phi"]))
                for l in range(1, 3):
                    mg.mg_set_density(h, 0, l, dev(inp[l]["rho"]))
                _, st = mg.mg_solve(h, 1)
                out = []
                for l in range(3):
                    phi = torch.zeros((32,) * 3, dtype=torch.float64, device="cuda")
                    mg.mg_forces(h, 0, l, phi, None)
                    torch.cuda.synchronize()
                    out.append((phi.cpu().numpy(), st[0][l]["rel_res"]))
                if mode == mg.MG_GUESS_INTERP:
                    g = torch.zeros((32,) * 3, dtype=torch.float64, device="cuda")
                    r = np.zeros((32,) * 3)
                    un.mg_interp_guess(h, 0, 1, g, r)
                    res["guess1"] = g.cpu().numpy()
                    res["resid1"] = r
                res[mode] = out
            finally:
                mg.mg_destroy(h)
    finally:
        un.mg_unet_destroy(u)
    for (a, ra), (b, rb) in zip(res[mg.MG_GUESS_INTERP], res[mg.MG_GUESS_LEARNED]):
        assert ra < 1e-10 and rb < 1e-10
        assert _rel(b, a) < 1e-8
    # the exported guess is the parent solution interpolated: close to the level's solution
    sol1 = res[mg.MG_GUESS_INTERP][1][0]
    assert _rel(res["guess1"], sol1) < 0.05
    # the exported residual is that of the guess: on cells away from the
    # buffer ring it equals the 7-point residual of the dense guess array
    from oracle import unet_ref as R
    g = res["guess1"]
    h1 = H.h(1)
    fr = [4 * np.pi * H.G * h1 * h1]
    rr = R.residual_h2(torch.from_numpy(g[None]), torch.from_numpy(inp[1]["rho"][None]), fr).numpy()[0]
    inner = (slice(1, -1),) * 3
    assert np.abs(res["resid1"][inner] - rr[inner]).max() <= 1e-12 * max(np.abs(rr).max(), 1e-30) + 1e-15
    # and vanishes (to round-off) for the converged solution: it is a real residual
    assert np.abs(rr[inner]).max() > 1e3 * np.abs(R.residual_h2(torch.from_numpy(sol1[None]),
                                                               torch.from_numpy(inp[1]["rho"][None]), fr)
                                                  .numpy()[0][inner]).max()
