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


def test_reference_tap_layout_by_hand():
    """Flat weights [27][Cin][Cout], tap = (dz+1)*9 + (dy+1)*3 + (dx+1), the
    input read at voxel + (dz, dy, dx) (arrays indexed [z][y][x]): a unit
    weight at one tap moves a point input to the voxel that reads it."""
    torch = pytest.importorskip("torch")
    import torch.nn.functional as Fn
    from oracle import unet_ref as R
    n = 6
    for (dz, dy, dx) in ((0, 0, 1), (1, 0, 0), (0, -1, 0), (-1, 1, -1)):
        tap = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)
        p = np.zeros(R.param_count())
        p[tap * 3 * 16 + 1 * 16 + 5] = 1.0          # conv 0: tap, cin 1 -> cout 5
        (w, b), = R.unpack(p)[0][:1]
        x = torch.zeros(1, 3, n, n, n, dtype=torch.float64)
        x[0, 1, 3, 3, 3] = 1.0                      # point input at (z, y, x) = (3, 3, 3), channel 1
        y = Fn.conv3d(x, w, b, padding=1)
        nz = torch.nonzero(y)
        assert nz.shape[0] == 1
        assert tuple(nz[0].tolist()) == (0, 5, 3 - dz, 3 - dy, 3 - dx)


def _routing_params(skip_channel):
    """Every convolution passes one input channel through its centre tap to
    output channel 0 (zero biases, unit 1x1 output on channel 0): the input
    channel of the decoder convolutions picks the upsampled path (0) or the
    skip path (skip_channel)."""
    from oracle import unet_ref as R
    p = np.zeros(R.param_count())
    off = 0
    for i, (cin, cout) in enumerate(R.CONV_DIMS):
        ci = skip_channel(i) if i >= 6 else 0
        p[off + 13 * cin * cout + ci * cout + 0] = 1.0
        off += 27 * cin * cout + cout
    p[off + 0] = 1.0                                 # 1x1 output weight of channel 0
    return p


def test_reference_wiring_by_hand():
    """Through the whole network with pass-through weights: taking channel 0
    of every decoder input (the upsampled coarse path) gives each voxel the
    mean of its 8x8x8 block (three 2x pools, three nearest 2x upsamplings);
    taking the skip channels instead gives the input itself at every scale."""
    torch = pytest.importorskip("torch")
    from oracle import unet_ref as R
    n = 16
    rng = np.random.default_rng(21)
    rho = torch.from_numpy(rng.uniform(0.5, 1.5, size=(1, n, n, n)))
    phi = torch.from_numpy(rng.uniform(-1, 1, size=(1, n, n, n)))
    res = torch.from_numpy(rng.uniform(-1, 1, size=(1, n, n, n)))
    x0 = rho / phi.abs().max()                        # channel 0 as the network sees it (frho = 1)
    # decoder inputs: [up(low) (Cu channels), skip]: Cu = 64, 32, 16 for convs 6, 7, 8
    y_up, _ = R.forward(torch.from_numpy(_routing_params(lambda i: 0)), rho, phi, res, [1.0])
    blk = x0[0].reshape(2, 8, 2, 8, 2, 8).mean(dim=(1, 3, 5))
    want = blk.repeat_interleave(8, 0).repeat_interleave(8, 1).repeat_interleave(8, 2)
    assert torch.allclose(y_up[0], want, rtol=0, atol=1e-14)
    # conv 8 from the first skip channel (index 16): s0, the input at full resolution
    y_skip, _ = R.forward(torch.from_numpy(_routing_params(lambda i: {6: 64, 7: 32, 8: 16}[i])), rho, phi, res, [1.0])
    assert torch.allclose(y_skip[0], x0[0], rtol=0, atol=1e-14)


def _dyadic_case(seed, n=8, B=1):
    """Inputs and parameters on coarse dyadic grids (integers, eighths) whose
    every sum the module forms is exact in FP32: max |phi| = max |resid| = 8
    (power-of-two scales), frho = 1, targets (phi_true - phi)/(8 n^2/16)
    integer; sparse integer weights and biases."""
    from oracle import unet_ref as R
    rng = np.random.default_rng(I.BASE_SEED + 700 + seed)
    sh = (B, n, n, n)
    rho = rng.integers(-4, 5, size=sh).astype(np.float64)
    phi = rng.integers(-7, 8, size=sh).astype(np.float64)
    phi[:, 0, 0, 0] = 8.0
    res = rng.integers(-7, 8, size=sh).astype(np.float64)
    res[:, 1, 2, 3] = -8.0
    scale = 8.0 * n * n / 16.0
    tru = phi + scale * rng.integers(-2, 3, size=sh)
    frho = np.ones(B)
    p = np.zeros(R.param_count(), dtype=np.float32)
    off = 0
    for cin, cout in R.CONV_DIMS:
        nw = 27 * cin * cout
        d = min(0.5, 2.5 / (27 * cin))
        p[off:off + nw] = rng.choice([-1.0, 0.0, 1.0], size=nw, p=[d / 2, 1 - d, d / 2])
        p[off + nw:off + nw + cout] = rng.choice([0.0, 1.0], size=cout)
        off += nw + cout
    p[off:off + 16] = rng.choice([-1.0, 1.0], size=16)
    return rho, phi, res, tru, frho, p


def test_dyadic_case_is_exact_in_fp32():
    """The emulated forward pass of the dyadic case gives the same values in
    float32 as in float64: every sum it forms is exact, so any order of
    summation (the module's FP32 tensor-core accumulation) gives them too."""
    torch = pytest.importorskip("torch")
    from oracle import unet_ref as R
    rho, phi, res, tru, frho, p = _dyadic_case(0)
    T = torch.from_numpy
    y64, _ = R.forward(T(p.astype(np.float64)), T(rho), T(phi), T(res), frho, emulate=True)
    y32, _ = R.forward(T(p), T(rho).float(), T(phi).float(), T(res).float(), frho, emulate=True)
    assert torch.equal(y64.float(), y32)
    assert (y64 != 0).float().mean() > 0.2          # the case exercises the network, not a zero output


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


@pytest.mark.gpu
def test_forward_and_gradient_elementwise_dyadic(un):
    """Element-wise parity on the dyadic case: the forward output equals the
    BF16-emulating float64 reference bit for bit (every sum exact, so only a
    wrong tap, layout, rounding point or wiring could differ); every weight
    and bias gradient lies within the FP32 summation bound of its terms,
    |g - g_ref| <= V 2^-24 sum |terms| (V = voxels summed), and the loss
    within the same bound."""
    import torch
    from oracle import unet_ref as R
    B, n = 1, 8
    rho, phi, res, tru, frho, p = _dyadic_case(0, n, B)
    u = un.mg_unet_create(n, B, seed=0)
    try:
        un.mg_unet_set_params(u, p)
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        y = un.mg_unet_forward(u, B, n, dev(rho), dev(phi), dev(res), frho)
        T = torch.from_numpy
        p64 = p.astype(np.float64)
        yr, _ = R.forward(T(p64), T(rho), T(phi), T(res), frho, emulate=True)
        yr = yr.detach().numpy().astype(np.float32)
        assert np.array_equal(np.asarray(y).reshape(yr.shape), yr), np.abs(np.asarray(y).reshape(yr.shape) - yr).max()
        loss = un.mg_unet_train_step(u, B, n, dev(rho), dev(phi), dev(res), dev(tru), frho, update=False)
        g = un.mg_unet_get_grad(u).astype(np.float64)
        lr, gr = R.loss_and_grad(p64, T(rho), T(phi), T(res), T(tru), frho, emulate=True)
        mag = R.weight_grad_magnitude(p64, T(rho), T(phi), T(res), T(tru), frho)
        V = B * n ** 3
        bound = V * 2.0 ** -24 * mag
        bad = np.abs(g - gr) > bound
        assert not bad.any(), (int(bad.sum()), np.flatnonzero(bad)[:10], (np.abs(g - gr) / np.maximum(mag, 1e-300)).max())
        assert (gr != 0).mean() > 0.01                 # gradients reach the parameters
        assert abs(loss - lr) <= V * 2.0 ** -24 * lr + 1e-30
    finally:
        un.mg_unet_destroy(u)


@pytest.mark.gpu
def test_learned_guess_gain_measured(un, capsys):
    """What the trained network gains: trained on solver-generated samples
    (32 samples from 16 hierarchies of three 32^3 levels with 1-8 random
    spheres), then held-out hierarchies solved to 1e-10 in mixed precision
    from the zero, the interpolated (Sec. 2.4) and the learned initial guess.
    Asserted: every form converges to the same solution, and the learned
    guess needs fewer V-cycles than the zero guess; printed: V-cycles and wall
    time of all three (the measured comparison with the interpolated guess)."""
    import torch
    from paper_2001_02327_gb300 import learned as LR
    data = LR.make_samples(torch, 32, n=32, seed0=I.BASE_SEED + 6000, levels=3)
    net = un.mg_unet_create(32, 4, seed=3)
    try:
        losses = LR.train(torch, net, data, steps=300, batch=4, lr=1e-3)
        assert np.mean(losses[-30:]) < 0.5 * np.mean(losses[:30])
        held = [LR.random_nested(I.BASE_SEED + 9000 + k, 32, 3) for k in range(3)]
        ev = LR.evaluate(torch, net, held, reps=3)
    finally:
        un.mg_unet_destroy(net)
    with capsys.disabled():
        print("\nlearned-guess evaluation (3 held-out hierarchies of 3 x 32^3, mixed, to 1e-10): " +
              ", ".join(f"{k}: {v['cycles']} V-cycles, {v['ms']:.2f} ms" for k, v in ev.items()))
    for k in ("interp", "learned"):
        assert ev[k]["max_rel_diff_vs_zero_guess"] < 1e-8, (k, ev[k])
    assert ev["learned"]["cycles"] < ev["zero"]["cycles"], ev


@pytest.mark.gpu
@pytest.mark.parametrize("persistent", ["0", "1"])
def test_tensor_core_wait_timeout_reports_code_4(persistent):
    """A convolution whose accumulator never completes (UNET_FAULT_WAIT=1:
    the issuing thread issues no MMA and no commit, so nothing is in flight)
    gives up after its clock budget, frees its tensor memory, and the call
    returns 4 instead of hanging -- with the one-tile-per-block halo kernel
    and with the persistent one (UNET_HALO_P=1), which also waits for the
    halo copies it has in flight before it leaves; the flags are read once
    per process, so the check runs in a child process."""
    import os
    import subprocess
    import sys
    import textwrap
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = textwrap.dedent("""
        import sys
        import numpy as np, torch
        sys.path.insert(0, %r)
        from paper_2001_02327_gb300 import unet as U
        u = U.mg_unet_create(16, 1, seed=1)
        x = torch.zeros((1, 16, 16, 16), dtype=torch.float64, device="cuda")
        try:
            U.mg_unet_forward(u, 1, 16, x, x, x, np.ones(1))
            print("NO ERROR")
        except U.UNetError as e:
            print("ERROR", e)
    """ % root)
    env = dict(os.environ, UNET_FAULT_WAIT="1", UNET_HALO_P=persistent)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600, cwd=root)
    assert "failed with code 4" in r.stdout, (r.stdout, r.stderr[-2000:])


@pytest.mark.gpu
def test_persistent_halo_kernel_equals_per_tile_kernel(tmp_path):
    """The persistent halo convolution (weights loaded once per block, two
    halo buffers and two accumulators, several tiles per block at 64^3) and
    the one-tile-per-block kernel issue the same products in the same order:
    the forward output is equal bit for bit, the loss and the gradients up to
    the order of their atomic FP32 sums.  The kernel choice is read once per
    process, so each form runs in a child process."""
    import os
    import subprocess
    import sys
    import textwrap
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = textwrap.dedent("""
        import sys
        import numpy as np, torch
        sys.path.insert(0, %r)
        from paper_2001_02327_gb300 import unet as U
        n, B = 64, 1
        rng = np.random.default_rng(2024)
        a = [rng.standard_normal((B, n, n, n)) for _ in range(4)]
        dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
        u = U.mg_unet_create(n, B, seed=9)
        try:
            y = U.mg_unet_forward(u, B, n, dev(a[0]), dev(a[1]), dev(a[2]), np.full(B, 0.3))
            loss = U.mg_unet_train_step(u, B, n, dev(a[0]), dev(a[1]), dev(a[2]), dev(a[3]), np.full(B, 0.3),
                                        update=False)
            g = U.mg_unet_get_grad(u)
        finally:
            U.mg_unet_destroy(u)
        np.savez(sys.argv[1], y=np.asarray(y), g=np.asarray(g), loss=np.asarray(loss))
    """ % root)
    out = {}
    for mode in ("0", "1"):
        env = dict(os.environ, UNET_HALO_P=mode)
        f = str(tmp_path / f"p{mode}.npz")
        r = subprocess.run([sys.executable, "-c", code, f], env=env, capture_output=True, text=True, timeout=600,
                           cwd=root)
        assert r.returncode == 0, r.stderr[-2000:]
        out[mode] = np.load(f)
    assert np.array_equal(out["0"]["y"], out["1"]["y"])
    assert abs(float(out["1"]["loss"]) / float(out["0"]["loss"]) - 1) < 1e-6
    g0, g1 = out["0"]["g"].astype(np.float64), out["1"]["g"].astype(np.float64)
    assert _rel(g1, g0) < 1e-5, _rel(g1, g0)
    assert np.isfinite(out["1"]["y"]).all() and np.abs(g1).max() > 0
