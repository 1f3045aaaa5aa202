"""Training data, training and evaluation of the learned initial guess.

Data come from the solver itself: for random nested hierarchies (each
refinement level an n^3 patch, 1-8 compact spheres in the finest box) the
plain FP64 method solves every level to 1e-10; for each level above the base
a sample is (density on Omega, the potential interpolated from the parent --
the initial guess the method would start from -- and the converged
potential).  The network learns the correction (solution - interpolated
guess) / s.  All arithmetic runs in libmg.so; this module only drives it.
"""
from __future__ import annotations

import time
from math import pi

import numpy as np

from . import inputs as I
from . import mg
from . import unet as U


def random_nested(seed, n=64, levels=3, max_spheres=8):
    rng = np.random.default_rng(seed)
    w = 2.0 ** (-(levels - 1))
    k = int(rng.integers(1, max_spheres + 1))
    sph = I.random_spheres(rng, k, -w, w)
    return I.nested_centred(3, levels, n, 1.0, 1.0, sph, f"train_s{seed}")


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def solve(H, torch, opt, unet=None, phi_out=False):
    """Solve a hierarchy; returns (stats per level, list of Omega potentials)."""
    h = mg.mg_create_hierarchy([mg.desc_from(H)], opt)
    try:
        if unet is not None:
            U.mg_set_unet(h, unet)
        inp = I.level_inputs(H)
        mg.mg_set_density(h, 0, 0, _dev(torch, inp[0]["rho"]), _dev(torch, inp[0]["bc_rho"]),
                          _dev(torch, inp[0]["bc_phi"]))
        for l in range(1, H.num_levels):
            mg.mg_set_density(h, 0, l, _dev(torch, inp[l]["rho"]))
        _, st = mg.mg_solve(h, 1, allow_noconv=True)
        phis = []
        if phi_out:
            for l in range(H.num_levels):
                p = torch.zeros((H.n[l],) * 3, dtype=torch.float64, device="cuda")
                mg.mg_forces(h, 0, l, p, None)
                phis.append(p)
        return st[0][:H.num_levels], phis, (h if phi_out else None)
    finally:
        if not phi_out:
            mg.mg_destroy(h)


def make_samples(torch, count, n=64, seed0=0, levels=3):
    """Generate `count` samples on the GPU from solver runs; returns dict of
    device tensors rho, phi_i, res (the h^2-scaled residual of phi_i), phi_t
    (count, n, n, n) and frho (count,)."""
    rho, pi_, rs, pt, fr = [], [], [], [], []
    opt = mg.options(nu_pre=2, nu_post=2, max_cycles=60, rel_tol=1e-10)
    s = seed0
    while len(rho) < count:
        H = random_nested(s, n, levels)
        s += 1
        st, phis, h = solve(H, torch, opt, phi_out=True)
        try:
            inp = I.level_inputs(H)
            for l in range(1, H.num_levels):
                g = torch.zeros((n,) * 3, dtype=torch.float64, device="cuda")
                r = torch.zeros_like(g)
                U.mg_interp_guess(h, 0, l, g, r)
                rho.append(_dev(torch, inp[l]["rho"]))
                pi_.append(g)
                rs.append(r)
                pt.append(phis[l])
                fr.append(4 * pi * H.G * H.h(l) ** 2)
        finally:
            mg.mg_destroy(h)
    torch.cuda.synchronize()
    return {"rho": torch.stack(rho[:count]), "phi_i": torch.stack(pi_[:count]), "res": torch.stack(rs[:count]),
            "phi_t": torch.stack(pt[:count]), "frho": np.array(fr[:count])}


def train(torch, net, data, steps, batch=4, lr=1e-3, wd=1e-5, seed=0, log_every=0):
    n = data["rho"].shape[1]
    N = data["rho"].shape[0]
    rng = np.random.default_rng(seed)
    losses = []
    for it in range(steps):
        idx = rng.choice(N, size=batch, replace=False)
        ti = torch.from_numpy(idx).cuda()
        r = data["rho"].index_select(0, ti).contiguous()
        pi_ = data["phi_i"].index_select(0, ti).contiguous()
        rs = data["res"].index_select(0, ti).contiguous()
        pt = data["phi_t"].index_select(0, ti).contiguous()
        cur_lr = lr * 0.5 * (1 + np.cos(np.pi * it / steps))        # cosine schedule
        losses.append(U.mg_unet_train_step(net, batch, n, r, pi_, rs, pt, data["frho"][idx], lr=cur_lr, wd=wd))
        if log_every and it % log_every == 0:
            print(f"step {it} loss {losses[-1]:.4e}", flush=True)
    return losses


def validation_loss(torch, net, data, batch=4):
    n = data["rho"].shape[1]
    N = data["rho"].shape[0]
    tot, k = 0.0, 0
    for s in range(0, N - batch + 1, batch):
        sl = slice(s, s + batch)
        tot += U.mg_unet_train_step(net, batch, n, data["rho"][sl].contiguous(), data["phi_i"][sl].contiguous(),
                                    data["res"][sl].contiguous(), data["phi_t"][sl].contiguous(), data["frho"][sl],
                                    update=False)
        k += 1
    return tot / max(k, 1)


def evaluate(torch, net, hierarchies, precision=mg.MG_MIXED, reps=3):
    """Per guess mode: total cycles, wall ms (median of reps) and worst error
    against the FP64 zero-guess solution."""
    out = {}
    ref = {}
    for mode, name in ((mg.MG_GUESS_ZERO, "zero"), (mg.MG_GUESS_INTERP, "interp"), (mg.MG_GUESS_LEARNED, "learned")):
        cyc, times, err = 0, [], 0.0
        for H in hierarchies:
            opt = mg.options(nu_pre=2, nu_post=2, max_cycles=80, rel_tol=1e-10, precision=precision, guess=mode)
            h = mg.mg_create_hierarchy([mg.desc_from(H)], opt)
            try:
                if mode == mg.MG_GUESS_LEARNED:
                    U.mg_set_unet(h, net)
                inp = I.level_inputs(H)
                d = [{k: _dev(torch, v) for k, v in x.items()} for x in inp]
                ts = []
                for r in range(reps + 1):
                    mg.mg_set_density(h, 0, 0, d[0]["rho"], d[0]["bc_rho"], d[0]["bc_phi"])
                    for l in range(1, H.num_levels):
                        mg.mg_set_density(h, 0, l, d[l]["rho"])
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    _, st = mg.mg_solve(h, 1)
                    torch.cuda.synchronize()
                    if r:
                        ts.append(time.perf_counter() - t0)
                times.append(float(np.median(ts)))
                cyc += sum(st[0][l]["cycles"] for l in range(H.num_levels))
                for l in range(H.num_levels):
                    p = torch.zeros((H.n[l],) * 3, dtype=torch.float64, device="cuda")
                    mg.mg_forces(h, 0, l, p, None)
                    key = (H.name, l)
                    if mode == mg.MG_GUESS_ZERO:
                        ref[key] = p.clone()
                    else:
                        err = max(err, float((p - ref[key]).abs().max() / ref[key].abs().max()))
            finally:
                mg.mg_destroy(h)
        out[name] = {"cycles": cyc, "ms": 1e3 * float(np.sum(times)), "max_rel_diff_vs_zero_guess": err}
    return out
