"""CPU reference of the learned-guess network (TEST INFRASTRUCTURE ONLY).

The same 4-scale 3D U-Net as the CUDA module, written with plain PyTorch CPU
operations in float64 and the same flat parameter layout: for each of the
nine 3x3x3 convolutions, weights [27][Cin][Cout] (tap = (dz+1)*9 + (dy+1)*3 +
(dx+1), the input read at voxel + (dz, dy, dx)) followed by [Cout] biases;
then the 1x1 output's 16 weights and bias.  Gradients come from autograd.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as Fn

CONV_DIMS = [(2, 16), (16, 16), (16, 32), (32, 32), (32, 64), (64, 64), (128, 32), (64, 16), (32, 16)]


def param_count():
    return sum(27 * a * b + b for a, b in CONV_DIMS) + 17


def unpack(p):
    """Flat parameter vector -> list of (weight[Cout,Cin,3,3,3], bias) and the output layer."""
    p = torch.as_tensor(p)
    out, off = [], 0
    for cin, cout in CONV_DIMS:
        w = p[off:off + 27 * cin * cout].reshape(27, cin, cout)
        off += 27 * cin * cout
        b = p[off:off + cout]
        off += cout
        # tap t = (dz+1)*9 + (dy+1)*3 + (dx+1) -> kernel index [kz][ky][kx]
        wt = w.permute(2, 1, 0).reshape(cout, cin, 3, 3, 3)
        out.append((wt, b))
    wo = p[off:off + 16]
    bo = p[off + 16:off + 17]
    return out, (wo, bo)


def forward(p, rho, phi_interp, frho):
    """rho, phi_interp: (B, n, n, n) float64 tensors; frho: (B,) factors.
    Returns (y (B,n,n,n), scale (B,))."""
    convs, (wo, bo) = unpack(p)
    B = rho.shape[0]
    s = torch.clamp(phi_interp.abs().reshape(B, -1).max(dim=1).values, min=0.0)
    s = torch.where(s > 0, s, torch.ones_like(s))
    sv = s.reshape(B, 1, 1, 1)
    fr = torch.as_tensor(frho, dtype=rho.dtype).reshape(B, 1, 1, 1)
    x = torch.stack([fr * rho / sv, phi_interp / sv], dim=1)            # (B, 2, n, n, n)

    def c3(t, i):
        return torch.relu(Fn.conv3d(t, convs[i][0], convs[i][1], padding=1))

    a0 = c3(x, 0)
    s0 = c3(a0, 1)
    a1 = c3(Fn.avg_pool3d(s0, 2), 2)
    s1 = c3(a1, 3)
    s2 = c3(Fn.avg_pool3d(s1, 2), 4)
    a3 = c3(Fn.avg_pool3d(s2, 2), 5)
    up = lambda t: Fn.interpolate(t, scale_factor=2, mode="nearest")
    d2 = c3(torch.cat([up(a3), s2], dim=1), 6)
    d1 = c3(torch.cat([up(d2), s1], dim=1), 7)
    d0 = c3(torch.cat([up(d1), s0], dim=1), 8)
    y = torch.einsum("bcxyz,c->bxyz", d0, wo) + bo
    return y, s


def loss_and_grad(p, rho, phi_interp, phi_true, frho):
    """Loss mean((y - (phi_true - phi_interp)/s)^2) and its gradient (float64)."""
    pt = torch.tensor(np.asarray(p, dtype=np.float64), requires_grad=True)
    y, s = forward(pt, rho, phi_interp, frho)
    tgt = (phi_true - phi_interp) / s.reshape(-1, 1, 1, 1)
    loss = ((y - tgt) ** 2).mean()
    loss.backward()
    return float(loss.detach()), pt.grad.numpy()
