"""CPU reference of the learned-guess network (TEST INFRASTRUCTURE ONLY).

The same 4-scale 3D U-Net as the CUDA module, written with plain PyTorch CPU
operations in float64 and the same flat parameter layout: for each of the
nine 3x3x3 convolutions, weights [27][Cin][Cout] (tap = (dz+1)*9 + (dy+1)*3 +
(dx+1), the input read at voxel + (dz, dy, dx)) followed by [Cout] biases;
then the 1x1 output's 16 weights and bias.  Gradients come from autograd.

emulate=True rounds to BF16 where the CUDA module stores BF16: the network
inputs, the convolution weights, every convolution's output (after bias and
ReLU) and every pooled mean; and, in the backward pass, the gradient that
enters each convolution's data-gradient and weight-gradient products (the
tensor-core products of the module take BF16 operands; its bias gradient
sums the unrounded gradient).  Everything else stays float64.  With data whose
every sum is exact in FP32 (dyadic values of few bits) the forward pass then
equals the CUDA module's bit for bit.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as Fn

CONV_DIMS = [(3, 16), (16, 16), (16, 32), (32, 32), (32, 64), (64, 64), (128, 32), (64, 16), (32, 16)]


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


def bf16(t):
    """Round float64 values to BF16 (nearest, ties to even) and back."""
    return t.to(torch.float32).to(torch.bfloat16).to(t.dtype)


class _RoundST(torch.autograd.Function):
    """BF16 rounding with an identity gradient (the module rounds stored
    activations but passes gradients through unchanged)."""

    @staticmethod
    def forward(ctx, x):
        return bf16(x)

    @staticmethod
    def backward(ctx, g):
        return g


class _ConvBF16(torch.autograd.Function):
    """3x3x3 convolution (padding 1) + bias as the module computes it: the
    data gradient multiplies the BF16-rounded output gradient by the BF16
    weights, the weight gradient the BF16 input by the BF16-rounded output
    gradient; the bias gradient sums the unrounded gradient."""

    @staticmethod
    def forward(ctx, x, w, b):
        ctx.save_for_backward(x, w)
        return Fn.conv3d(x, w, b, padding=1)

    @staticmethod
    def backward(ctx, g):
        x, w = ctx.saved_tensors
        gx = torch.nn.grad.conv3d_input(x.shape, w, bf16(g), padding=1)
        gw = torch.nn.grad.conv3d_weight(x, w.shape, bf16(g), padding=1)
        return gx, gw, g.sum(dim=(0, 2, 3, 4))


def _max_abs(t):
    B = t.shape[0]
    s = t.abs().reshape(B, -1).max(dim=1).values
    return torch.where(s > 0, s, torch.ones_like(s))


def forward(p, rho, phi_interp, resid, frho, emulate=False, absgrad=False):
    """rho, phi_interp, resid: (B, n, n, n) float64 tensors (resid = the
    h^2-scaled residual of phi_interp); frho: (B,) factors 4 pi G h^2.
    Returns (y (B,n,n,n), output scale (B,)): the correction is scale * y with
    scale = max|resid| n^2 / 16.  absgrad (with emulate): weight and bias
    gradients sum absolute values (weight_grad_magnitude)."""
    convs, (wo, bo) = unpack(p)
    B, n = rho.shape[0], rho.shape[1]
    if emulate:
        # scales and inputs as the module forms them: FP32 maxima and quotients
        f32 = lambda t: t.to(torch.float32).to(t.dtype)
        s = _max_abs(f32(phi_interp))
        sr = _max_abs(f32(resid))
    else:
        s = _max_abs(phi_interp)
        sr = _max_abs(resid)
    sv, srv = s.reshape(B, 1, 1, 1), sr.reshape(B, 1, 1, 1)
    fr = torch.as_tensor(frho, dtype=rho.dtype).reshape(B, 1, 1, 1)
    x = torch.stack([fr * rho / sv, phi_interp / sv, resid / srv], dim=1)   # (B, 3, n, n, n)
    rnd = _RoundST.apply if emulate else (lambda t: t)
    x = rnd(x)

    def c3(t, i):
        w, b = convs[i]
        if emulate:
            conv = _ConvBF16Abs if absgrad else _ConvBF16
            return rnd(torch.relu(conv.apply(t, _RoundST.apply(w), b)))
        return torch.relu(Fn.conv3d(t, w, b, padding=1))

    pool = lambda t: rnd(Fn.avg_pool3d(t, 2))
    a0 = c3(x, 0)
    s0 = c3(a0, 1)
    a1 = c3(pool(s0), 2)
    s1 = c3(a1, 3)
    s2 = c3(pool(s1), 4)
    a3 = c3(pool(s2), 5)
    up = lambda t: Fn.interpolate(t, scale_factor=2, mode="nearest")
    d2 = c3(torch.cat([up(a3), s2], dim=1), 6)
    d1 = c3(torch.cat([up(d2), s1], dim=1), 7)
    d0 = c3(torch.cat([up(d1), s0], dim=1), 8)
    if absgrad:
        y = _OutAbs.apply(d0, wo, bo)
    else:
        y = torch.einsum("bcxyz,c->bxyz", d0, wo) + bo
    return y, sr * (n * n / 16.0)


def residual_h2(phi, rho, frho):
    """h^2 (4 pi G rho - lap_h phi) on the interior of dense (B, n, n, n)
    arrays (the 7-point Laplacian of Eq. 4; edge cells are left zero)."""
    fr = torch.as_tensor(frho, dtype=rho.dtype).reshape(-1, 1, 1, 1)
    r = torch.zeros_like(phi)
    c = phi[:, 1:-1, 1:-1, 1:-1]
    nb = (phi[:, :-2, 1:-1, 1:-1] + phi[:, 2:, 1:-1, 1:-1] + phi[:, 1:-1, :-2, 1:-1] + phi[:, 1:-1, 2:, 1:-1]
          + phi[:, 1:-1, 1:-1, :-2] + phi[:, 1:-1, 1:-1, 2:])
    r[:, 1:-1, 1:-1, 1:-1] = fr * rho[:, 1:-1, 1:-1, 1:-1] - (nb - 6.0 * c)
    return r


def loss_and_grad(p, rho, phi_interp, resid, phi_true, frho, emulate=False):
    """Loss mean((y - (phi_true - phi_interp)/scale)^2) and its gradient (float64)."""
    pt = torch.tensor(np.asarray(p, dtype=np.float64), requires_grad=True)
    y, s = forward(pt, rho, phi_interp, resid, frho, emulate)
    tgt = (phi_true - phi_interp) / s.reshape(-1, 1, 1, 1)
    loss = ((y - tgt) ** 2).mean()
    loss.backward()
    return float(loss.detach()), pt.grad.numpy()


class _ConvBF16Abs(_ConvBF16):
    """As _ConvBF16, but the weight and bias gradients sum the absolute
    values of their terms (the data gradient stays signed)."""

    @staticmethod
    def backward(ctx, g):
        x, w = ctx.saved_tensors
        gx = torch.nn.grad.conv3d_input(x.shape, w, bf16(g), padding=1)
        gw = torch.nn.grad.conv3d_weight(x.abs(), w.shape, bf16(g).abs(), padding=1)
        return gx, gw, g.abs().sum(dim=(0, 2, 3, 4))


class _OutAbs(torch.autograd.Function):
    """The 1x1 output layer with absolute-value weight and bias gradients."""

    @staticmethod
    def forward(ctx, d0, wo, bo):
        ctx.save_for_backward(d0, wo)
        return torch.einsum("bcxyz,c->bxyz", d0, wo) + bo

    @staticmethod
    def backward(ctx, g):
        d0, wo = ctx.saved_tensors
        gd0 = torch.einsum("bxyz,c->bcxyz", g, wo)
        gw = torch.einsum("bxyz,bcxyz->c", g.abs(), d0.abs())
        return gd0, gw, g.abs().sum().reshape(1)


def weight_grad_magnitude(p, rho, phi_interp, resid, phi_true, frho):
    """Per weight and bias, the sum over voxels of the absolute values of the
    terms its gradient adds up (|input| x |output gradient|), in the emulated
    pass: the scale of the rounding error of any order of that summation."""
    pt = torch.tensor(np.asarray(p, dtype=np.float64), requires_grad=True)
    y, s = forward(pt, rho, phi_interp, resid, frho, emulate=True, absgrad=True)
    tgt = (phi_true - phi_interp) / s.reshape(-1, 1, 1, 1)
    loss = ((y - tgt) ** 2).mean()
    loss.backward()
    return pt.grad.numpy()
