"""torch.autograd.Function over the C ABI for training the sparse coefficient field.

``RenderL1.apply`` returns Loss = mean |W S - target| for one camera, where W is the sparse
coefficient map rendered from the Gaussians (Sec. 3.4) and S the codebook (Eq. 7).  Its
forward calls lsv2_project / lsv2_bin_sort / lsv2_splat_coeffs and the fused decode + L1
kernel, which also produces dLoss/dW and dLoss/dS in the same pass (F is never stored).
Its backward calls lsv2_splat_backward (transmittance recomputed from the final T) for the
gradients of the coefficient weights, opacities, means, scales and quaternions.

Inputs are activated values (scales > 0, opacity in (0, 1)); apply exp / sigmoid in torch
before calling it and autograd chains those derivatives.

``Sparsify.apply`` (or ``sparsify``) turns the per-Gaussian L-dim parameters into the K
(index, weight) pairs of Sec. 3.3 (softmax, top K, renormalised) through lsv2_sparsify, and its
backward calls lsv2_sparsify_backward, so logits -> sparsify -> render_l1 trains end to end.
"""
from __future__ import annotations

import torch

from . import _lib as L
from .pipeline import DeviceScene, Frame, _ptr, _stream


class RenderL1(torch.autograd.Function):
    @staticmethod
    def forward(ctx, means, scales, quats, opacity, weights, codebook, idx, cam, target, capacity=None):
        scene = DeviceScene(means.detach().contiguous(), scales.detach().contiguous(), quats.detach().contiguous(),
                            opacity.detach().contiguous(), idx.contiguous(), weights.detach().contiguous(),
                            codebook.detach().contiguous())
        frame = Frame(scene, cam, capacity=capacity, device=means.device)
        frame.render()
        P, lev, D = frame.P, scene.levels, scene.D
        loss = torch.zeros(1, dtype=torch.float32, device=means.device)
        dcoeff = torch.empty_like(frame.coeff)
        dcodebook = torch.zeros_like(scene.codebook)
        L.lsv2_l1_decode_backward(lev, P, 64, D, _ptr(frame.coeff), _ptr(scene.codebook), _ptr(target.contiguous()),
                                  _ptr(loss), _ptr(dcoeff), _ptr(dcodebook), _ptr(frame.status), _stream(None))
        frame.check()
        ctx.frame, ctx.dcoeff, ctx.dcodebook = frame, dcoeff, dcodebook
        return loss[0]

    @staticmethod
    def backward(ctx, gloss):
        frame: Frame = ctx.frame
        s = frame.scene
        n = s.n
        dev = s.means.device
        dw = torch.zeros_like(s.weights)
        dop = torch.zeros(n, dtype=torch.float32, device=dev)
        dm = torch.zeros_like(s.means)
        ds = torch.zeros_like(s.scales)
        dq = torch.zeros_like(s.quats)
        ws_bytes = L.lsv2_splat_backward_workspace_bytes(n)
        ws = torch.empty(max(ws_bytes, 16), dtype=torch.uint8, device=dev)
        L.lsv2_splat_backward(frame.ccam, n, _ptr(s.means), _ptr(s.scales), _ptr(s.quats), frame.proj,
                              _ptr(frame.tile_ranges), _ptr(frame.gauss_ids), s.levels, s.K, 64, _ptr(s.idx),
                              _ptr(s.weights), _ptr(frame.final_T), _ptr(frame.n_last), _ptr(ctx.dcoeff), _ptr(ws),
                              ws_bytes, _ptr(dw), _ptr(dop), _ptr(dm), _ptr(ds), _ptr(dq), _ptr(frame.status),
                              _stream(None))
        g = gloss
        return dm * g, ds * g, dq * g, dop * g, dw * g, ctx.dcodebook * g, None, None, None, None


def render_l1(means, log_scales, quats, opacity_logits, weights, codebook, idx, cam, target, capacity=None):
    """Loss = mean |W S - target| with the activations applied here (exp, sigmoid)."""
    return RenderL1.apply(means, torch.exp(log_scales), quats, torch.sigmoid(opacity_logits), weights, codebook,
                          idx, cam, target, capacity)


class Sparsify(torch.autograd.Function):
    """logits [..., L] -> (weights [..., K] float32, differentiable; idx [..., K] uint8)."""

    @staticmethod
    def forward(ctx, logits, K):
        z = logits.detach().contiguous().float()
        Lz = z.shape[-1]
        rows = z.numel() // Lz
        idx = torch.empty(z.shape[:-1] + (K,), dtype=torch.uint8, device=z.device)
        w = torch.empty(z.shape[:-1] + (K,), dtype=torch.float32, device=z.device)
        L.lsv2_sparsify(rows, Lz, K, _ptr(z), _ptr(idx), _ptr(w), _stream(None))
        ctx.save_for_backward(idx, w)
        ctx.Lz, ctx.K = Lz, K
        ctx.mark_non_differentiable(idx)
        return w, idx

    @staticmethod
    def backward(ctx, gw, gidx):
        idx, w = ctx.saved_tensors
        dz = torch.empty(w.shape[:-1] + (ctx.Lz,), dtype=torch.float32, device=w.device)
        L.lsv2_sparsify_backward(w.numel() // ctx.K, ctx.Lz, ctx.K, _ptr(idx), _ptr(w), _ptr(gw.contiguous().float()),
                                 _ptr(dz), _stream(None))
        return dz, None


def sparsify(logits, K: int):
    """Sec. 3.3 sparse coefficients of logits [..., L]: (weights [..., K], idx [..., K] uint8)."""
    return Sparsify.apply(logits, K)
