"""The decoder-based comparison path (LangSplat*, Sec. 3.1 and Table 1) on the same library.

LangSplat renders a d = 3 latent feature per pixel and level (Eq. 4: the same front-to-back
blend as Eq. 3, with a d-dim feature per Gaussian) and decodes it to the 512-d CLIP space with
an MLP g_d.  Table 1 times the decode as LangSplat*'s dominant stage; LangSplatV2 replaces it by
the linear decode of Eq. 7.  Here:

* the latent render is ``lsv2_splat_coeffs`` with L = 8 output channels and K = 4 pairs per
  level: pair k < 3 carries (index k, weight f_k), the fourth pair (index 3, weight 0) pads K,
  so the splat accumulates exactly sum_i f_i alpha_i T_i into channels 0..2 and channels 3..7
  stay zero;
* the decode is ``lsv2_mlp_decode`` over all levels' pixels as rows, the latent's 3 channels
  padded to 8 (zero columns in x, zero rows in the first weight matrix): by default one library
  GEMM per layer over row blocks, or, with ``block_rows=L.LSV2_MLP_FUSED``, the fused tensor-core
  kernel (every layer on tcgen05, the hidden activations kept on chip, a workspace of < 2 MB).

PyTorch holds the buffers; every step runs in the CUDA library.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as L
from .pipeline import DeviceScene, Frame, _ptr, _stream

LATENT_CHANNELS = 8   # the splat's and the MLP's input width: 3 latent channels + 5 zero channels
PAIRS = 4


def latent_pairs(latent: torch.Tensor) -> tuple[torch.Tensor, torch.Tensor]:
    """(index, weight) pairs that make the sparse splat blend a d-dim latent feature (d <= 4):
    latent f32 [n, levels, d] -> idx u8 [n, levels, 4] = (0, 1, 2, 3), w f32 [n, levels, 4] =
    (f_0, .., f_{d-1}, 0, ..)."""
    n, levels, d = latent.shape
    if d > PAIRS:
        raise ValueError(f"a latent of {d} channels needs more than {PAIRS} pairs")
    idx = torch.arange(PAIRS, dtype=torch.uint8, device=latent.device).expand(n, levels, PAIRS).contiguous()
    w = torch.zeros((n, levels, PAIRS), dtype=torch.float32, device=latent.device)
    w[..., :d] = latent
    return idx, w


class Decoder:
    """The MLP's weights packed for lsv2_mlp_decode: BF16 weight matrices one after another
    (row-major [w_in][w_out]), BF16 biases, the widths in host memory.  The first layer's input
    is padded to LATENT_CHANNELS with zero weight rows."""

    def __init__(self, layers, device="cuda"):
        widths = [LATENT_CHANNELS] + [int(W.shape[1]) for W, _ in layers]
        d_in = int(layers[0][0].shape[0])
        if d_in > LATENT_CHANNELS:
            raise ValueError(f"decoder input width {d_in} exceeds {LATENT_CHANNELS}")
        mats, biases = [], []
        for i, (W, b) in enumerate(layers):
            W = torch.as_tensor(np.asarray(W), dtype=torch.float32)
            if i == 0:
                W = torch.cat([W, torch.zeros((LATENT_CHANNELS - d_in, W.shape[1]))], 0)
            mats.append(W.reshape(-1))
            biases.append(torch.as_tensor(np.asarray(b), dtype=torch.float32).reshape(-1))
        self.n_layers = len(layers)
        self.widths = (C.c_int32 * len(widths))(*widths)
        self.out_width = widths[-1]
        self.weights = torch.cat(mats).to(device=device, dtype=torch.bfloat16).contiguous()
        self.biases = torch.cat(biases).to(device=device, dtype=torch.bfloat16).contiguous()

    def flops_per_row(self) -> int:
        w = list(self.widths)
        return sum(2 * w[i] * w[i + 1] for i in range(self.n_layers))

    def workspace_bytes(self, rows: int, x_dtype: int = L.LSV2_F32, block_rows: int = 0) -> int:
        return L.lsv2_mlp_decode_workspace_bytes(rows, self.n_layers, self.widths, x_dtype, block_rows)

    def __call__(self, x: torch.Tensor, y: torch.Tensor, ws: torch.Tensor, block_rows: int = 0, stream=None,
                 status: torch.Tensor | None = None):
        """y [rows, out] (BF16) = g_d(x [rows, LATENT_CHANNELS] (F32 or BF16)).  block_rows >= 0: library
        GEMMs over blocks of that many rows (0: 2^20); L.LSV2_MLP_FUSED: the fused tensor-core
        kernel.  status: an int32 device word that records a device-side timeout (optional)."""
        rows = x.numel() // LATENT_CHANNELS
        x_dt = L.LSV2_BF16 if x.dtype == torch.bfloat16 else L.LSV2_F32
        L.lsv2_mlp_decode(rows, self.n_layers, self.widths, _ptr(x), x_dt, _ptr(self.weights), _ptr(self.biases),
                          _ptr(y), block_rows, _ptr(ws), ws.numel(), _ptr(status),
                          _stream(stream))


class DecoderFrame:
    """One camera of the decoder-based path: project -> bin_sort -> latent splat -> MLP decode."""

    def __init__(self, scene: DeviceScene, latent: torch.Tensor, decoder: Decoder, cam, block_rows: int = 0,
                 device="cuda"):
        idx, w = latent_pairs(latent.to(device))
        levels = int(latent.shape[1])
        # no codebook on this path: a width-0 placeholder fixes the splat's L at LATENT_CHANNELS
        self.scene = DeviceScene(scene.means, scene.scales, scene.quats, scene.opacity, idx, w,
                                 torch.empty((levels, LATENT_CHANNELS, 0), device=device))
        self.frame = Frame(self.scene, cam, device=device)
        self.decoder, self.block_rows = decoder, block_rows
        self.rows = levels * self.frame.P
        self.ws = torch.empty(max(decoder.workspace_bytes(self.rows, L.LSV2_F32, block_rows), 16), dtype=torch.uint8,
                              device=device)

    @property
    def latent_map(self) -> torch.Tensor:
        """f32 [levels, P, LATENT_CHANNELS]: channels 0..d-1 the rendered latent (Eq. 4), the rest 0."""
        return self.frame.coeff

    def project(self, stream=None):
        self.frame.project(stream)

    def bin_sort(self, stream=None):
        self.frame.bin_sort(stream)

    def splat(self, stream=None):
        self.frame.splat(stream)

    def render(self, stream=None):
        self.frame.render(stream)

    def decode(self, out: torch.Tensor, stream=None):
        """out bf16 [levels, P, D] = g_d(latent map)."""
        self.decoder(self.frame.coeff, out, self.ws, self.block_rows, stream, self.frame.status)

    def check(self):
        self.frame.check()
