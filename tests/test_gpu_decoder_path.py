"""GPU parity of the decoder-based comparison path (LangSplat*, Sec. 3.1, Table 1), through the C ABI.

* Latent render (Eq. 4) with lsv2_splat_coeffs at L = 8: channels 0..2 within 1e-5 of the oracle's
  FP64 blend of the d = 3 latent, relative to the blend of |f| (the latent is signed, so the bound
  scales with the sum of magnitudes, not with the possibly cancelled result); channels 3..7 zero.
* lsv2_mlp_decode on integer-valued inputs, weights and biases whose every intermediate is an
  integer below 256 (exact in BF16, exact in FP32 accumulation): equal to the oracle bit for bit,
  over several row blocks and a ragged tail, on both implementations -- a check of the layouts,
  bias, ReLU placement and blocking with no rounding in the way.
* The fused tensor-core kernel (LSV2_MLP_FUSED) on integer-valued MLPs of other shapes, each equal
  to the oracle bit for bit: widths of 16 mod 32 (the epilogue's last piece is 16 columns), a
  last layer cut into parts of 256 and 144 outputs, a single layer, an input of 24 columns, and the
  workload's seven layers over enough rows that every CTA of the persistent grid runs several
  tiles (with a ragged tail and the BF16 input).
* lsv2_mlp_decode with the random decoder of the workload: within the BF16 bound of the FP64
  oracle.  The GPU rounds the input and each of the seven layer outputs to BF16 (relative 2^-9
  each); eight such roundings add in quadrature to about sqrt(8) 2^-9 = 0.55% of a row's norm.
  Bound: 3% normwise per row and 0.1 x the row's RMS per element.
* The whole path at 300,000 Gaussians, 1440x1080, three levels on sampled pixels, with the library
  decoder and with the fused one (4.67 M rows: about 246 tiles per persistent CTA).
"""
import ctypes as C

import numpy as np
import pytest

import lsv2_synth as syn
from oracle import oracle as O

from gpu_helpers import KNIFE_EDGE

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2507_07136_b300 import _lib as L  # noqa: E402
from paper_2507_07136_b300.decoder_path import LATENT_CHANNELS, Decoder, DecoderFrame  # noqa: E402
from paper_2507_07136_b300.pipeline import DeviceScene  # noqa: E402

NORMWISE_TOL = 3e-2
ELEMENT_TOL = 0.1


def assert_decoder_close(got, ref, what):
    got = np.asarray(got, np.float64)
    nrm = np.linalg.norm(got - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), 1e-30)
    assert nrm.max() <= NORMWISE_TOL, f"{what}: normwise {nrm.max():.4f}"
    rms = np.sqrt((ref ** 2).mean(axis=1, keepdims=True))
    el = (np.abs(got - ref) / rms).max()
    assert el <= ELEMENT_TOL, f"{what}: element {el:.4f} of the row RMS"


def tiny_latent_scene():
    sc = syn.make_scene(2000, 3, mean_kind="uniform", mean_param=1.0, log_scale_mu=-3.0, log_scale_sigma=0.3)
    return sc, syn.orbit_camera(128, 96, 4.0), syn.latent_features(sc.n, 3)


def test_latent_render_tiny():
    sc, cam, lat = tiny_latent_scene()
    ds = DeviceScene.from_numpy(sc)
    dec = Decoder(syn.decoder_mlp())
    fr = DecoderFrame(ds, torch.as_tensor(lat), dec, cam)
    fr.render()
    fr.check()
    got = fr.latent_map.cpu().numpy().astype(np.float64)
    assert got.shape == (3, cam.num_pixels, LATENT_CHANNELS)
    assert np.all(got[:, :, 3:] == 0.0)
    r = O.render(sc, cam)
    ref = O.blend(cam, r.proj, sc.opacity, r.ids, r.ranges, dense=lat.astype(np.float64), mode=2)
    mag = O.blend(cam, r.proj, sc.opacity, r.ids, r.ranges, dense=np.abs(lat).astype(np.float64), mode=2)
    ok = ref.margin > KNIFE_EDGE
    err = np.abs(got[:, ok, :3] - ref.out[:, ok])
    bound = 1e-5 * mag.out[:, ok] + 1e-9
    assert np.all(err <= bound), f"latent map: worst x{(err / bound).max():.2f} of bound"
    assert np.abs(ref.out).max() > 0.1
    np.testing.assert_array_equal(fr.frame.n_last.cpu().numpy()[ok], ref.n_last[ok])


def integer_decoder(widths, fan_in, rng):
    """Weights in {-1, 0, +1} with `fan_in` nonzeros per output column spread over the whole input
    range, biases in {-1, 0, 1}."""
    layers = []
    for l in range(len(widths) - 1):
        W = np.zeros((widths[l], widths[l + 1]), np.float32)
        for j in range(widths[l + 1]):
            rows = rng.choice(widths[l], min(fan_in, widths[l]), replace=False)
            W[rows, j] = rng.choice([-1.0, 1.0], rows.size)
        layers.append((W, rng.integers(-1, 2, widths[l + 1]).astype(np.float32)))
    return layers


@pytest.mark.parametrize("block_rows", [0, 1024, L.LSV2_MLP_FUSED])
def test_mlp_exact_on_integers(block_rows):
    rng = np.random.default_rng(21)
    widths = (LATENT_CHANNELS, 64, 128, 512)
    layers = integer_decoder(widths, 4, rng)   # |h| <= ((2*4 + 1)*4 + 1)*4 + 1 = 149
    rows = 5 * 1024 + 77                       # five blocks of 1024 and a ragged tail
    x = rng.integers(-2, 3, (rows, LATENT_CHANNELS)).astype(np.float32)
    ref = O.mlp_decode(x, layers)
    assert np.abs(ref).max() < 256 and np.all(ref == np.round(ref))
    dec = Decoder(layers)
    xd = torch.as_tensor(x, device="cuda")
    y = torch.empty((rows, widths[-1]), dtype=torch.bfloat16, device="cuda")
    ws = torch.empty(dec.workspace_bytes(rows, L.LSV2_F32, block_rows), dtype=torch.uint8, device="cuda")
    dec(xd, y, ws, block_rows)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(y.float().cpu().numpy().astype(np.float64), ref)
    # the same from a BF16 input (x is exact in BF16)
    ws16 = torch.empty(dec.workspace_bytes(rows, L.LSV2_BF16, block_rows), dtype=torch.uint8, device="cuda")
    y16 = torch.empty_like(y)
    dec(xd.to(torch.bfloat16), y16, ws16, block_rows)
    torch.cuda.synchronize()
    assert torch.equal(y16, y)


def pack_layers(layers):
    W = torch.cat([torch.as_tensor(np.asarray(w, np.float32)).reshape(-1) for w, _ in layers])
    b = torch.cat([torch.as_tensor(np.asarray(bb, np.float32)).reshape(-1) for _, bb in layers])
    return W.to("cuda", torch.bfloat16).contiguous(), b.to("cuda", torch.bfloat16).contiguous()


def run_mlp(layers, x, block_rows=0, x_dtype=torch.float32):
    """lsv2_mlp_decode through the C ABI on host arrays; returns the output as float64 and the status."""
    widths = [x.shape[1]] + [int(w.shape[1]) for w, _ in layers]
    wc = (C.c_int32 * len(widths))(*widths)
    W, b = pack_layers(layers)
    rows = x.shape[0]
    xd = torch.as_tensor(x, device="cuda").to(x_dtype).contiguous()
    dt = L.LSV2_BF16 if x_dtype == torch.bfloat16 else L.LSV2_F32
    y = torch.full((rows, widths[-1]), float("nan"), dtype=torch.bfloat16, device="cuda")
    ws = torch.empty(max(L.lsv2_mlp_decode_workspace_bytes(rows, len(layers), wc, dt, block_rows), 16),
                     dtype=torch.uint8, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    L.lsv2_mlp_decode(rows, len(layers), wc, xd.data_ptr(), dt, W.data_ptr(), b.data_ptr(), y.data_ptr(),
                      block_rows, ws.data_ptr(), ws.numel(), st.data_ptr(), 0)
    torch.cuda.synchronize()
    return y.float().cpu().numpy().astype(np.float64), int(st.item())


@pytest.mark.parametrize("widths,fan_in,x_max,rows", [
    ((8, 48, 80, 400), 4, 2, 3 * 1024 + 77),         # widths of 16 mod 32; last layer 256 + 144
    ((8, 64), 4, 2, 1000),                           # one layer: input straight to output
    ((24, 256, 256, 512), 2, 2, 2 * 1024 + 5),       # input of 24 columns, zero-padded to 32
    ((8, 16, 32, 64, 128, 256, 256, 512), 2, 1, 148 * 128 * 5 + 77),   # several tiles per CTA
])
def test_mlp_fused_exact_on_integers(widths, fan_in, x_max, rows):
    rng = np.random.default_rng(24)
    layers = integer_decoder(widths, fan_in, rng)
    x = rng.integers(-x_max, x_max + 1, (rows, widths[0])).astype(np.float32)
    ref = O.mlp_decode(x, layers)
    assert np.abs(ref).max() <= 256 and np.all(ref == np.round(ref))
    got, st = run_mlp(layers, x, block_rows=L.LSV2_MLP_FUSED)
    assert st == 0
    np.testing.assert_array_equal(got, ref)
    got16, st = run_mlp(layers, x, block_rows=L.LSV2_MLP_FUSED, x_dtype=torch.bfloat16)
    assert st == 0
    np.testing.assert_array_equal(got16, ref)


@pytest.mark.parametrize("rows", [1, 127, 128, 129, 148 * 128, 148 * 128 + 1])
def test_mlp_fused_row_counts(rows):
    """Tile and grid boundaries of the persistent kernel: a single row (grid of one CTA, one
    ragged tile), one row short of / exactly / one past a 128-row tile, exactly one tile per SM,
    and one tile past that (the first CTA takes a second tile)."""
    rng = np.random.default_rng(27)
    widths = (8, 16, 32, 64, 128, 256, 256, 512)
    layers = integer_decoder(widths, 2, rng)
    x = rng.integers(-1, 2, (rows, 8)).astype(np.float32)
    ref = O.mlp_decode(x, layers)
    got, st = run_mlp(layers, x, block_rows=L.LSV2_MLP_FUSED)
    assert st == 0
    np.testing.assert_array_equal(got, ref)


def test_mlp_fused_and_library_agree_on_the_workload_decoder():
    """The fused kernel and the library GEMMs round the same FP32 sums to BF16 after every layer and
    differ only in summation order: both within the BF16 bound of the FP64 oracle, and of each other."""
    rng = np.random.default_rng(25)
    layers = syn.decoder_mlp()
    rows = 4096 + 33
    x = np.zeros((rows, LATENT_CHANNELS), np.float32)
    x[:, :3] = rng.standard_normal((rows, 3))
    W0 = np.concatenate([layers[0][0], np.zeros((LATENT_CHANNELS - 3, layers[0][0].shape[1]), np.float32)])
    padded = [(W0, layers[0][1])] + list(layers[1:])
    fused, st = run_mlp(padded, x, block_rows=L.LSV2_MLP_FUSED)
    assert st == 0
    lib_, _ = run_mlp(padded, x, block_rows=1024)
    ref = O.mlp_decode(x[:, :3], layers)
    assert_decoder_close(fused, ref, "fused")
    assert_decoder_close(lib_, ref, "library")
    assert_decoder_close(fused, lib_, "fused vs library")


def test_mlp_random_decoder_against_oracle():
    rng = np.random.default_rng(22)
    layers = syn.decoder_mlp()
    rows = 3 * 1024 + 129
    x = np.zeros((rows, LATENT_CHANNELS), np.float32)
    x[:, :3] = rng.standard_normal((rows, 3)) * rng.choice([0.3, 1.0, 3.0], (rows, 1))
    ref = O.mlp_decode(x[:, :3], layers)
    dec = Decoder(layers)
    y = torch.empty((rows, 512), dtype=torch.bfloat16, device="cuda")
    for block_rows in (0, 1024, L.LSV2_MLP_FUSED):
        ws = torch.empty(dec.workspace_bytes(rows, L.LSV2_F32, block_rows), dtype=torch.uint8, device="cuda")
        y.fill_(float("nan"))
        dec(torch.as_tensor(x, device="cuda"), y, ws, block_rows)
        torch.cuda.synchronize()
        assert_decoder_close(y.float().cpu().numpy(), ref, f"block_rows {block_rows}")


def test_mlp_empty_and_rejected_calls():
    dec = Decoder(syn.decoder_mlp())
    ws = torch.empty(dec.workspace_bytes(0), dtype=torch.uint8, device="cuda")
    x = torch.zeros((1, LATENT_CHANNELS), device="cuda")
    y = torch.zeros((1, 512), dtype=torch.bfloat16, device="cuda")
    L.lsv2_mlp_decode(0, dec.n_layers, dec.widths, x.data_ptr(), L.LSV2_F32, dec.weights.data_ptr(),
                      dec.biases.data_ptr(), y.data_ptr(), 0, ws.data_ptr(), ws.numel(), 0, 0)
    assert float(y.float().abs().sum()) == 0.0
    with pytest.raises(L.LSV2Error) as e:   # a workspace one byte short
        L.lsv2_mlp_decode(1, dec.n_layers, dec.widths, x.data_ptr(), L.LSV2_F32, dec.weights.data_ptr(),
                          dec.biases.data_ptr(), y.data_ptr(), 0, ws.data_ptr(), dec.workspace_bytes(1) - 1, 0, 0)
    assert e.value.code == L.LSV2_ERR_INVALID_ARGUMENT
    bad = (C.c_int32 * 3)(8, 12, 512)       # a width that is not a multiple of 8
    with pytest.raises(L.LSV2Error) as e:
        L.lsv2_mlp_decode(1, 2, bad, x.data_ptr(), L.LSV2_F32, dec.weights.data_ptr(), dec.biases.data_ptr(),
                          y.data_ptr(), 0, ws.data_ptr(), ws.numel(), 0, 0)
    assert e.value.code == L.LSV2_ERR_UNSUPPORTED


def test_decoder_path_at_scale_sampled():
    """300,000 Gaussians, three levels, 1440x1080 (4.67 M decoder rows, 72 row blocks): the latent
    map and the decoded features on 1,500 sampled pixels against the oracle's render and decoder."""
    sc, cam, lat, layers = syn.latent_at_scale()
    ds = DeviceScene.from_numpy(sc)
    dec = Decoder(layers)
    fr = DecoderFrame(ds, torch.as_tensor(lat), dec, cam)
    F = torch.empty((3, cam.num_pixels, 512), dtype=torch.bfloat16, device="cuda")
    fr.render()
    fr.decode(F)
    fr.check()
    rng = np.random.default_rng(23)
    px = rng.integers(0, cam.width, 1500).astype(np.int32)
    py = rng.integers(0, cam.height, 1500).astype(np.int32)
    pr = O.project(cam, sc.means, sc.scales, sc.quats)
    ids, ranges = O.bin(cam, pr)
    ref = O.blend(cam, pr, sc.opacity, ids, ranges, dense=lat.astype(np.float64), mode=2, px=px, py=py)
    mag = O.blend(cam, pr, sc.opacity, ids, ranges, dense=np.abs(lat).astype(np.float64), mode=2, px=px, py=py)
    ok = ref.margin > KNIFE_EDGE
    assert ok.sum() > 1400
    flat = torch.as_tensor((py.astype(np.int64) * cam.width + px)[ok], device="cuda")
    got_lat = fr.latent_map[:, flat].cpu().numpy().astype(np.float64)
    err = np.abs(got_lat[:, :, :3] - ref.out[:, ok])
    bound = 1e-5 * mag.out[:, ok] + 1e-9
    assert np.all(err <= bound), f"latent map: worst x{(err / bound).max():.2f} of bound"
    assert np.all(got_lat[:, :, 3:] == 0.0)
    got_F = F[:, flat].float().cpu().numpy().reshape(-1, 512)
    ref_F = O.mlp_decode(ref.out[:, ok].reshape(-1, 3), layers)
    assert_decoder_close(got_F, ref_F, "decoded features")
    # the fused tensor-core decoder over the same 4.67 M rows (about 246 tiles per persistent CTA,
    # output offsets past 2^31 elements): the same sampled rows within the same bars
    fr_fused = DecoderFrame(ds, torch.as_tensor(lat), dec, cam, block_rows=L.LSV2_MLP_FUSED)
    fr_fused.frame.coeff.copy_(fr.frame.coeff)
    F2 = torch.full_like(F, float("nan"))
    fr_fused.decode(F2)
    fr_fused.check()
    got_F2 = F2[:, flat].float().cpu().numpy().reshape(-1, 512)
    assert_decoder_close(got_F2, ref_F, "decoded features (fused kernel)")
    assert not torch.isnan(F2[:, -1]).any()   # the last row of every level was written
