"""GPU gradients (lsv2_l1_decode_backward, lsv2_splat_backward, RenderL1) against the FP64 oracle
and FP64 central finite differences.

The L1 loss decides sign(F - target) per element; where |F - target| is within rounding of 0
the two sides may take different signs, so pixels holding such near-ties are left out of the
per-pixel comparison and their possible effect is added to the bound of the sums."""
import numpy as np
import pytest

import lsv2_synth as syn
from oracle import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2507_07136_b300 import _lib as L  # noqa: E402
from paper_2507_07136_b300.autograd import RenderL1, render_l1  # noqa: E402
from paper_2507_07136_b300.pipeline import DeviceScene, Frame, _ptr, _stream  # noqa: E402


def fd_problem(D=512):
    sc, cam = syn.fd_subset()
    if D != 512:
        sc.codebook = syn.codebooks(77, 1, 64, D)
    rng = np.random.default_rng(9)
    target = rng.normal(0, 0.05, (1, cam.num_pixels, D)).astype(np.float32)
    return sc, cam, target


def gpu_splat_backward(sc, cam, dW):
    """Run the GPU splat + projection backward for a given dLoss/dW (float32 [lev, P, 64])."""
    ds = DeviceScene.from_numpy(sc)
    fr = Frame(ds, cam)
    fr.render()
    n = sc.n
    out = {k: torch.zeros(shape, device="cuda") for k, shape in
           [("dw", sc.weights.shape), ("dop", (n,)), ("dm", (n, 3)), ("ds", (n, 3)), ("dq", (n, 4))]}
    wsb = L.lsv2_splat_backward_workspace_bytes(n)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    g = torch.as_tensor(np.ascontiguousarray(dW, np.float32), device="cuda")
    L.lsv2_splat_backward(fr.ccam, n, _ptr(ds.means), _ptr(ds.scales), _ptr(ds.quats), fr.proj, _ptr(fr.tile_ranges),
                          _ptr(fr.gauss_ids), ds.levels, ds.K, 64, _ptr(ds.idx), _ptr(ds.weights), _ptr(fr.final_T),
                          _ptr(fr.n_last), _ptr(g), _ptr(ws), wsb, _ptr(out["dw"]), _ptr(out["dop"]), _ptr(out["dm"]),
                          _ptr(out["ds"]), _ptr(out["dq"]), _ptr(fr.status), _stream(None))
    fr.check()
    return {k: v.cpu().numpy().astype(np.float64) for k, v in out.items()}


def close_groupwise(got, ref, rel=2e-4, what=""):
    """Per parameter group: every entry within rel of the group's largest magnitude, and the
    whole group within rel in norm."""
    scale = np.abs(ref).max() + 1e-30
    err = np.abs(got - ref)
    assert err.max() <= rel * scale, f"{what}: max err {err.max():.3e} vs scale {scale:.3e}"
    assert np.linalg.norm(got - ref) <= rel * np.linalg.norm(ref) + 1e-30, what


def test_splat_backward_matches_oracle_fd_subset():
    sc, cam, target = fd_problem()
    g = O.l1_grads(sc, cam, target)
    out = gpu_splat_backward(sc, cam, g.dW)
    close_groupwise(out["dw"], g.dw, what="dw")
    close_groupwise(out["dop"], g.dopacity, what="dopacity")
    close_groupwise(out["dm"], g.dmeans, what="dmeans")
    close_groupwise(out["ds"], g.dscales, what="dscales")
    close_groupwise(out["dq"], g.dquats, what="dquats")


def test_l1_decode_backward_matches_oracle():
    sc, cam, target = fd_problem()
    r = O.render(sc, cam)
    ds = DeviceScene.from_numpy(sc)
    fr = Frame(ds, cam)
    fr.render()
    loss = torch.zeros(1, device="cuda")
    dW = torch.empty_like(fr.coeff)
    dS = torch.zeros_like(ds.codebook)
    tg = torch.as_tensor(target, device="cuda")
    L.lsv2_l1_decode_backward(1, fr.P, 64, 512, _ptr(fr.coeff), _ptr(ds.codebook), _ptr(tg), _ptr(loss), _ptr(dW),
                              _ptr(dS), _ptr(fr.status), _stream(None))
    fr.check()
    # reference from the GPU's own W (isolates the decode/L1 adjoint)
    Wg = fr.coeff.cpu().numpy().astype(np.float64)
    S = sc.codebook.astype(np.float64)
    F = np.einsum("lpj,ljd->lpd", Wg, S)
    res = F - target
    n = float(res.size)
    tie = np.abs(res) < 1e-6
    GF = np.sign(res) / n
    assert float(loss.item()) == pytest.approx(np.abs(res).mean(), rel=1e-5)
    dW_ref = np.einsum("lpd,ljd->lpj", GF, S)
    ok = ~tie.any(-1)[0]
    Wd = dW.cpu().numpy()
    bound = 1e-5 * np.einsum("lpd,ljd->lpj", np.abs(GF), np.abs(S)) + 1e-12
    assert np.all(np.abs(Wd[:, ok] - dW_ref[:, ok]) <= bound[:, ok])
    dS_ref = np.einsum("lpj,lpd->ljd", Wg, GF)
    slack = 2.0 * np.einsum("lpj,lpd->ljd", Wg, tie / n)
    dbound = 1e-5 * np.einsum("lpj,lpd->ljd", np.abs(Wg), np.abs(GF)) + slack + 1e-12
    assert np.all(np.abs(dS.cpu().numpy() - dS_ref) <= dbound)


def test_gpu_gradient_against_central_fd():
    """GPU gradients of the L1 loss against FP64 central differences (h = 1e-6) of the oracle's
    forward, on the 200-Gaussian 64x48 subset; coordinates whose +-h evaluations change a
    discrete decision are left out."""
    sc, cam, target = fd_problem(D=128)
    dev = "cuda"
    t = {k: torch.as_tensor(v, device=dev).requires_grad_(True) for k, v in
         [("m", sc.means), ("s", sc.scales), ("q", sc.quats), ("o", sc.opacity), ("w", sc.weights)]}
    cb = torch.as_tensor(sc.codebook, device=dev)
    idx = torch.as_tensor(sc.idx, device=dev)
    tg = torch.as_tensor(target, device=dev)
    loss = RenderL1.apply(t["m"], t["s"], t["q"], t["o"], t["w"], cb, idx, cam, tg)
    loss.backward()
    grads = [t[k].grad.cpu().numpy().astype(np.float64) for k in ["m", "s", "q", "o", "w"]]
    pr = O.project(cam, sc.means, sc.scales, sc.quats)
    ids, ranges = O.bin(cam, pr)
    denom = float(cam.num_pixels * 128)
    params = [sc.means.astype(np.float64), sc.scales.astype(np.float64), sc.quats.astype(np.float64),
              sc.opacity.astype(np.float64), sc.weights.astype(np.float64)]
    rng = np.random.default_rng(21)
    vis = np.nonzero(pr.visible)[0]
    GX = cam.grid[0]
    checked = 0
    worst = 0.0
    for gid in rng.choice(vis, 8, replace=False):
        mask = np.zeros(cam.num_tiles, np.uint8)
        for ty in range(pr.rect[gid, 1], pr.rect[gid, 3]):
            for tx in range(pr.rect[gid, 0], pr.rect[gid, 2]):
                mask[ty * GX + tx] = 1
        _, sig0 = O.l1_loss_fd_eval(params, cam, ids, ranges, mask, sc.idx, sc.codebook, target)
        for a in range(5):
            npar = params[a].reshape(params[a].shape[0], -1).shape[1]
            for j in range(npar):
                vals, sigs = [], []
                for sgn in (1, -1):
                    pp = [x.copy() for x in params]
                    pp[a].reshape(pp[a].shape[0], -1)[gid, j] += sgn * 1e-6
                    v, sg = O.l1_loss_fd_eval(pp, cam, ids, ranges, mask, sc.idx, sc.codebook, target)
                    vals.append(v)
                    sigs.append(sg)
                if sigs[0] != sig0 or sigs[1] != sig0:
                    continue
                fd = (vals[0] - vals[1]).sum() / 2e-6 / denom
                ga = grads[a].reshape(grads[a].shape[0], -1)[gid, j]
                scale = np.abs(grads[a]).max()
                worst = max(worst, abs(fd - ga) / (scale + 1e-30))
                checked += 1
    assert checked >= 60
    assert worst <= 2e-4, worst


def test_autograd_activations_chain():
    """Gradients w.r.t. log-scales and opacity logits: exp and sigmoid chained by torch."""
    sc, cam, target = fd_problem(D=128)
    dev = "cuda"
    g = O.l1_grads(sc, cam, target)
    log_s = torch.as_tensor(np.log(sc.scales.astype(np.float64)).astype(np.float32), device=dev).requires_grad_(True)
    o = sc.opacity.astype(np.float64)
    logit = torch.as_tensor(np.log(o / (1 - o)).astype(np.float32), device=dev).requires_grad_(True)
    m = torch.as_tensor(sc.means, device=dev).requires_grad_(True)
    q = torch.as_tensor(sc.quats, device=dev).requires_grad_(True)
    w = torch.as_tensor(sc.weights, device=dev).requires_grad_(True)
    cb = torch.as_tensor(sc.codebook, device=dev).requires_grad_(True)
    loss = render_l1(m, log_s, q, logit, w, cb, torch.as_tensor(sc.idx, device=dev), cam,
                     torch.as_tensor(target, device=dev))
    loss.backward()
    close_groupwise(log_s.grad.cpu().numpy(), g.dscales * sc.scales, what="dlog_scales")
    close_groupwise(logit.grad.cpu().numpy(), g.dopacity * o * (1 - o), what="dlogits")
    assert cb.grad is not None and float(cb.grad.abs().sum()) > 0


def oracle_blend_adjoint(sc, cam, dW):
    """The oracle's blend adjoint for a given dLoss/dW, chained through the projection Jacobian:
    (dw, dopacity, dmeans, dscales, dquats)."""
    import ctypes as C
    r = O.render(sc, cam)
    n, lev, K = sc.n, sc.levels, sc.K
    dw = np.zeros((n, lev, K))
    dop = np.zeros(n)
    dm2 = np.zeros((n, 2))
    dcn = np.zeros((n, 3))
    c = O.cam_struct(cam)
    op32, ids32, rng32 = O._f32(sc.opacity), np.ascontiguousarray(r.ids, np.uint32), np.ascontiguousarray(r.ranges)
    if ids32.size == 0:
        ids32 = np.zeros(1, np.uint32)
    idx8, w32, G64 = np.ascontiguousarray(sc.idx), O._f32(sc.weights), np.ascontiguousarray(dW, np.float64)
    O.lib().orc_blend_backward(C.byref(c), n, O._p(r.proj.mean2d), O._p(r.proj.conic), O._p(op32), O._p(ids32),
                               O._p(rng32), lev, K, 64, O._p(idx8), O._p(w32), O._p(G64), O._p(dw), O._p(dop),
                               O._p(dm2), O._p(dcn))
    jac = O.project_jacobian(cam, sc.means, sc.scales, sc.quats)
    dp = np.einsum("nk,nkp->np", np.concatenate([dm2, dcn], 1), jac)
    dp[~r.proj.visible] = 0
    return dw, dop, dp[:, :3], dp[:, 3:6], dp[:, 6:]


@pytest.mark.parametrize("levels,K,tile", [(1, 2, 16), (1, 8, 16), (1, 4, 8), (3, 4, 16), (2, 4, 16)])
def test_splat_adjoint_configurations(levels, K, tile):
    """Every (levels, K) the adjoint supports, on both of its kernels: at one level with 16 x 16
    tiles the persistent one with dLoss/dW in tensor memory (K = 2: four Gaussians per
    reduce-scatter, K = 8: two), otherwise one CTA per tile with shared-memory columns."""
    sc = syn.make_scene(3000, levels, seed=31 + K, mean_kind="uniform", mean_param=1.0, log_scale_mu=-3.2,
                        log_scale_sigma=0.4, K=K)
    cam = syn.orbit_camera(150, 110, 4.0, tile=(tile, tile))
    rng = np.random.default_rng(14)
    dW = (rng.standard_normal((levels, cam.num_pixels, 64)) * 1e-3).astype(np.float32)
    out = gpu_splat_backward(sc, cam, dW)
    ref = oracle_blend_adjoint(sc, cam, dW)
    for k, r in zip(("dw", "dop", "dm", "ds", "dq"), ref):
        assert np.abs(r).max() > 0, k
        close_groupwise(out[k], r, what=k)


def test_backward_full_scale_splat_adjoint():
    """100,000 Gaussians at 720x540: feed the same dLoss/dW to the GPU splat backward and the
    oracle's blend adjoint; per-Gaussian gradients must agree."""
    sc, cam = syn.differentiation()
    rng = np.random.default_rng(13)
    dW = (rng.standard_normal((1, cam.num_pixels, 64)) * 1e-7).astype(np.float32)
    out = gpu_splat_backward(sc, cam, dW)
    r = O.render(sc, cam)
    n = sc.n
    import ctypes as C
    dw = np.zeros((n, 1, 4))
    dop = np.zeros(n)
    dm2 = np.zeros((n, 2))
    dcn = np.zeros((n, 3))
    c = O.cam_struct(cam)
    op32, ids32, rng32 = O._f32(sc.opacity), np.ascontiguousarray(r.ids, np.uint32), np.ascontiguousarray(r.ranges)
    idx8, w32, G64 = np.ascontiguousarray(sc.idx), O._f32(sc.weights), dW.astype(np.float64)
    O.lib().orc_blend_backward(C.byref(c), n, O._p(r.proj.mean2d), O._p(r.proj.conic), O._p(op32), O._p(ids32),
                               O._p(rng32), 1, 4, 64, O._p(idx8), O._p(w32), O._p(G64), O._p(dw), O._p(dop),
                               O._p(dm2), O._p(dcn))
    close_groupwise(out["dw"], dw, what="dw")
    close_groupwise(out["dop"], dop, what="dopacity")
    jac = O.project_jacobian(cam, sc.means, sc.scales, sc.quats)
    dp = np.einsum("nk,nkp->np", np.concatenate([dm2, dcn], 1), jac)
    dp[~r.proj.visible] = 0
    close_groupwise(out["dm"], dp[:, :3], what="dmeans")
    close_groupwise(out["ds"], dp[:, 3:6], what="dscales")
    close_groupwise(out["dq"], dp[:, 6:], what="dquats")
