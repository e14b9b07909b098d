"""Pins for the FP64 oracle: closed forms, invariants and brute force (CPU only).

The paper prints no worked numeric example, so the oracle is pinned to what its
equations fix: closed-form projections of isotropic/axis-aligned Gaussians (Eq. 2 +
EWA), the transmittance products of Eq. 3/7 for stacked Gaussians of known alpha,
Sec. 3.4's statement that blending zero coefficients does not change the result,
Eq. 7's linearity, brute-force tile enumeration, the relevancy score's special
cases, and finite differences for the gradients.  Each test is chosen so that a
plausible slip in the oracle (dropped term, swapped index, wrong sign) fails it.
"""
import json
import math
import os

import numpy as np
import pytest

import lsv2_synth as syn
from oracle import oracle as O

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))


def _scene(means, scales, quats, opac, idx, w, cb=None, L=64, D=32, seed=1):
    n = len(means)
    idx = np.asarray(idx, np.uint8).reshape(n, -1, np.asarray(idx).shape[-1])
    w = np.asarray(w, np.float32).reshape(idx.shape)
    if cb is None:
        cb = syn.codebooks(seed, idx.shape[1], L, D)
    return syn.Scene(np.asarray(means, np.float32), np.asarray(scales, np.float32),
                     np.asarray(quats, np.float32), np.asarray(opac, np.float32), idx, w, cb)


# ----------------------------------------------------------------------------- projection

def test_isotropic_on_axis_closed_form():
    """Eq. 2 + EWA: isotropic Sigma on the optical axis -> Sigma' = (f s/z)^2 I + 0.3 I."""
    cam = syn.orbit_camera(129, 97, 4.0)
    rng = np.random.default_rng(0)
    q = syn.unit_rows(rng.standard_normal((6, 4)))
    z_world = np.array([-1.0, -0.5, 0.0, 0.5, 1.0, 2.0])
    s = np.array([0.01, 0.02, 0.05, 0.03, 0.07, 0.04])
    means = np.stack([np.zeros(6), np.zeros(6), z_world], 1)
    scales = np.repeat(s[:, None], 3, 1)
    pr = O.project(cam, means, scales, q)
    for g in range(6):
        m32 = np.float32(z_world[g]).astype(np.float64)
        z = m32 + 4.0
        s32 = np.float64(np.float32(s[g]))
        var = (cam.fx * s32 / z) ** 2 + float(np.float32(0.3))
        assert pr.mean2d[g] == pytest.approx([cam.cx, cam.cy], abs=1e-12)
        np.testing.assert_allclose(pr.conic[g], [1 / var, 0.0, 1 / var], rtol=1e-6, atol=1e-12)
        np.testing.assert_allclose(pr.cov2d[g], [var, 0.0, var], rtol=1e-6, atol=1e-12)


def test_isotropic_off_axis_closed_form():
    """EWA Jacobian inside the guard band: Sigma'_00 = s^2 f^2 (1/z^2 + x^2/z^4) + 0.3."""
    cam = syn.orbit_camera(200, 150, 5.0)
    xs = np.array([-1.0, -0.3, 0.4, 1.2])
    means = np.stack([xs, np.zeros(4), np.zeros(4)], 1).astype(np.float32)
    s = 0.05
    scales = np.full((4, 3), s, np.float32)
    q = np.tile([1.0, 0, 0, 0], (4, 1)).astype(np.float32)
    pr = O.project(cam, means, scales, q)
    f = cam.fx
    for g in range(4):
        x = float(means[g, 0])
        z = 5.0
        s2 = float(np.float32(s)) ** 2
        c00 = s2 * f * f * (1 / z**2 + x**2 / z**4) + float(np.float32(0.3))
        c11 = s2 * f * f / z**2 + float(np.float32(0.3))
        np.testing.assert_allclose(pr.cov2d[g], [c00, 0.0, c11], rtol=1e-6, atol=1e-12)
        assert pr.mean2d[g, 0] == pytest.approx(f * x / z + cam.cx, abs=1e-9)


def test_axis_aligned_rotated_in_plane():
    """Anisotropic Gaussian on the axis rotated by theta about the view axis:
    Sigma' = R2(theta) diag((f s0/z)^2, (f s1/z)^2) R2(theta)^T + 0.3 I."""
    cam = syn.orbit_camera(101, 101, 4.0)
    th = 0.7
    q = np.array([[math.cos(th / 2), 0, 0, math.sin(th / 2)]], np.float32)
    s = np.array([[0.06, 0.02, 0.04]], np.float32)
    pr = O.project(cam, np.zeros((1, 3), np.float32), s, q)
    f, z = cam.fx, 4.0
    qd = q.astype(np.float64)[0]
    qd /= np.linalg.norm(qd)
    thd = 2 * math.atan2(qd[3], qd[0])
    R2 = np.array([[math.cos(thd), -math.sin(thd)], [math.sin(thd), math.cos(thd)]])
    sd = s.astype(np.float64)[0]
    Sig = R2 @ np.diag([(f * sd[0] / z) ** 2, (f * sd[1] / z) ** 2]) @ R2.T + float(np.float32(0.3)) * np.eye(2)
    np.testing.assert_allclose(pr.cov2d[0], [Sig[0, 0], Sig[0, 1], Sig[1, 1]], rtol=1e-9)
    inv = np.linalg.inv(Sig)
    np.testing.assert_allclose(pr.conic[0], [inv[0, 0], inv[0, 1], inv[1, 1]], rtol=1e-9)


def test_quaternion_sign_and_scale_invariance():
    """q and -q, and q scaled by a power of two, are the same rotation: decisions bit-equal."""
    sc, cam = syn.tiny()
    a = O.project(cam, sc.means, sc.scales, sc.quats)
    b = O.project(cam, sc.means, sc.scales, -sc.quats)
    c = O.project(cam, sc.means, sc.scales, 2.0 * sc.quats)
    for o in (b, c):
        assert np.array_equal(a.flags, o.flags) and np.array_equal(a.rect, o.rect)
        assert np.array_equal(a.radius, o.radius)
        assert np.array_equal(a.depth_key.view(np.uint32), o.depth_key.view(np.uint32))
        np.testing.assert_allclose(a.conic, o.conic, rtol=1e-12, atol=1e-12)


def test_culling_cases():
    """Behind the near plane, zero quaternion, or off screen -> not visible."""
    cam = syn.orbit_camera(64, 48, 4.0)
    means = np.array([[0, 0, -3.9], [0, 0, -5.0], [0, 0, 0], [100, 0, 0], [0, 0, 0]], np.float32)
    q = np.array([[1, 0, 0, 0]] * 4 + [[0, 0, 0, 0]], np.float32)
    pr = O.project(cam, means, np.full((5, 3), 0.05, np.float32), q)
    assert list(pr.visible) == [False, False, True, False, False]


def test_decision_path_agrees_with_fp64_projection():
    """The FP32 decision spec (N N^T form) and the FP64 projection (J W Sigma W^T J^T form)
    are independent formulations; radius and rectangle must agree except at knife edges."""
    sc, cam = syn.tiny()
    pr = O.project(cam, sc.means, sc.scales, sc.quats)
    v = pr.visible
    c00, c01, c11 = pr.cov2d[:, 0], pr.cov2d[:, 1], pr.cov2d[:, 2]
    mid = 0.5 * (c00 + c11)
    lam = mid + np.sqrt(np.maximum(0.1, (0.5 * (c00 - c11)) ** 2 + c01**2))
    r3 = 3.0 * np.sqrt(lam)
    r64 = np.ceil(r3)
    safe = v & (np.abs(r3 - np.round(r3)) > 1e-4)
    assert safe.sum() > 0.9 * v.sum()
    assert np.array_equal(r64[safe].astype(np.int32), pr.radius[safe])
    u, vv = pr.mean2d[:, 0], pr.mean2d[:, 1]
    x0 = np.clip(np.floor((u - pr.radius) / 16), 0, cam.grid[0])
    y1 = np.clip(np.floor((vv + pr.radius + 15) / 16), 0, cam.grid[1])
    edge = np.minimum(np.abs((u - pr.radius) / 16 - np.round((u - pr.radius) / 16)),
                      np.abs((vv + pr.radius + 15) / 16 - np.round((vv + pr.radius + 15) / 16)))
    ok = safe & (edge > 1e-5)
    assert np.array_equal(x0[ok].astype(np.int32), pr.rect[ok, 0])
    assert np.array_equal(y1[ok].astype(np.int32), pr.rect[ok, 3])


def test_rect_covers_three_sigma_footprint():
    """The tile rectangle (3DGS convention: x0 = floor((u-r)/16), x1 = floor((u+r+15)/16))
    covers every pixel column in [u-r, u+r-1] and row in [v-r, v+r-1]."""
    sc, cam = syn.tiny()
    pr = O.project(cam, sc.means, sc.scales, sc.quats)
    for g in np.nonzero(pr.visible)[0][:300]:
        u, v = pr.mean2d[g]
        r = float(pr.radius[g])
        for (x, y) in [(u - r + 1e-3, v), (u + r - 1 - 1e-3, v), (u, v - r + 1e-3), (u, v + r - 1 - 1e-3)]:
            if 0 <= x < cam.width and 0 <= y < cam.height:
                tx, ty = int(x) // 16, int(y) // 16
                assert pr.rect[g, 0] <= tx < pr.rect[g, 2] and pr.rect[g, 1] <= ty < pr.rect[g, 3]


def test_degenerate_branch_needle():
    """A needle Gaussian (one log-scale -14) seen edge-on takes the FP64 decision branch."""
    cam = syn.orbit_camera(128, 96, 4.0)
    s = np.array([[math.exp(-14), math.exp(-14), 0.2], [0.05, 0.05, 0.05]], np.float32)
    q = np.array([[1, 0, 0, 0], [1, 0, 0, 0]], np.float32)
    means = np.array([[0.1, 0.1, 0.0], [0.1, 0.1, 0.0]], np.float32)
    s[0] = [math.exp(-14), 0.2, math.exp(-14)]
    pr = O.project(cam, means, s, q)
    assert pr.flags[0] & 2 and not (pr.flags[1] & 2)
    assert pr.visible.all()


# ----------------------------------------------------------------------------- binning

def test_binning_brute_force():
    """Tile lists by brute-force enumeration of (tile, Gaussian) pairs; depth order by Python sort."""
    sc, cam = syn.tiny()
    pr = O.project(cam, sc.means, sc.scales, sc.quats)
    ids, ranges = O.bin(cam, pr)
    GX, GY = cam.grid
    assert ids.size == pr.tiles_touched.sum()
    vis = np.nonzero(pr.visible)[0]
    for ty in range(GY):
        for tx in range(GX):
            t = ty * GX + tx
            inside = [g for g in vis if pr.rect[g, 0] <= tx < pr.rect[g, 2] and pr.rect[g, 1] <= ty < pr.rect[g, 3]]
            inside.sort(key=lambda g: (float(pr.depth_key[g]), g))
            got = list(ids[ranges[t, 0]:ranges[t, 1]])
            assert got == inside


# ----------------------------------------------------------------------------- blending

def test_stacked_half_alpha_closed_form():
    """Eq. 3/7: 20 Gaussians of alpha 0.5 at one pixel -> 13 contributors, T = 2^-13."""
    gold = GOLD["stacked_half_alpha"]
    cam = syn.orbit_camera(33, 33, 4.0)
    n = 20
    means = np.stack([np.zeros(n), np.zeros(n), 0.1 * np.arange(n)], 1)
    idx = np.stack([np.arange(n), 20 + np.arange(n), 40 + np.arange(n), 60 + np.arange(n) % 4], 1)[:, None, :]
    w = np.tile([0.5, 0.25, 0.125, 0.125], (n, 1))[:, None, :]
    sc = _scene(means, np.full((n, 3), 0.05), np.tile([1, 0, 0, 0], (n, 1)), np.full(n, 0.5), idx, w)
    r = O.render(sc, cam, px=np.array([16]), py=np.array([16]))
    assert r.blend.n_contrib[0] == gold["n_contrib"]
    assert r.blend.final_T[0] == gold["final_T"]
    expect = np.zeros(64)
    for k, e in enumerate(gold["e"]):
        for j in range(4):
            expect[idx[k, 0, j]] += w[k, 0, j] * e
    assert np.array_equal(r.blend.out[0, 0], expect)
    assert r.blend.out[0, 0].sum() == 1.0 - 2.0**-13


def test_single_gaussian_closed_form():
    """One isotropic Gaussian on the axis: W(v) = w min(0.99, o exp(-|v-c|^2 / (2 var)))."""
    cam = syn.orbit_camera(65, 49, 4.0)
    s, o = 0.03, 0.8
    sc = _scene([[0, 0, 0]], [[s, s, s]], [[1, 0, 0, 0]], [o], [[[3, 9, 27, 63]]],
                [[[0.5, 0.25, 0.125, 0.125]]])
    px, py = O.all_pixels(cam)
    r = O.render(sc, cam, px=px, py=py)
    var = (cam.fx * float(np.float32(s)) / 4.0) ** 2 + float(np.float32(0.3))
    d2 = (px - cam.cx) ** 2 + (py - cam.cy) ** 2
    alpha = np.minimum(float(np.float32(0.99)), float(np.float32(o)) * np.exp(-0.5 * d2 / var))
    tx, ty = px // 16, py // 16
    pr = r.proj
    in_rect = (tx >= pr.rect[0, 0]) & (tx < pr.rect[0, 2]) & (ty >= pr.rect[0, 1]) & (ty < pr.rect[0, 3])
    alpha = np.where((alpha >= O.ALPHA_MIN) & in_rect, alpha, 0.0)
    np.testing.assert_allclose(r.blend.out[0][:, 9], 0.25 * alpha, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(r.blend.final_T, 1 - alpha, rtol=1e-12)


def test_coefficient_sum_is_one_minus_T():
    """With sum_k w_k = 1 exactly, sum_l W_l = sum_i e_i = 1 - T_final (telescoping of Eq. 3)."""
    sc, cam = syn.tiny()
    sc.weights[:] = np.array([0.5, 0.25, 0.125, 0.125], np.float32)
    r = O.render(sc, cam)
    np.testing.assert_allclose(r.blend.out[0].sum(-1), 1.0 - r.blend.final_T, rtol=0, atol=1e-14)


def test_sparse_equals_dense_L():
    """Sec. 3.4: blending only the K nonzeros equals blending the full L-vector."""
    sc, cam = syn.tiny()
    r = O.render(sc, cam)
    dense = np.zeros((sc.n, 1, 64))
    for k in range(4):
        np.add.at(dense, (np.arange(sc.n), 0, sc.idx[:, 0, k].astype(int)), sc.weights[:, 0, k])
    d = O.blend(cam, r.proj, sc.opacity, r.ids, r.ranges, dense=dense, mode=1)
    np.testing.assert_allclose(d.out, r.blend.out, rtol=0, atol=1e-15)
    assert np.array_equal(d.final_T, r.blend.final_T)


def test_duplicate_and_permuted_pairs():
    """A repeated index sums its weights; permuting the K pairs changes nothing."""
    sc, cam = syn.tiny()
    base = O.render(sc, cam).blend.out
    perm = sc.subset(sc.n)
    perm.idx = perm.idx[:, :, ::-1].copy()
    perm.weights = perm.weights[:, :, ::-1].copy()
    np.testing.assert_allclose(O.render(perm, cam).blend.out, base, rtol=0, atol=1e-15)
    dup = sc.subset(sc.n)
    dup.idx[:, 0, 1] = dup.idx[:, 0, 0]
    merged = sc.subset(sc.n)
    merged.weights[:, 0, 0] = dup.weights[:, 0, 0].astype(np.float64) + dup.weights[:, 0, 1]
    merged.weights[:, 0, 1] = 0.0
    a, b = O.render(dup, cam).blend.out, O.render(merged, cam).blend.out
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-7)


def test_linearity_eq7():
    """Eq. 6 = Eq. 7: splatting f_i = w_i S directly equals decode(splat(W))."""
    sc, cam = syn.tiny()
    r = O.render(sc, cam)
    S = sc.codebook.astype(np.float64)
    feats = np.zeros((sc.n, 1, S.shape[2]))
    for k in range(4):
        feats[:, 0] += sc.weights[:, 0, k, None].astype(np.float64) * S[0, sc.idx[:, 0, k]]
    direct = O.blend(cam, r.proj, sc.opacity, r.ids, r.ranges, dense=feats, mode=2)
    via = O.decode(r.blend.out, sc.codebook)
    np.testing.assert_allclose(direct.out, via, rtol=0, atol=1e-13)


# ----------------------------------------------------------------------------- decode, relevancy

def test_decode_is_matmul():
    rng = np.random.default_rng(3)
    W = rng.random((2, 37, 64))
    S = rng.standard_normal((2, 64, 40)).astype(np.float32)
    bound = 1e-14 * np.matmul(np.abs(W), np.abs(S.astype(np.float64)))
    assert np.all(np.abs(O.decode(W, S) - np.matmul(W, S.astype(np.float64))) <= bound)


def test_relevancy_special_cases():
    tau = 10.0
    rng = np.random.default_rng(4)
    D = 512
    t = syn.unit_rows(rng.standard_normal((1, 5, D)))
    # negatives orthogonal to the positive
    for k in range(1, 5):
        t[0, k] -= t[0, 0] * (t[0, k] @ t[0, 0])
    t = syn.unit_rows(t).astype(np.float32)
    F = np.stack([3.0 * t[0, 0].astype(np.float64), np.zeros(D)])[None]
    rel = O.relevancy(F, t, tau)
    assert rel[0, 0, 0] == pytest.approx(math.exp(tau) / (math.exp(tau) + 1.0), abs=1e-6)
    assert rel[0, 0, 1] == 0.5
    # positive equal to one negative: that pairwise term is 1/2, so the min is <= 1/2
    t2 = t.copy()
    t2[0, 3] = t2[0, 0]
    G = rng.standard_normal((1, 7, D))
    assert np.all(O.relevancy(G, t2, tau)[0, 0] <= 0.5 + 1e-12)
    # with the positive equal to a negative, the pairwise term for it is exactly 1/2
    t3 = np.stack([t[0, 0], t[0, 0]])[None].astype(np.float32)
    np.testing.assert_allclose(O.relevancy(G, t3, tau)[0, 0], 0.5, atol=1e-12)


def test_relevancy_min_over_negatives_and_scale():
    """Monotone in the largest negative cosine; invariant to scaling F and t."""
    rng = np.random.default_rng(5)
    D = 64
    F = rng.standard_normal((1, 20, D))
    t = syn.unit_rows(rng.standard_normal((2, 5, D))).astype(np.float32)
    rel = O.relevancy(F, t, 10.0)
    np.testing.assert_allclose(O.relevancy(7.5 * F, t, 10.0), rel, rtol=1e-12)
    Fn = F / np.linalg.norm(F, axis=-1, keepdims=True)
    td = t.astype(np.float64)
    td = td / np.linalg.norm(td, axis=-1, keepdims=True)
    for q in range(2):
        c = Fn[0] @ td[q].T
        worst = c[:, 1:].max(1)
        expect = 1.0 / (1.0 + np.exp(-10.0 * (c[:, 0] - worst)))
        np.testing.assert_allclose(rel[q, 0], expect, rtol=1e-10)


# ----------------------------------------------------------------------------- gradients

def test_projection_jacobian_complex_step_vs_fd():
    sc, cam = syn.fd_subset()
    pr = O.project(cam, sc.means, sc.scales, sc.quats)
    gs = np.nonzero(pr.visible)[0][:25]
    m, s, q = (sc.means[gs].astype(np.float64), sc.scales[gs].astype(np.float64),
               sc.quats[gs].astype(np.float64))
    jac = O.project_jacobian(cam, m, s, q)
    x = np.concatenate([m, s, q], 1)
    for p in range(10):
        h = 1e-6 * max(1e-3, float(np.abs(x[:, p]).mean()))
        xp, xm = x.copy(), x.copy()
        xp[:, p] += h
        xm[:, p] -= h
        a = np.concatenate(O.project64(cam, xp[:, :3], xp[:, 3:6], xp[:, 6:]), 1)
        b = np.concatenate(O.project64(cam, xm[:, :3], xm[:, 3:6], xm[:, 6:]), 1)
        fd = (a - b) / (2 * h)
        scale = np.abs(jac[:, :, p]).max() + 1e-12
        np.testing.assert_allclose(jac[:, :, p], fd, rtol=0, atol=2e-5 * scale)


def _fd_problem(D=32):
    sc, cam = syn.fd_subset()
    sc.codebook = syn.codebooks(77, 1, 64, D)
    rng = np.random.default_rng(9)
    target = rng.normal(0, 0.05, (1, cam.num_pixels, D)).astype(np.float32)
    return sc, cam, target


def test_l1_gradient_matches_central_fd():
    """FP64 central differences (h = 1e-6) of the L1 feature loss vs the analytic oracle
    gradient, on the 200-Gaussian 64x48 subset; differences that cross a branch (contributor
    set, clamp, termination, L1 sign) are detected by signature and left out."""
    sc, cam, target = _fd_problem()
    g = O.l1_grads(sc, cam, target)
    pr = O.project(cam, sc.means, sc.scales, sc.quats)
    ids, ranges = O.bin(cam, pr)
    denom = float(cam.num_pixels * sc.codebook.shape[2])
    params = [sc.means.astype(np.float64), sc.scales.astype(np.float64),
              sc.quats.astype(np.float64), sc.opacity.astype(np.float64),
              sc.weights.astype(np.float64)]
    analytic = [g.dmeans, g.dscales, g.dquats, g.dopacity, g.dw]
    rng = np.random.default_rng(11)
    vis = np.nonzero(pr.visible)[0]
    chosen = rng.choice(vis, 10, replace=False)
    GX = cam.grid[0]
    checked = skipped = 0
    for gid in chosen:
        mask = np.zeros(cam.num_tiles, np.uint8)
        for ty in range(pr.rect[gid, 1], pr.rect[gid, 3]):
            for tx in range(pr.rect[gid, 0], pr.rect[gid, 2]):
                mask[ty * GX + tx] = 1
        _, sig0 = O.l1_loss_fd_eval(params, cam, ids, ranges, mask, sc.idx, sc.codebook, target)
        for a, (arr, an) in enumerate(zip(params, analytic)):
            nparam = arr.reshape(arr.shape[0], -1).shape[1]
            for j in range(nparam):
                h = 1e-6
                vals = []
                sigs = []
                for sgn in (+1, -1):
                    pp = [x.copy() for x in params]
                    pp[a].reshape(pp[a].shape[0], -1)[gid, j] += sgn * h
                    v, sg = O.l1_loss_fd_eval(pp, cam, ids, ranges, mask, sc.idx, sc.codebook, target)
                    vals.append(v)
                    sigs.append(sg)
                if sigs[0] != sig0 or sigs[1] != sig0:
                    skipped += 1
                    continue
                fd = (vals[0] - vals[1]).sum() / (2 * h) / denom
                ana = an.reshape(an.shape[0], -1)[gid, j]
                assert abs(fd - ana) <= 1e-6 * abs(ana) + 1e-9 / denom, (a, j, fd, ana)
                checked += 1
    assert checked >= 100 and skipped <= checked // 4


def test_decode_adjoint_fd():
    """dS = W^T G_F: finite differences of the loss in a few codebook entries."""
    sc, cam, target = _fd_problem(D=16)
    g = O.l1_grads(sc, cam, target)
    W = O.render(sc, cam).blend.out
    S = sc.codebook.astype(np.float64)

    def loss_terms(Sx):
        return np.abs(np.einsum("lpj,ljd->lpd", W, Sx) - target)
    rng = np.random.default_rng(2)
    for _ in range(12):
        j, d = rng.integers(64), rng.integers(16)
        h = 1e-7
        Sp, Sm = S.copy(), S.copy()
        Sp[0, j, d] += h
        Sm[0, j, d] -= h
        fd = (loss_terms(Sp) - loss_terms(Sm)).sum() / (2 * h) / W.shape[1] / 16
        assert fd == pytest.approx(g.dS[0, j, d], rel=1e-5, abs=1e-12)


# ----------------------------------------------------------------------------- post-processing

@pytest.mark.parametrize("k,H,W", [(1, 7, 9), (3, 13, 11), (7, 20, 17), (15, 9, 33)])
def test_mean_filter_is_border_normalised_uniform_filter(k, H, W):
    """Avg(M) (appendix "Evaluation Details") = scipy's zero-padded k x k mean divided by the same
    mean of an all-ones image: the mean over the in-image part of the window."""
    ndimage = pytest.importorskip("scipy.ndimage")
    M = np.random.default_rng(k * 100 + H).random((H, W))
    ref = (ndimage.uniform_filter(M, size=k, mode="constant", cval=0.0)
           / ndimage.uniform_filter(np.ones((H, W)), size=k, mode="constant", cval=0.0))
    assert np.allclose(O.mean_filter(M, k), ref, rtol=1e-12, atol=1e-14)


def test_mean_filter_of_a_ramp_closed_form():
    """A linear ramp M(x, y) = a x + b y + c: the mean over the clipped window [x0, x1] x [y0, y1]
    is a (x0 + x1)/2 + b (y0 + y1)/2 + c, so it stays a x + b y + c away from the border and is
    pulled inwards by the clipping at the border."""
    H, W, k = 10, 14, 5
    r = (k - 1) // 2
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    a, b, c = 0.25, -0.5, 3.0
    out = O.mean_filter(a * x + b * y + c, k)
    x0, x1 = np.maximum(x - r, 0), np.minimum(x + r, W - 1)
    y0, y1 = np.maximum(y - r, 0), np.minimum(y + r, H - 1)
    assert np.allclose(out, a * (x0 + x1) / 2 + b * (y0 + y1) / 2 + c, atol=1e-12)
    inner = (slice(r, H - r), slice(r, W - r))
    assert np.allclose(out[inner], (a * x + b * y + c)[inner], atol=1e-12)


def test_mean_filter_impulse():
    """One impulse of height 1: every pixel within the window's reach gets 1 / (its window's
    in-image pixel count); the corner pixel (0, 0) of a 3 x 3 window sees 4 pixels."""
    M = np.zeros((6, 6))
    M[0, 0] = 1.0
    out = O.mean_filter(M, 3)
    assert out[0, 0] == pytest.approx(1 / 4)
    assert out[1, 1] == pytest.approx(1 / 9)
    assert out[0, 1] == pytest.approx(1 / 6)
    assert out[2, 2] == 0.0


def test_postprocess_ramp_mask_and_point_closed_form():
    """k = 1 (no smoothing) on a ramp M = x / (W - 1) in every row: the normalised map is the
    ramp itself, the mask is the columns with x / (W - 1) > thr, and the point is the first
    pixel of the last column (row 0)."""
    H, W, thr = 5, 21, 0.3
    ramp = np.tile(np.arange(W) / (W - 1), (H, 1)).reshape(1, 1, -1)
    r = O.postprocess(ramp, H, W, k=1, mode=0, thr=thr)
    assert tuple(r.point[0]) == (W - 1, 0) and r.level[0] == 0 and r.score[0] == 1.0
    cols = np.arange(W) / (W - 1) > thr
    assert np.array_equal(r.mask[0].reshape(H, W), np.tile(cols, (H, 1)).astype(np.uint8))
    assert r.mask[0].sum() == H * int(np.sum(cols))


def _blob(H, W, cx, cy, sigma, peak, base):
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    return base + (peak - base) * np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / (2 * sigma ** 2))


def test_postprocess_level_rules_differ_as_the_appendix_says():
    """LERF picks the level with the highest relevancy value; 3D-OVS / Mip-NeRF360 pick the level
    with the highest mean inside its own mask.  Level 0 has a tall single-pixel spike (0.9) on a
    broad plateau (0.6 over most of the image), level 1 a broad blob up to 0.8 on 0.1: LERF
    takes level 0 (0.9 > 0.8); the mask rule takes level 1 (its masked mean ~0.7 > level 0's,
    whose mask is the plateau at ~0.6).  With k = 1 both modes see S = M."""
    H, W = 24, 32
    lev0 = np.full((H, W), 0.6)
    lev0[:, :4] = 0.0
    lev0[5, 20] = 0.9
    lev1 = _blob(H, W, 10.0, 12.0, 4.0, 0.8, 0.1)
    rel = np.stack([lev0.reshape(-1), lev1.reshape(-1)])[None]
    lerf = O.postprocess(rel, H, W, k=1, mode=0, thr=0.5)
    assert lerf.level[0] == 0 and tuple(lerf.point[0]) == (20, 5) and lerf.score[0] == 0.9
    ovs = O.postprocess(rel, H, W, k=1, mode=1, thr=0.5)
    assert ovs.level[0] == 1 and tuple(ovs.point[0]) == (10, 12)
    m1 = lev1 > 0.1 + 0.5 * (0.8 - 0.1)
    assert np.array_equal(ovs.mask[0].reshape(H, W), m1.astype(np.uint8))
    # mode 1 smooths as 0.5 (M + Avg(M)): with k = 3 the spike drops to 0.5 (0.9 + mean)
    ovs3 = O.postprocess(rel, H, W, k=3, mode=1, thr=0.5)
    spike_avg = (0.9 + 8 * 0.6) / 9
    assert ovs3.smoothed[0, 0, 5 * W + 20] == pytest.approx(0.5 * (0.9 + spike_avg))


def test_postprocess_ties_take_lowest_level_and_first_pixel():
    """Two levels with identical maps and two equal maxima: level 0 and the first maximum in
    row-major order; an exactly constant map normalises to 0 everywhere (empty mask).  (Smoothing
    a constant map can leave one-ulp differences, which min-max normalisation then amplifies, so
    the constant case is taken unsmoothed.)"""
    H, W = 6, 8
    M = np.zeros((H, W))
    M[4, 1] = M[2, 6] = 1.0
    rel = np.stack([M.reshape(-1)] * 2)[None]
    r = O.postprocess(rel, H, W, k=1, mode=0, thr=0.5)
    assert r.level[0] == 0 and tuple(r.point[0]) == (6, 2)
    flat = O.postprocess(np.full((1, 1, H * W), 0.7), H, W, k=1, mode=0, thr=0.5)
    assert flat.mask.sum() == 0 and flat.score[0] == pytest.approx(0.7)


# ---- Sec. 3.3 sparse coefficients (softmax, top K, renormalisation) and their gradient ----

def test_sparsify_closed_form():
    """Logits log(p) for p = (0.05, 0.4, 0.1, 0.3, 0.15): softmax = p; top 2 = entries 1, 3;
    renormalised 0.4 / 0.7, 0.3 / 0.7.  Top 3 adds entry 4: 0.4 / 0.85, 0.3 / 0.85, 0.15 / 0.85."""
    p = np.array([0.05, 0.4, 0.1, 0.3, 0.15])
    z = np.log(p).astype(np.float32)
    idx, w = O.sparsify(z, 2)
    assert idx.tolist() == [1, 3]
    np.testing.assert_allclose(w, [0.4 / 0.7, 0.3 / 0.7], rtol=1e-6)
    idx, w = O.sparsify(z, 3)
    assert idx.tolist() == [1, 3, 4]
    np.testing.assert_allclose(w, np.array([0.4, 0.3, 0.15]) / 0.85, rtol=1e-6)


def test_sparsify_all_kept_is_the_softmax():
    """K = L keeps everything: the weights are scipy's softmax of the logits, in descending order."""
    from scipy.special import softmax
    rng = np.random.default_rng(3)
    z = rng.normal(0, 2, (50, 64)).astype(np.float32)
    idx, w = O.sparsify(z, 64)
    ref = softmax(z.astype(np.float64), axis=1)
    np.testing.assert_allclose(w, np.take_along_axis(ref, idx.astype(np.int64), axis=1), rtol=1e-12)
    assert np.all(np.diff(w, axis=1) <= 0)


def test_sparsify_shift_invariance_and_unit_sum():
    """Logits on a 1/1024 grid, so that adding 8 is exact in float32 (ties included)."""
    rng = np.random.default_rng(4)
    z = (rng.integers(-4096, 4096, (200, 64)) / 1024.0).astype(np.float32)
    idx, w = O.sparsify(z, 4)
    np.testing.assert_allclose(w.sum(axis=1), 1.0, rtol=1e-12)
    idx2, w2 = O.sparsify(z + np.float32(8.0), 4)
    assert np.array_equal(idx, idx2)
    np.testing.assert_allclose(w, w2, rtol=1e-12)
    # the kept logits are the K largest
    zs = np.sort(z, axis=1)[:, ::-1]
    np.testing.assert_array_equal(np.take_along_axis(z, idx.astype(np.int64), axis=1), zs[:, :4])


def test_sparsify_ties_take_the_lower_index():
    z = np.array([0.5, 2.0, 2.0, 0.5, 2.0, 1.0], np.float32)
    idx, w = O.sparsify(z, 2)
    assert idx.tolist() == [1, 2]
    np.testing.assert_allclose(w, [0.5, 0.5], rtol=1e-15)
    idx, _ = O.sparsify(np.zeros(8, np.float32), 3)
    assert idx.tolist() == [0, 1, 2]


def test_sparsify_backward_matches_central_fd():
    """d(sum_k dw_k w_k)/dz by FP64 central differences (step 1e-6) of the forward, on logits whose
    top K is separated from the rest by a margin (the selection does not change under the step)."""
    rng = np.random.default_rng(5)
    L, K = 16, 4
    for _ in range(10):
        z = rng.normal(0, 1, L)
        z[rng.choice(L, K, replace=False)] += 3.0
        dw = rng.normal(0, 1, K)
        idx, w = O.sparsify(z.astype(np.float32), K)
        g = O.sparsify_backward(idx, w, dw, L)

        def f(zz):
            zz = zz.astype(np.float64)
            p = np.exp(zz - zz.max())
            p /= p.sum()
            pk = p[idx.astype(np.int64)]
            return float((dw * pk / pk.sum()).sum())

        zd = z.astype(np.float32).astype(np.float64)
        fd = np.zeros(L)
        for j in range(L):
            e = np.zeros(L)
            e[j] = 1e-6
            fd[j] = (f(zd + e) - f(zd - e)) / 2e-6
        np.testing.assert_allclose(g, fd, atol=1e-8)


def test_sparsify_backward_invariants():
    """Zero outside the kept entries; the gradient sums to zero (the weights sum to one)."""
    rng = np.random.default_rng(6)
    z = rng.normal(0, 1, (100, 64)).astype(np.float32)
    idx, w = O.sparsify(z, 4)
    dw = rng.normal(0, 1, (100, 4))
    g = O.sparsify_backward(idx, w, dw, 64)
    mask = np.zeros((100, 64), bool)
    np.put_along_axis(mask, idx.astype(np.int64), True, axis=1)
    assert np.all(g[~mask] == 0)
    np.testing.assert_allclose(g.sum(axis=1), 0.0, atol=1e-14)
    # top 1: the weight is 1 and the gradient vanishes
    idx1, w1 = O.sparsify(z, 1)
    assert np.all(w1 == 1.0)
    assert np.all(O.sparsify_backward(idx1, w1, dw[:, :1], 64) == 0)


# ----------------------------------------------------------------------------- decoder-based path

def test_mlp_decode_worked_example():
    """A two-layer g_d evaluated by hand.  x = (1, -2): the hidden pre-activation is
    x W1 + b1 = (1 + 2 + 0.5, -2 + 0, 2 + 0 - 3) = (3.5, -2, -1), ReLU keeps (3.5, 0, 0), and the
    output is 3.5 * 2 - 1 = 6.  x = (-1, 0): pre-activation (-0.5, 0, -5), all cut by the ReLU, so
    the output is the last bias, -1 (negative: no ReLU after the last layer)."""
    W1 = np.array([[1.0, 0.0, 2.0], [-1.0, 1.0, 0.0]])
    b1 = np.array([0.5, 0.0, -3.0])
    W2 = np.array([[2.0], [5.0], [7.0]])
    b2 = np.array([-1.0])
    y = O.mlp_decode(np.array([[1.0, -2.0], [-1.0, 0.0]]), [(W1, b1), (W2, b2)])
    assert y.shape == (2, 1)
    assert y[0, 0] == 6.0 and y[1, 0] == -1.0


def test_mlp_decode_relu_identity_and_homogeneity():
    """With zero biases a ReLU network is positively homogeneous, f(c x) = c f(x) for c > 0, and
    for one hidden layer relu(a) - relu(-a) = a gives f(x) - f(-x) = x W1 W2 (a missing ReLU would
    give twice that; a ReLU after the last layer would make every output nonnegative)."""
    rng = np.random.default_rng(11)
    W1, W2 = rng.standard_normal((3, 16)), rng.standard_normal((16, 5))
    z1, z2 = np.zeros(16), np.zeros(5)
    x = rng.standard_normal((50, 3))
    f = O.mlp_decode(x, [(W1, z1), (W2, z2)])
    fm = O.mlp_decode(-x, [(W1, z1), (W2, z2)])
    np.testing.assert_allclose(f - fm, x @ W1 @ W2, rtol=0, atol=1e-12)
    assert (f < 0).any()
    layers = [(l[0], np.zeros_like(l[1])) for l in syn.decoder_mlp()]
    np.testing.assert_allclose(O.mlp_decode(2.5 * x, layers), 2.5 * O.mlp_decode(x, layers), rtol=1e-12, atol=1e-12)


def test_mlp_decode_identity_layers():
    """Identity weights and zero biases: the hidden ReLUs clamp negatives to zero and the last
    layer passes its input through, so g_d(x) = relu(x); a bias shifts the output by exactly b."""
    x = np.array([[1.5, -2.0, 0.25], [-0.5, 3.0, -1.0]])
    eye, z = np.eye(3), np.zeros(3)
    np.testing.assert_array_equal(O.mlp_decode(x, [(eye, z), (eye, z), (eye, z)]), np.maximum(x, 0.0))
    b = np.array([0.5, -1.0, 2.0])
    np.testing.assert_array_equal(O.mlp_decode(x, [(eye, z), (eye, b)]), np.maximum(x, 0.0) + b)


def test_latent_render_as_pairs():
    """Eq. 4 with a d = 3 latent per Gaussian (blend mode 2) equals the sparse blend of the pairs
    (index k, weight f_k) for k < 3 plus (3, 0) over an 8-column map: channels 0..2 carry the
    latent render, channels 3..7 stay exactly zero."""
    sc, cam = syn.tiny()
    r = O.render(sc, cam)
    lat = syn.latent_features(sc.n, 1)
    direct = O.blend(cam, r.proj, sc.opacity, r.ids, r.ranges, dense=lat.astype(np.float64), mode=2)
    idx = np.broadcast_to(np.arange(4, dtype=np.uint8), (sc.n, 1, 4)).copy()
    w = np.concatenate([lat, np.zeros((sc.n, 1, 1), np.float32)], axis=2)
    pairs = O.blend(cam, r.proj, sc.opacity, r.ids, r.ranges, idx=idx, w=w, C_out=8)
    np.testing.assert_allclose(pairs.out[:, :, :3], direct.out, rtol=0, atol=1e-14)
    assert np.all(pairs.out[:, :, 3:] == 0.0)
    assert np.abs(direct.out).max() > 0.1
