"""Pins for the oracle's network operators, architecture counts, adjoint,
Eq. 2 loss and Adam step."""
import json
import math
import os

import numpy as np
import pytest

from oracle import network as N

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_network_counts.json")))


def _conv_direct(x, W, b):
    """Seven nested loops: y[o,i,j] = b[o] + sum_c sum_u sum_v W[o,c,u,v] x[c, i+u-p, j+v-p]."""
    co, ci, k, _ = W.shape
    p = (k - 1) // 2
    C, H, Wd = x.shape
    y = np.zeros((co, H, Wd))
    for o in range(co):
        for i in range(H):
            for j in range(Wd):
                s = b[o]
                for c in range(ci):
                    for u in range(k):
                        for v in range(k):
                            ii, jj = i + u - p, j + v - p
                            if 0 <= ii < H and 0 <= jj < Wd:
                                s += W[o, c, u, v] * x[c, ii, jj]
                y[o, i, j] = s
    return y


@pytest.mark.parametrize("k", [1, 3])
def test_conv_matches_direct_summation(k):
    rng = np.random.default_rng(1)
    x = rng.standard_normal((3, 5, 7))
    W = rng.standard_normal((4, 3, k, k))
    b = rng.standard_normal(4)
    np.testing.assert_allclose(N.conv2d(x, W, b), _conv_direct(x, W, b), rtol=1e-13, atol=1e-13)


def test_conv_matches_asymmetric_kernel_orientation():
    """A single off-centre tap shifts the image: W[0,0,0,2] = 1 reads x[i-1, j+1]."""
    x = np.arange(20.0).reshape(1, 4, 5)
    W = np.zeros((1, 1, 3, 3))
    W[0, 0, 0, 2] = 1.0
    y = N.conv2d(x, W, np.zeros(1))
    assert y[0, 2, 1] == x[0, 1, 2]
    assert y[0, 0, 1] == 0.0 and y[0, 2, 4] == 0.0  # zero padding


def test_ops_match_torch_fp64():
    torch = pytest.importorskip("torch")
    F = torch.nn.functional
    rng = np.random.default_rng(2)
    x = rng.standard_normal((6, 8, 12))
    W = rng.standard_normal((5, 6, 3, 3))
    b = rng.standard_normal(5)
    ref = F.conv2d(torch.from_numpy(x)[None], torch.from_numpy(W), torch.from_numpy(b), padding=1)[0].numpy()
    np.testing.assert_allclose(N.conv2d(x, W, b), ref, rtol=1e-12, atol=1e-12)
    ref = F.avg_pool2d(torch.from_numpy(x)[None], 2)[0].numpy()
    np.testing.assert_allclose(N.avgpool2(x), ref, rtol=1e-14, atol=1e-14)
    ref = F.interpolate(torch.from_numpy(x)[None], scale_factor=2, mode="bilinear", align_corners=False)[0].numpy()
    np.testing.assert_allclose(N.upsample2(x), ref, rtol=1e-13, atol=1e-13)


def test_upsample_closed_form():
    x = np.array([[[0.0, 4.0], [8.0, 12.0]]])
    y = N.upsample2(x)
    # row 0 sits at source 0 (clamped), column 1 at source 0.25
    assert y[0, 0, 0] == 0.0
    assert y[0, 0, 1] == pytest.approx(1.0)
    # row 1, column 1 sit at source (0.25, 0.25): 0.75 (0.75*0 + 0.25*4) + 0.25 (0.75*8 + 0.25*12)
    assert y[0, 1, 1] == pytest.approx(3.0)
    assert y[0, 3, 3] == 12.0


@pytest.mark.parametrize("name", ["conv3", "conv1", "pool", "up"])
def test_adjoint_dot_product_identity(name):
    """<A x, y> = <x, A^T y> for every linear operator in the network."""
    rng = np.random.default_rng(3)
    x = rng.standard_normal((4, 6, 10))
    if name.startswith("conv"):
        k = 3 if name == "conv3" else 1
        W = rng.standard_normal((5, 4, k, k))
        Ax = N.conv2d(x, W, np.zeros(5))
        y = rng.standard_normal(Ax.shape)
        ATy, dW, db = N.conv2d_adjoint(y, x, W)
        # and the weight adjoint: <A_W x, y> is linear in W
        assert np.sum(Ax * y) == pytest.approx(np.sum(W * dW), rel=1e-12)
    elif name == "pool":
        Ax = N.avgpool2(x)
        y = rng.standard_normal(Ax.shape)
        ATy = N.avgpool2_adjoint(y)
    else:
        Ax = N.upsample2(x)
        y = rng.standard_normal(Ax.shape)
        ATy = N.upsample2_adjoint(y)
    assert np.sum(Ax * y) == pytest.approx(np.sum(x * ATy), rel=1e-12)


def test_architecture_counts_match_paper():
    t3 = N.layer_table(3)
    assert [n for (n, *_r) in t3] == ["enc0_3x3", "enc0_1x1", "enc1_3x3", "enc1_1x1", "bott_3x3",
                                     "bott_1x1", "dec1_3x3", "dec1_1x1", "dec0_3x3", "dec0_1x1", "head"]
    nc = GOLD["network_cost"]
    for lv in ("3", "5"):
        L = int(lv)
        assert sum(N.macs_per_pixel_by_level(L)) == nc[lv]["macs_per_pixel"]
        # printed to the last shown digit (653,648 is printed as 653.7K)
        assert abs(N.param_count(L) / 1000.0 - nc[lv]["params_thousands"]) <= (0.005 if L == 3 else 0.06)
    per = GOLD["params_per_level_5lvl_thousands"]["values"]
    gm = GOLD["gmac_per_level_5lvl_1024x2048"]
    npx = gm["height"] * gm["width"]
    macs = N.macs_per_pixel_by_level(5)
    for lvl in range(5):
        assert round(macs[lvl] * npx / 1e9, 2) == pytest.approx(gm["values"][lvl])
        params = macs[lvl] * 4 ** lvl
        assert round(params / 1000.0, 2) == pytest.approx(per[lvl], abs=0.051)
    # 5-level FP32 size ~ 2.5 MB (Sec. 3.5)
    assert round(N.param_count(5) * 4 / 2 ** 20, 1) == GOLD["fp32_size_mb"]["value"]


def _rand_theta(levels, seed=0, scale=1.0):
    rng = np.random.default_rng(seed)
    parts = []
    for (_, ci, co, k) in N.layer_table(levels):
        parts.append(rng.standard_normal(co * ci * k * k) * scale * math.sqrt(2.0 / (ci * k * k)))
        parts.append(rng.standard_normal(co) * 0.1)
    return np.concatenate(parts)


def test_forward_range_and_shapes():
    rng = np.random.default_rng(4)
    x = rng.standard_normal((4, 16, 24))
    th = _rand_theta(3)
    v, t = N.forward(x, th, keep=True)
    assert v.shape == (16, 24)
    assert ((v > 0) & (v < 1)).all()
    assert t["bott_in"].shape == (32, 4, 6)
    assert t["dec1_in"].shape == (32, 8, 12)
    # the skip is the level-1 encoder output, merged by a sum
    np.testing.assert_allclose(t["dec1_in"], N.upsample2(t["bott_out"]) + t["enc1_h1"])
    # level 0 has no skip
    np.testing.assert_allclose(t["dec0_in"], N.upsample2(t["dec1_out"]))


def test_backward_matches_central_finite_differences():
    """dL/dtheta against central differences (h = 1e-3, FP64) on a 32x32 crop,
    for the scalar L = <g, vis>; coordinates whose stencil crosses a ReLU kink
    are excluded by checking that the forward pattern does not change."""
    rng = np.random.default_rng(5)
    x = rng.standard_normal((4, 32, 32))
    th = _rand_theta(3, seed=6)
    g = rng.standard_normal((32, 32))
    v, t = N.forward(x, th, keep=True)
    grad, gfeat = N.backward(g, th, t)
    h = 1e-3
    idx = rng.choice(th.size, 60, replace=False)
    offs = np.cumsum([0] + [co * ci * k * k + co for (_, ci, co, k) in N.layer_table(3)])
    idx = np.concatenate([idx, offs[:-1], offs[1:] - 1])  # first weight and last bias of every layer

    def pattern(tt):
        return np.concatenate([(tt[k] > 0).ravel() for k in tt if k.endswith(("_a3", "_a1"))])

    checked = 0
    for i in idx:
        tp = th.copy(); tp[i] += h
        tm = th.copy(); tm[i] -= h
        vp, ttp = N.forward(x, tp, keep=True)
        vm, ttm = N.forward(x, tm, keep=True)
        if not (np.array_equal(pattern(ttp), pattern(t)) and np.array_equal(pattern(ttm), pattern(t))):
            continue
        fd = (np.sum(g * vp) - np.sum(g * vm)) / (2 * h)
        assert fd == pytest.approx(grad[i], rel=1e-6, abs=1e-9), i
        checked += 1
    assert checked >= 40
    # input gradient, a few coordinates
    for (c, yy, xx) in [(0, 3, 4), (1, 16, 16), (2, 31, 0), (3, 10, 29)]:
        xp = x.copy(); xp[c, yy, xx] += h
        xm = x.copy(); xm[c, yy, xx] -= h
        fd = (np.sum(g * N.forward(xp, th)) - np.sum(g * N.forward(xm, th))) / (2 * h)
        assert fd == pytest.approx(gfeat[c, yy, xx], rel=1e-5, abs=1e-9)


def test_loss_eq2_closed_form_and_gradient():
    x0 = np.array([[0.2, 0.5], [0.9, 0.4]])
    tgt = np.array([[0.0, 0.5], [1.0, 1.0]])
    x1 = np.array([[0.3, 0.5], [0.9, 0.1]])
    x2 = np.array([[0.1, 0.6], [0.8, 0.4]])
    loss, g = N.loss_l1(x0, tgt, [x1, x2], alpha=0.9)
    expect = 0.9 * (0.2 + 0 + 0.1 + 0.6) / 4 + 0.9 * (0.1 + 0 + 0 + 0.3) / 4 + 0.9 * (0.1 + 0.1 + 0.1 + 0) / 4
    assert loss == pytest.approx(expect, rel=1e-14)
    np.testing.assert_allclose(g, 0.9 / 4 * np.array([[1 - 1 + 1, 0 + 0 - 1], [-1 + 0 + 1, -1 + 1 + 0]]))
    assert GOLD["loss"]["alpha"] == 0.9


def test_adam_closed_form_first_steps():
    th = np.array([1.0, -2.0, 0.0])
    g = np.array([0.5, -0.1, 0.0])
    m = np.zeros(3); v = np.zeros(3)
    th1, m1, v1 = N.adam_update(th, g, m, v, 1, lr=0.01)
    # step 1: m_hat = g, v_hat = g^2 -> update = lr * sign(g) (up to eps)
    np.testing.assert_allclose(th1, th - 0.01 * np.array([1.0, -1.0, 0.0]), atol=1e-9)
    th2, m2, v2 = N.adam_update(th1, g, m1, v1, 2, lr=0.01)
    np.testing.assert_allclose(th2, th1 - 0.01 * np.array([1.0, -1.0, 0.0]), atol=1e-9)
    np.testing.assert_allclose(m2, 0.19 * g)


def test_train_step_gradient_is_loss_gradient():
    """The batch gradient equals central differences of the Eq. 2 loss
    (with the perturbed outputs x_i held fixed, as the stop-gradient says)."""
    rng = np.random.default_rng(8)
    B, T, H, W = 2, 3, 8, 8
    feats = [[rng.standard_normal((4, H, W)) for _ in range(T)] for _ in range(B)]
    tgts = [rng.uniform(0, 1, (H, W)) for _ in range(B)]
    th = _rand_theta(3, seed=9)
    _, _, _, loss, grad = N.train_step(feats, tgts, th, np.zeros_like(th), np.zeros_like(th), 1)
    xs = [[N.forward(f, th) for f in feats[b][1:]] for b in range(B)]

    def L(tt):
        tot = 0.0
        for b in range(B):
            tot += N.loss_l1(N.forward(feats[b][0], tt), tgts[b], xs[b])[0] / B
        return tot

    assert loss == pytest.approx(L(th), rel=1e-12)
    h = 1e-6
    for i in rng.choice(th.size, 12, replace=False):
        tp = th.copy(); tp[i] += h
        tm = th.copy(); tm[i] -= h
        fd = (L(tp) - L(tm)) / (2 * h)
        assert fd == pytest.approx(grad[i], rel=1e-4, abs=1e-9)


def test_round_bf16_definition():
    # exact values stay, halfway cases go to even, 8 significant bits survive
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -7, -3.140625, 0.0, 2.0 ** -130])
    r = N.round_bf16(x)
    assert list(r[:5]) == [1.0, 1.0, 1.0 + 2 ** -6, 1.0 + 2 ** -7, -3.140625]
    assert r[5] == 0.0 and r[6] == np.float32(2.0 ** -130)  # a binary32 subnormal with 7 mantissa bits fits
    rng = np.random.default_rng(11)
    y = rng.standard_normal(10000) * 100
    rel = np.abs(N.round_bf16(y) - y) / np.abs(y)
    assert rel.max() <= 2 ** -8
    torch = pytest.importorskip("torch")
    ref = torch.from_numpy(y.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(N.round_bf16(y), ref)
    # the hi + lo pair keeps about 16 bits
    assert (np.abs(N.round_bf16_pair(y) - y.astype(np.float32)) / np.abs(y)).max() <= 2 ** -15


def test_forward_rounded_identity_and_sensitivity():
    rng = np.random.default_rng(12)
    x = rng.standard_normal((4, 8, 12))
    th = _rand_theta(3, seed=13)
    ident = lambda a: np.asarray(a, np.float64)
    np.testing.assert_allclose(N.forward_rounded(x, th, ident), N.forward(x, th), rtol=1e-12, atol=1e-14)
    v = N.forward_rounded(x, th, N.round_bf16)
    d = np.abs(v - N.forward(x, th))
    assert 0 < d.max() < 0.05


# ------------------------------------------------------------------ E4M3 (FP8 form)
def _e4m3_decode(byte):
    """Value of an E4M3 byte from its bit fields (OCP 8-bit floating point,
    E4M3: bias 7, no infinities, S.1111.111 is NaN)."""
    s, e, m = (byte >> 7) & 1, (byte >> 3) & 0xF, byte & 7
    if e == 15 and m == 7:
        return float("nan")
    v = (m / 8.0) * 2.0 ** -6 if e == 0 else (1 + m / 8.0) * 2.0 ** (e - 7)
    return -v if s else v


def test_e4m3_value_set_matches_the_bit_fields():
    v = N.e4m3_values()
    assert v.size == 127 and v[0] == 0.0 and v[-1] == 448.0
    dec = sorted({_e4m3_decode(b) for b in range(128) if b != 0x7F})
    np.testing.assert_array_equal(v, np.array(dec))
    # a few codes of the format's table
    assert _e4m3_decode(0x38) == 1.0 and _e4m3_decode(0x7E) == 448.0 and _e4m3_decode(0x01) == 2.0 ** -9
    assert _e4m3_decode(0x08) == 2.0 ** -6 and _e4m3_decode(0xB8) == -1.0


def test_round_e4m3_is_nearest_with_ties_to_even_and_saturates():
    v = N.e4m3_values()
    full = np.concatenate([-v[::-1], v[1:]])
    rng = np.random.default_rng(8)
    x = np.concatenate([rng.normal(0, 10, 4000), rng.uniform(-2 ** -5, 2 ** -5, 2000), [500.0, -1e6, 448.0]])
    x = x.astype(np.float32).astype(np.float64)
    q = N.round_e4m3(x)
    xs = np.clip(x, -448.0, 448.0)
    # brute force: q is one of the nearest representable values
    d = np.abs(xs[:, None] - full[None, :])
    assert np.all(np.abs(xs - q) <= d.min(axis=1))
    # exact midpoints go to the even mantissa field
    for lo_i in range(1, v.size - 1):
        mid = 0.5 * (v[lo_i] + v[lo_i + 1])
        even = v[lo_i] if lo_i % 2 == 0 else v[lo_i + 1]
        if np.float32(mid) == mid:
            assert N.round_e4m3(np.array([mid]))[0] == even
    assert N.round_e4m3(np.array([1e9]))[0] == 448.0


def test_round_e4m3_per_out_channel_keeps_each_row_maximum():
    rng = np.random.default_rng(9)
    W = rng.normal(0, 0.3, (8, 5, 3, 3))
    Q = N.round_e4m3_per_out_channel(W)
    for o in range(8):
        i = np.argmax(np.abs(W[o]))
        assert abs(Q[o].flat[i] - W[o].flat[i]) <= 1e-12 * abs(W[o].flat[i])
        s = np.abs(W[o]).max() / 448.0
        big = np.abs(W[o]) >= 2 ** -6 * s  # normal range: relative error <= 2^-4
        assert np.all(np.abs(Q[o] - W[o])[big] <= 2 ** -4 * np.abs(W[o])[big] + 1e-15)


def test_round_e4m3_terms_pins():
    """The multi-term E4M3 split: one term is round_e4m3; an E4M3 value is
    reproduced exactly (later terms zero) and a value a quarter-ulp off one by
    its second term; otherwise the error of three terms is within half a unit of
    the third term's last place: 2^-12 of |x| in the normal range, plus 2^-18
    absolute where a residual falls into the subnormals (2^-10 / 256); values
    beyond 448 + 28 + 1.75 saturate there."""
    rng = np.random.default_rng(11)
    x = rng.standard_normal(5000) * 50.0
    np.testing.assert_array_equal(N.round_e4m3_terms(x, 1), N.round_e4m3(x))
    # an E4M3 value is its own first term, and the later terms are zero
    v = N.e4m3_values()
    vs = np.concatenate([v, -v])
    np.testing.assert_array_equal(N.round_e4m3_terms(vs, 3), vs)
    # a value one E4M3 ulp-quarter off a binade start needs the second term:
    # 1 + 2^-5 -> a_0 = 1, a_1 = e4m3(16 * 2^-5) / 16 = 2^-5 exactly
    assert N.round_e4m3(np.array([1.0 + 2.0 ** -5]))[0] == 1.0
    assert N.round_e4m3_terms(np.array([1.0 + 2.0 ** -5]), 2)[0] == 1.0 + 2.0 ** -5
    y = np.concatenate([rng.uniform(-400, 400, 20000), rng.uniform(-1e-2, 1e-2, 5000)])
    err = np.abs(N.round_e4m3_terms(y, 3) - y)
    assert np.all(err <= 2.0 ** -12 * np.abs(y) + 2.0 ** -18)
    assert N.round_e4m3_terms(np.array([1e4]), 3)[0] == 448.0 + 448.0 / 16.0 + 448.0 / 256.0
    # fewer terms are coarser: two terms leave up to 2^-8 of |x|
    e2 = np.abs(N.round_e4m3_terms(y, 2) - y)
    assert e2.max() > 16 * err.max()
    W = rng.standard_normal((8, 5, 3, 3))
    Q = N.round_e4m3_terms_per_out_channel(W, 3)
    assert np.all(np.abs(Q - W) <= 2.0 ** -12 * np.abs(W) + 2.0 ** -18 * np.abs(W).reshape(8, -1).max(1)[:, None, None, None] / 448)


def test_three_term_e4m3_network_meets_the_bar():
    """The trained 3-level network with every stored value (features, level
    outputs, 3x3 outputs, up-sampled inputs) and every weight in the
    three-term E4M3 form stays within 5e-3 max-abs / 1e-8 MSE of the FP64
    forward (under the 1e-2 / 1e-4 bar) on a 64-object frame, while one term
    per value does not meet the bar."""
    import scenegen
    from oracle import gather as G
    f = scenegen.soft_frame(96, 128, 512, 512, 64, 7)
    feat, _, _ = G.features(f.pos4, f.nrm4, f.sm, f.view_proj, f.light_pos, f.cam_pos, f.r_hat, f.z_far, f.bias)
    theta = scenegen.trained_weights().astype(np.float64)
    ref = N.forward(feat, theta)
    r3 = lambda x: N.round_e4m3_terms(x, 3)
    q3 = N.forward_rounded(feat, theta, r3, rnd_in=r3, rnd_w=N.round_e4m3_terms_per_out_channel, rnd_mid=r3)
    e3 = np.abs(q3 - ref)
    assert e3.max() <= 5e-3 and np.mean(e3 ** 2) <= 1e-8, (e3.max(), np.mean(e3 ** 2))
    q1 = N.forward_rounded(feat, theta, N.round_e4m3, rnd_in=N.round_e4m3, rnd_w=N.round_e4m3_per_out_channel,
                           rnd_mid=N.round_e4m3)
    assert np.abs(q1 - ref).max() > 1e-2


def test_band_forward_equals_the_full_frame():
    """bench.py measures errors on a band of rows with the oracle run on the
    band plus a 32-row margin: the receptive field of the 3-level net is about
    20 pixels, so the band rows equal the full-frame forward exactly."""
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    import scenegen
    from oracle import gather as G
    f = scenegen.soft_frame(192, 160, 256, 256, 10, 23)
    th = scenegen.he_init_weights(4, N.layer_table(3)).astype(np.float64)
    feat, _, _ = G.features(f.pos4, f.nrm4, f.sm, f.view_proj, f.light_pos, f.cam_pos, f.r_hat, f.z_far, f.bias)
    full = N.forward(feat, th)
    for y0, y1 in ((0, 40), (76, 100), (148, 192)):
        np.testing.assert_array_equal(bench.oracle_band(f, th, y0, y1), full[y0:y1])


# ------------------------------------------------------------------ space-to-depth topology
def _naive_conv(x, W, b):
    co, ci, k, _ = W.shape
    p = (k - 1) // 2
    C, H, Wd = x.shape
    y = np.zeros((co, H, Wd))
    for o in range(co):
        for i in range(H):
            for j in range(Wd):
                acc = b[o]
                for c in range(ci):
                    for u in range(k):
                        for v in range(k):
                            ii, jj = i + u - p, j + v - p
                            if 0 <= ii < H and 0 <= jj < Wd:
                                acc += W[o, c, u, v] * x[c, ii, jj]
                y[o, i, j] = acc
    return y


def _naive_up(x):
    # bilinear x2, half-pixel centres, edge clamp: source coordinate o / 2 - 1/4
    C, H, W = x.shape
    y = np.zeros((C, 2 * H, 2 * W))
    for c in range(C):
        for i in range(2 * H):
            for j in range(2 * W):
                sy, sx = i / 2 - 0.25, j / 2 - 0.25
                y0, x0 = int(np.floor(sy)), int(np.floor(sx))
                fy, fx = sy - y0, sx - x0
                cl = lambda v, n: min(max(v, 0), n - 1)
                a = x[c, cl(y0, H), cl(x0, W)] * (1 - fx) + x[c, cl(y0, H), cl(x0 + 1, W)] * fx
                b = x[c, cl(y0 + 1, H), cl(x0, W)] * (1 - fx) + x[c, cl(y0 + 1, H), cl(x0 + 1, W)] * fx
                y[c, i, j] = a * (1 - fy) + b * fy
    return y


def test_space_to_depth_index_map_and_inverse():
    rng = np.random.default_rng(31)
    x = rng.normal(size=(4, 6, 8))
    y = N.space_to_depth(x)
    assert y.shape == (16, 3, 4)
    for c in range(4):
        for i in range(6):
            for j in range(8):
                assert y[4 * (2 * (i % 2) + (j % 2)) + c, i // 2, j // 2] == x[c, i, j]


def test_s2d_output_places_details_and_upsamples_channel0():
    rng = np.random.default_rng(32)
    o = rng.normal(size=(4, 3, 5))
    z = o.copy()
    z[0] = 0
    d = N.s2d_output(z)
    assert np.all(d[0::2, 0::2] == 0)
    np.testing.assert_array_equal(d[0::2, 1::2], o[1])
    np.testing.assert_array_equal(d[1::2, 0::2], o[2])
    np.testing.assert_array_equal(d[1::2, 1::2], o[3])
    z = np.zeros_like(o)
    z[0] = o[0]
    np.testing.assert_allclose(N.s2d_output(z), _naive_up(o[0:1])[0], rtol=0, atol=1e-14)


def test_forward_s2d_matches_direct_summation_network():
    """forward_s2d against a network written out with direct-summation
    convolutions, explicit bilinear weights and loops (8 x 8 input)."""
    rng = np.random.default_rng(33)
    t = N.layer_table_s2d(3)
    n = sum(ci * co * k * k + co for (_, ci, co, k) in t)
    theta = rng.normal(0, 0.2, n)
    feat = rng.normal(0, 1, (4, 8, 8))
    P = N.unpack_s2d(theta)
    relu = lambda v: np.maximum(v, 0)
    x = np.zeros((16, 4, 4))
    for a in range(2):
        for b in range(2):
            for c in range(4):
                x[4 * (2 * a + b) + c] = feat[c, a::2, b::2]
    s1 = relu(_naive_conv(relu(_naive_conv(x, *P["enc1_3x3"])), *P["enc1_1x1"]))
    p1 = 0.25 * (s1[:, 0::2, 0::2] + s1[:, 0::2, 1::2] + s1[:, 1::2, 0::2] + s1[:, 1::2, 1::2])
    bo = relu(_naive_conv(relu(_naive_conv(p1, *P["bott_3x3"])), *P["bott_1x1"]))
    d1 = relu(_naive_conv(relu(_naive_conv(_naive_up(bo) + s1, *P["dec1_3x3"])), *P["dec1_1x1"]))
    o = _naive_conv(d1, *P["head"])
    pre = _naive_up(o[0:1])[0]
    for i in range(8):
        for j in range(8):
            a, b = i % 2, j % 2
            if (a, b) != (0, 0):
                pre[i, j] += o[2 * a + b, i // 2, j // 2]
    ref = 1 / (1 + np.exp(-pre))
    np.testing.assert_allclose(N.forward_s2d(feat, theta), ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("levels", [3, 4])
def test_forward_matches_direct_summation_network(levels):
    """forward against the Sec. 3.5 network written out level by level with
    direct-summation convolutions, explicit 2x2 means and the loop bilinear
    up-sampling (8 x 8 input: the 4-level bottleneck is 1 x 1): per encoder
    level 3x3, ReLU, 1x1, ReLU, the rectified output kept as the skip at
    levels 1 .. L-2, then the mean of each 2 x 2 block; the bottleneck; per
    decoder level up-sampling (plus the skip), 3x3, ReLU, 1x1, ReLU; the 16 -> 1
    head and the sigmoid."""
    rng = np.random.default_rng(40 + levels)
    n = N.param_count(levels, with_bias=True)
    theta = rng.normal(0, 0.25, n)
    feat = rng.normal(0, 1, (4, 8, 8))
    P = N.unpack(theta, levels)
    relu = lambda v: np.maximum(v, 0)

    def block(x, key):
        return relu(_naive_conv(relu(_naive_conv(x, *P[f"{key}_3x3"])), *P[f"{key}_1x1"]))

    def pool(x):
        C, H, W = x.shape
        y = np.zeros((C, H // 2, W // 2))
        for c in range(C):
            for i in range(H // 2):
                for j in range(W // 2):
                    y[c, i, j] = 0.25 * (x[c, 2 * i, 2 * j] + x[c, 2 * i, 2 * j + 1] + x[c, 2 * i + 1, 2 * j] +
                                         x[c, 2 * i + 1, 2 * j + 1])
        return y

    h, skips = feat, {}
    for l in range(levels - 1):
        h = block(h, f"enc{l}")
        if l >= 1:
            skips[l] = h
        h = pool(h)
    h = block(h, "bott")
    for l in range(levels - 2, -1, -1):
        x = _naive_up(h)
        if l >= 1:
            x = x + skips[l]
        h = block(x, f"dec{l}")
    ref = 1 / (1 + np.exp(-_naive_conv(h, *P["head"])[0]))
    np.testing.assert_allclose(N.forward(feat, theta, levels=levels), ref, rtol=0, atol=1e-12)


def test_forward_s2d_head_bias_closed_form():
    """Zero weights everywhere but the head biases: every output is the
    sigmoid of b0 plus the detail bias of its square offset."""
    t = N.layer_table_s2d(3)
    n = sum(ci * co * k * k + co for (_, ci, co, k) in t)
    theta = np.zeros(n)
    bias = np.array([0.3, -0.7, 1.1, 0.2])
    theta[-4:] = bias
    v = N.forward_s2d(np.ones((4, 12, 16)), theta)
    sig = lambda z: 1 / (1 + np.exp(-z))
    np.testing.assert_allclose(v[0::2, 0::2], sig(bias[0]), atol=1e-15)
    np.testing.assert_allclose(v[0::2, 1::2], sig(bias[0] + bias[1]), atol=1e-15)
    np.testing.assert_allclose(v[1::2, 0::2], sig(bias[0] + bias[2]), atol=1e-15)
    np.testing.assert_allclose(v[1::2, 1::2], sig(bias[0] + bias[3]), atol=1e-15)
    assert sum(ci * co * k * k for (_, ci, co, k) in t) == 35904  # 39,248 - level 0 - old head + 16x4 head


def test_trained_weights_input():
    """The committed trained weights (an input of the GPU tests and the
    benchmark): canonical size, finite, and on held-out scenes (seeds outside
    the training range) far closer to the ray-cast visibility than the He-init
    weights training started from."""
    import scenegen
    from oracle import gather as G
    th = scenegen.trained_weights().astype(np.float64)
    assert th.shape == (N.param_count(3, with_bias=True),) and np.isfinite(th).all()
    he = scenegen.he_init_weights(3, N.layer_table(3))
    for soft in (False, True):
        f = scenegen.render_frame(scenegen.random_scene(3000 + soft, 64, soft=soft), 128, 224, 512, 512)
        target = (scenegen.soft_visibility(f, spp_side=8) if soft else scenegen.hard_visibility(f)).astype(np.float64)
        feat, _, _ = G.features(f.pos4, f.nrm4, f.sm, f.view_proj, f.light_pos, f.cam_pos, f.r_hat, f.z_far, f.bias)
        mse_tr = np.mean((N.forward(feat, th) - target) ** 2)
        mse_he = np.mean((N.forward(feat, he) - target) ** 2)
        assert mse_tr < 0.25 * mse_he, (soft, mse_tr, mse_he)


def test_s2d_adjoint_operators_dot_product():
    """<A x, y> = <x, A^T y> for space_to_depth and s2d_output."""
    rng = np.random.default_rng(21)
    x = rng.standard_normal((4, 8, 12))
    y = rng.standard_normal((16, 4, 6))
    assert np.vdot(N.space_to_depth(x), y) == pytest.approx(np.vdot(x, N.space_to_depth_adjoint(y)), rel=1e-12)
    o = rng.standard_normal((4, 4, 6))
    g = rng.standard_normal((8, 12))
    assert np.vdot(N.s2d_output(o), g) == pytest.approx(np.vdot(o, N.s2d_output_adjoint(g)), rel=1e-12)


def test_s2d_backward_matches_central_finite_differences():
    """The space-to-depth network's adjoint against central differences
    (h = 1e-4, FP64: at 1e-3 the truncation error reaches ~2e-6 relative on
    some weights) on a 16 x 16 input, stencils crossing a ReLU kink excluded;
    weights and the input features."""
    rng = np.random.default_rng(22)
    x = rng.standard_normal((4, 16, 16))
    th = scenegen_s2d_theta(23)
    g = rng.standard_normal((16, 16))
    v, t = N.forward_s2d(x, th, keep=True)
    np.testing.assert_allclose(v, N.forward_s2d(x, th), rtol=0, atol=0)
    grad, gfeat = N.backward_s2d(g, th, t)
    h = 1e-4

    def pattern(tt):
        return np.concatenate([(tt[k] > 0).ravel() for k in tt if k.endswith(("_a3", "_a1"))])

    offs = np.cumsum([0] + [co * ci * k * k + co for (_, ci, co, k) in N.layer_table_s2d(3)])
    idx = np.concatenate([rng.choice(th.size, 60, replace=False), offs[:-1], offs[1:] - 1])
    checked = 0
    for i in idx:
        tp = th.copy(); tp[i] += h
        tm = th.copy(); tm[i] -= h
        vp, ttp = N.forward_s2d(x, tp, keep=True)
        vm, ttm = N.forward_s2d(x, tm, keep=True)
        if not (np.array_equal(pattern(ttp), pattern(t)) and np.array_equal(pattern(ttm), pattern(t))):
            continue
        fd = (np.sum(g * vp) - np.sum(g * vm)) / (2 * h)
        assert fd == pytest.approx(grad[i], rel=1e-6, abs=1e-9), i
        checked += 1
    assert checked >= 40
    for (c, yy, xx) in [(0, 3, 4), (2, 10, 7), (3, 15, 15), (1, 0, 0)]:
        xp = x.copy(); xp[c, yy, xx] += h
        xm = x.copy(); xm[c, yy, xx] -= h
        vp, ttp = N.forward_s2d(xp, th, keep=True)
        vm, ttm = N.forward_s2d(xm, th, keep=True)
        if np.array_equal(pattern(ttp), pattern(t)) and np.array_equal(pattern(ttm), pattern(t)):
            assert (np.sum(g * vp) - np.sum(g * vm)) / (2 * h) == pytest.approx(gfeat[c, yy, xx], rel=1e-6, abs=1e-9)


def test_s2d_train_step_matches_the_3level_form_of_its_parts():
    """train_step_s2d's loss and gradient are the Eq. 2 loss of forward_s2d and
    the adjoint above (composition check on a 2-item batch)."""
    rng = np.random.default_rng(24)
    feats = [[rng.standard_normal((4, 8, 8)) for _ in range(2)] for _ in range(2)]
    targets = [rng.random((8, 8)) for _ in range(2)]
    th = scenegen_s2d_theta(25)
    z = np.zeros_like(th)
    _, _, _, loss, grad = N.train_step_s2d(feats, targets, th, z, z, 1)
    ref_loss, ref_grad = 0.0, np.zeros_like(th)
    for b in range(2):
        x0, t = N.forward_s2d(feats[b][0], th, keep=True)
        l, g = N.loss_l1(x0, targets[b], [N.forward_s2d(feats[b][1], th)])
        ref_loss += l / 2
        ref_grad += N.backward_s2d(g / 2, th, t)[0]
    assert loss == pytest.approx(ref_loss, rel=1e-12)
    np.testing.assert_allclose(grad, ref_grad, rtol=1e-12, atol=1e-15)


def scenegen_s2d_theta(seed):
    import scenegen
    rng = np.random.default_rng(seed)
    parts = []
    for (_, ci, co, k) in N.layer_table_s2d(3):
        parts.append(rng.standard_normal(co * ci * k * k) * np.sqrt(2.0 / (ci * k * k)))
        parts.append(rng.standard_normal(co) * 0.05)
    del scenegen
    return np.concatenate(parts)


def test_trained_s2d_weights_input():
    """The committed trained weights of the space-to-depth network: canonical
    size, finite, and on held-out scenes far closer to the ray-cast visibility
    than the He-init weights training started from."""
    import scenegen
    from oracle import gather as G
    th = scenegen.trained_weights_s2d().astype(np.float64)
    assert th.shape == (sum(ci * co * k * k + co for (_, ci, co, k) in N.layer_table_s2d(3)),)
    assert np.isfinite(th).all()
    he = scenegen.he_init_weights(3, N.layer_table_s2d(3))
    for soft in (False, True):
        f = scenegen.render_frame(scenegen.random_scene(3000 + soft, 64, soft=soft), 128, 224, 512, 512)
        target = (scenegen.soft_visibility(f, spp_side=8) if soft else scenegen.hard_visibility(f)).astype(np.float64)
        feat, _, _ = G.features(f.pos4, f.nrm4, f.sm, f.view_proj, f.light_pos, f.cam_pos, f.r_hat, f.z_far, f.bias)
        mse_tr = np.mean((N.forward_s2d(feat, th) - target) ** 2)
        mse_he = np.mean((N.forward_s2d(feat, he) - target) ** 2)
        assert mse_tr < 0.25 * mse_he, (soft, mse_tr, mse_he)


def test_recompute_from_exact_checkpoints_is_forward():
    """With no rounding, the checkpoints of forward_rounded and the
    intermediates recomputed from them equal forward's, and the adjoint built
    on them equals backward on forward's intermediates."""
    rng = np.random.default_rng(11)
    x = rng.standard_normal((4, 16, 24))
    th = N.pack({n: (rng.standard_normal((co, ci, k, k)) * 0.3, rng.standard_normal(co) * 0.1)
                 for (n, ci, co, k) in N.layer_table(3)})
    ident = lambda a: a
    ck = {}
    vis = N.forward_rounded(x, th, ident, ckpt=ck)
    ref, t = N.forward(x, th, keep=True)
    np.testing.assert_allclose(vis, ref, rtol=0, atol=1e-14)
    t2 = N.recompute_from_checkpoints(x, ck, th)
    for k in ("enc0_a3", "enc1_in", "enc1_a1", "bott_in", "bott_a3", "dec1_in", "dec1_a1", "dec0_in", "dec0_a3",
              "dec0_out", "vis"):
        np.testing.assert_allclose(t2[k], t[k], rtol=0, atol=1e-12, err_msg=k)
    g = rng.standard_normal(vis.shape)
    np.testing.assert_allclose(N.backward(g, th, t2)[0], N.backward(g, th, t)[0], rtol=1e-12, atol=1e-13)
