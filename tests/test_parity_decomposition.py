"""The identity behind a coarse-grid form of an up-sampling decoder level
(Sec. 3.5: bilinear x2 up-sampling, then a 3x3 convolution): away from the
image border, a 3x3 convolution of the x2 up-sampled input equals four 3x3
convolutions of the coarse input, one per output parity (a, b), with effective
weights

    W_eff[a][b][o][c][dy][dx] = sum_{ky,kx} W[o][c][ky][kx] q(a, ky, dy) q(b, kx, dx)

where q(a, k, d) is the bilinear weight of coarse index i + d - 1 in fine index
2i + a + k - 1.  Checked against the oracle's own operators; the border ring
(2 fine pixels wide), where the up-sampling clamps and the convolution
zero-pads, is where the identity does not hold."""
import numpy as np

from oracle import network as N


def q(a, k, d):
    """Weight of coarse offset d - 1 in fine index 2i + a + k - 1 (half-pixel centres)."""
    m, par = divmod(a + k - 1, 2)  # fine index = 2 (i + m) + par
    taps = {m - 1: 0.25, m: 0.75} if par == 0 else {m: 0.75, m + 1: 0.25}
    return taps.get(d - 1, 0.0)


def effective_weights(W):
    E = np.zeros((2, 2) + W.shape)
    for a in range(2):
        for b in range(2):
            for dy in range(3):
                for dx in range(3):
                    for ky in range(3):
                        for kx in range(3):
                            E[a, b, :, :, dy, dx] += W[:, :, ky, kx] * q(a, ky, dy) * q(b, kx, dx)
    return E


def parity_form(x, W, bias):
    C, h, w = x.shape
    E = effective_weights(W)
    y = np.zeros((W.shape[0], 2 * h, 2 * w))
    for a in range(2):
        for b in range(2):
            y[:, a::2, b::2] = N.conv2d(x, E[a, b], bias)
    return y


def test_coefficients_partition_unity():
    # every fine index is a convex combination of two coarse neighbours
    for a in range(2):
        for k in range(3):
            w = [q(a, k, d) for d in range(3)]
            assert sum(w) == 1.0 and sorted(w) == [0.0, 0.25, 0.75]


def test_interior_equals_upsample_then_conv():
    rng = np.random.default_rng(5)
    for (c, o, h, w) in ((16, 16, 9, 13), (32, 32, 6, 7)):
        x = rng.standard_normal((c, h, w))
        W = rng.standard_normal((o, c, 3, 3))
        bias = rng.standard_normal(o)
        ref = N.conv2d(N.upsample2(x), W, bias)
        got = parity_form(x, W, bias)
        np.testing.assert_allclose(got[:, 2:-2, 2:-2], ref[:, 2:-2, 2:-2], rtol=1e-12, atol=1e-12)


def test_border_ring_differs():
    rng = np.random.default_rng(6)
    x = rng.standard_normal((4, 6, 8))
    W = rng.standard_normal((4, 4, 3, 3))
    bias = np.zeros(4)
    d = np.abs(parity_form(x, W, bias) - N.conv2d(N.upsample2(x), W, bias))
    assert d[:, 2:-2, 2:-2].max() < 1e-12
    ring = np.ones(d.shape[1:], bool)
    ring[2:-2, 2:-2] = False
    assert d[:, ring].max() > 1e-3  # the ring needs the exact path


def parity_form_replicate(x, W, bias):
    """The parity form over the coarse input extended by edge replication (one
    coarse pixel each side) instead of zeros: the form the level-0 decoder
    kernels evaluate."""
    E = effective_weights(W)
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1)), mode="edge")
    C, h, w = x.shape
    y = np.zeros((W.shape[0], 2 * h, 2 * w))
    for a in range(2):
        for b in range(2):
            y[:, a::2, b::2] = N.conv2d(xp, E[a, b], bias)[:, 1:-1, 1:-1]
    return y


def test_replicate_extension_leaves_a_one_pixel_ring():
    """With the coarse input extended by replication, the up-sampled input is
    reproduced exactly on every fine row and column of the image (the clamp of
    the bilinear taps), and also one step outside it, where the convolution
    reads zeros instead: only the outermost fine ring differs."""
    rng = np.random.default_rng(7)
    for (c, o, h, w) in ((16, 16, 9, 13), (4, 4, 6, 8), (16, 16, 2, 3)):
        x = rng.standard_normal((c, h, w))
        W = rng.standard_normal((o, c, 3, 3))
        bias = rng.standard_normal(o)
        ref = N.conv2d(N.upsample2(x), W, bias)
        got = parity_form_replicate(x, W, bias)
        np.testing.assert_allclose(got[:, 1:-1, 1:-1], ref[:, 1:-1, 1:-1], rtol=1e-12, atol=1e-12)
        ring = np.ones(got.shape[1:], bool)
        ring[1:-1, 1:-1] = False
        assert np.abs(got - ref)[:, ring].max() > 1e-3


def test_ring_correction_by_the_taps_outside():
    """On the ring, the replicate form minus the exact value is the sum of the
    taps that fall outside the fine image, each applied to the up-sampled
    input at the clamped position."""
    rng = np.random.default_rng(8)
    c, o, h, w = 3, 2, 4, 5
    x = rng.standard_normal((c, h, w))
    W = rng.standard_normal((o, c, 3, 3))
    U = N.upsample2(x)
    H2, W2 = 2 * h, 2 * w
    diff = parity_form_replicate(x, W, np.zeros(o)) - N.conv2d(U, W, np.zeros(o))
    for fy in range(H2):
        for fx in range(W2):
            corr = np.zeros(o)
            for ky in range(3):
                for kx in range(3):
                    y, xx = fy + ky - 1, fx + kx - 1
                    if 0 <= y < H2 and 0 <= xx < W2:
                        continue
                    u = U[:, min(max(y, 0), H2 - 1), min(max(xx, 0), W2 - 1)]
                    corr += W[:, :, ky, kx] @ u
            np.testing.assert_allclose(diff[:, fy, fx], corr, rtol=1e-12, atol=1e-12)


def test_oracle_effective_weights_and_coarse_model():
    """The oracle's own statement of the effective weights equals this file's;
    its coarse-grid level-0 decoder with no rounding equals the plain forward
    on a rendered frame (interior by the identity, ring by the exact path)."""
    import scenegen
    from oracle import gather as G
    rng = np.random.default_rng(9)
    W = rng.standard_normal((16, 16, 3, 3))
    np.testing.assert_allclose(N.upsample_conv_weights(W), effective_weights(W), rtol=0, atol=1e-13)
    f = scenegen.soft_frame(36, 52, 128, 128, 6, 3)
    feat, _, _ = G.features(f.pos4, f.nrm4, f.sm, f.view_proj, f.light_pos, f.cam_pos, f.r_hat, f.z_far, f.bias)
    th = scenegen.trained_weights().astype(np.float64)
    ref = N.forward(feat, th)
    got = N.forward_rounded(feat, th, lambda x: x, coarse_dec0=True)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13)
