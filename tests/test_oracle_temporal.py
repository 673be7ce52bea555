"""Pins of the temporal-instability metric (Sec. 3.4, Eq. 3) and the
penumbra-size depth rule (Sec. 3.6) of oracle/temporal.py."""
import math

import numpy as np
import pytest

import scenegen
from oracle import temporal as TM


def _cam(scene, H, W):
    return scenegen.camera_vector(scene, H, W)


def _pixel_rays(cam, H, W):
    """FP64 unit rays through the pixel centres of the pinhole camera (the
    construction the ray caster uses), (H, W, 3)."""
    C, f, r, u, th, asp = cam[0:3], cam[3:6], cam[6:9], cam[9:12], cam[12], cam[13]
    x = (2.0 * (np.arange(W) + 0.5) / W - 1.0) * th * asp
    y = (1.0 - 2.0 * (np.arange(H) + 0.5) / H) * th
    d = f[None, None, :] + x[None, :, None] * r[None, None, :] + y[:, None, None] * u[None, None, :]
    return d / np.linalg.norm(d, axis=-1, keepdims=True)


def test_reprojection_of_pixel_rays_is_the_pixel():
    scene = scenegen.random_scene(3, 8)
    H, W = 24, 40
    cam = _cam(scene, H, W)
    rays = _pixel_rays(cam, H, W)
    jj, ii = np.mgrid[0:H, 0:W]
    for t in (0.7, 2.5, 9.0):
        P = cam[0:3] + t * rays
        i, j, z, ok = TM.reproject_fp32(P, cam, H, W)
        assert ok.all()
        np.testing.assert_array_equal(i, ii)
        np.testing.assert_array_equal(j, jj)
        # z is the distance along the forward axis
        np.testing.assert_allclose(z, t * (rays @ cam[3:6]), rtol=1e-6)


def test_reprojection_rejects_behind_and_outside():
    scene = scenegen.random_scene(3, 8)
    cam = _cam(scene, 16, 16)
    C, f, r = cam[0:3], cam[3:6], cam[6:9]
    P = np.stack([C - 2.0 * f, C + 1.0 * f + 50.0 * r, C + 1.0 * f])
    _, _, _, ok = TM.reproject_fp32(P, cam, 16, 16)
    assert ok.tolist() == [False, False, True]


def _static_pair(seed=5, H=48, W=64):
    f = scenegen.render_frame(scenegen.random_scene(seed, 16), H, W, 64, 64)
    return f, _cam(f.scene, H, W)


def test_identical_frames_give_zero_and_accept_every_covered_pixel():
    f, cam = _static_pair()
    rng = np.random.default_rng(0)
    I = rng.random((f.H, f.W)).astype(np.float32)
    s, c = TM.instability_pair(I, I, f.pos4, f.nrm4, f.pos4, f.nrm4, cam)
    assert s == 0.0
    assert c == int((f.pos4[..., 3] > 0).sum()) == f.H * f.W


def test_constant_difference_closed_form():
    f, cam = _static_pair()
    I0 = np.full((f.H, f.W), 0.25, np.float32)
    I1 = np.full((f.H, f.W), 0.75, np.float32)
    s, c = TM.instability_pair(I1, I0, f.pos4, f.nrm4, f.pos4, f.nrm4, cam, alpha=3.0)
    assert s == pytest.approx(c * (math.exp(1.5) - 1.0), rel=1e-12)
    E, cnt = TM.temporal_instability([I0, I1, I1], [f.pos4] * 3, [f.nrm4] * 3, [cam] * 3)
    assert cnt == 2 * c
    assert E == pytest.approx(c * (math.exp(1.5) - 1.0) / (2 * f.H * f.W), rel=1e-12)


def test_depth_and_normal_rejection():
    f, cam = _static_pair()
    I = np.zeros((f.H, f.W), np.float32)
    J = np.ones((f.H, f.W), np.float32)
    prev_pos, prev_nrm = f.pos4.copy(), f.nrm4.copy()
    prev_pos[0:8, :, 3] *= 1.05    # 5% deeper: rejected
    prev_pos[8:16, :, 3] *= 1.005  # 0.5%: kept
    prev_nrm[16:24, :, :3] *= -1   # flipped normals: rejected
    prev_pos[24:32, :, 3] = 0      # nothing seen: rejected
    _, c = TM.instability_pair(J, I, f.pos4, f.nrm4, prev_pos, prev_nrm, cam)
    assert c == f.H * f.W - 3 * 8 * f.W


def test_reprojection_finds_the_same_surface_point():
    """Camera moved between frames: an accepted pixel's reprojection sees
    (within about a pixel footprint) the same world point in the previous
    frame's G-buffer."""
    H, W = 96, 128
    s1 = scenegen.random_scene(9, 12)
    s0 = scenegen.dataclasses.replace(s1, cam_pos=s1.cam_pos + np.array([0.05, -0.03, 0.02]))
    f1 = scenegen.render_frame(s1, H, W, 64, 64)
    f0 = scenegen.render_frame(s0, H, W, 64, 64)
    cam0 = _cam(s0, H, W)
    i, j, z, ok = TM.reproject_fp32(f1.pos4[..., :3], cam0, H, W)
    acc = ok & TM.accept_fp32(z, np.where(ok, f0.pos4[..., 3][j, i], 0), f1.nrm4[..., :3], f0.nrm4[..., :3][j, i])
    assert acc.mean() > 0.8
    gap = np.linalg.norm(f0.pos4[..., :3][j, i] - f1.pos4[..., :3], axis=-1)[acc]
    footprint = 2.0 * z[acc] * cam0[12] / H  # one pixel at the reprojected depth
    assert np.median(gap / footprint) < 1.0
    assert np.percentile(gap / footprint, 95) < 4.0  # grazing ground pixels stretch along the view


def test_screen_width_matches_projected_endpoints():
    """w H / (2 d tan) equals the pixel distance between the projections of
    two points w apart across the view axis at depth d."""
    scene = scenegen.random_scene(3, 8)
    H, W = 1080, 1920
    cam = _cam(scene, H, W)
    C, f, u = cam[0:3], cam[3:6], cam[9:12]
    for d, w in ((1.0, 0.01), (3.5, 0.2), (7.0, 0.05)):
        a = C + d * f - 0.5 * w * u
        b = C + d * f + 0.5 * w * u
        ya = (0.5 - 0.5 * ((a - C) @ u) / (d * cam[12])) * H
        yb = (0.5 - 0.5 * ((b - C) @ u) / (d * cam[12])) * H
        assert TM.screen_width_px(w, d, H, cam[12]) == pytest.approx(abs(ya - yb), rel=1e-12)


def test_p95_and_depth_rule():
    assert TM.p95_from_histogram([100, 0, 0], 0.5) == 0.5
    assert TM.p95_from_histogram([90, 5, 5], 1.0) == 2.0
    assert TM.p95_from_histogram([0, 0, 0], 1.0) == 0.0
    # uniform widths on [0, 100) px: the 95th percentile is 95
    w = np.arange(0, 100, 0.01) + 0.005
    h = TM.penumbra_histogram(w, 1.0, 200)
    assert TM.p95_from_histogram(h, 1.0) == 95.0
    # out-of-range widths: negative in bin 0, huge in the last bin
    h = TM.penumbra_histogram([-3.0, 1e9], 1.0, 8)
    assert h[0] == 1 and h[-1] == 1
    # receptive fields 3 * 2^l = 24 / 96 / 384 of the 3 / 5 / 7-level nets (Sec. 3.6)
    assert [TM.depth_for_width(p) for p in (24.0, 96.0, 384.0)] == [3, 5, 7]
    assert TM.depth_for_width(25.0) == 4 and TM.depth_for_width(23.9) == 3
    assert TM.depth_for_width(2.0) == 1
