"""Pins for the seeded scene generator (ray casting of G-buffer, shadow map,
brute-force and Monte-Carlo visibility) against closed forms."""
import math

import numpy as np
import pytest

import scenegen


def test_splitmix64_reference_values():
    # SplitMix64 seeded with 0: published first outputs of the generator
    r = scenegen.SplitMix64(0)
    assert r.next_u64() == 0xE220A8397B1DCDAF
    assert r.next_u64() == 0x6E789E6AA1B965F4
    assert r.next_u64() == 0x06C45D188009454F


def test_ray_sphere_closed_form():
    obj = [[0, 0.0, 0.0, 1.0, 0.5]]
    t, n = scenegen.trace_one([0, 0, 5.0], [0, 0, -1.0], obj, with_plane=False)
    assert t == pytest.approx(3.5, abs=1e-12)
    np.testing.assert_allclose(n, [0, 0, 1], atol=1e-12)
    # oblique ray grazing at distance h from the centre: chord half-length sqrt(s^2 - h^2)
    h = 0.3
    t, n = scenegen.trace_one([h, -4.0, 1.0], [0, 1.0, 0], obj, with_plane=False)
    assert t == pytest.approx(4.0 - math.sqrt(0.25 - h * h), abs=1e-12)
    t, _ = scenegen.trace_one([0.6, -4.0, 1.0], [0, 1.0, 0], obj, with_plane=False)
    assert t == -1.0


def test_ray_box_closed_form():
    obj = [[1, 0.0, 0.0, 1.0, 0.25]]
    t, n = scenegen.trace_one([0.1, 0.05, 3.0], [0, 0, -1.0], obj, with_plane=False)
    assert t == pytest.approx(3.0 - 1.25, abs=1e-12)
    np.testing.assert_allclose(n, [0, 0, 1], atol=0)
    d = np.array([1.0, 0.0, -0.0])
    t, n = scenegen.trace_one([-2.0, 0.1, 1.1], d, obj, with_plane=False)
    assert t == pytest.approx(2.0 - 0.25, abs=1e-12)
    np.testing.assert_allclose(n, [-1, 0, 0], atol=0)
    # diagonal ray into the edge region
    d = np.array([1.0, 1.0, 0.0]) / math.sqrt(2)
    t, n = scenegen.trace_one([-1.0, -0.9, 1.0], d, obj, with_plane=False)
    # enters through x = -0.25 at t = 0.75 sqrt(2) (y there = -0.15, inside)
    assert t == pytest.approx(0.75 * math.sqrt(2), abs=1e-12)
    np.testing.assert_allclose(n, [-1, 0, 0], atol=0)


def test_ray_plane_and_ties():
    t, n = scenegen.trace_one([0.3, 0.2, 2.0], np.array([0.6, 0.0, -0.8]), [], with_plane=True)
    assert t == pytest.approx(2.5, abs=1e-12)
    np.testing.assert_allclose(n, [0, 0, 1])
    # the plane loses an exact tie against a box whose bottom face lies on z = 0
    obj = [[1, 0.0, 0.0, 0.25, 0.25]]
    t, n = scenegen.trace_one([0.0, 0.0, -1.0], [0, 0, 1.0], obj, with_plane=True)
    assert t == pytest.approx(1.0)
    np.testing.assert_allclose(n, [0, 0, -1])


def test_gbuffer_geometry():
    f = scenegen.hard_frame(48, 64, 64, 64, 8, 3)
    assert f.mask.all()  # every camera ray points down and meets the ground
    P = f.pos4[..., :3].astype(np.float64)
    n = f.nrm4[..., :3].astype(np.float64)
    np.testing.assert_allclose(np.linalg.norm(n, axis=-1), 1.0, atol=1e-6)
    assert (f.pos4[..., 3] > 0).all()
    # view depth d = (P - C) . fwd
    C = f.scene.cam_pos
    fwd = np.asarray(f.scene.cam_target) - C
    fwd /= np.linalg.norm(fwd)
    np.testing.assert_allclose(f.pos4[..., 3], (P - C) @ fwd, rtol=2e-6, atol=2e-6)
    # ground pixels lie on z = 0 with normal +z
    ground = np.abs(n[..., 2] - 1.0) < 1e-9
    assert ground.mean() > 0.5
    # surfaces face the camera
    assert (np.sum(n * (C - P), axis=-1) > -1e-6).all()


def test_shadowmap_depth_is_distance_to_first_hit():
    f = scenegen.hard_frame(16, 16, 32, 32, 6, 11)
    L = np.asarray(f.scene.light_pos, np.float64)
    fwd, right, up, t, VP = scenegen.light_frustum(L)
    for (i, j) in [(0, 0), (5, 17), (16, 16), (31, 31), (20, 3)]:
        nx = 2 * (i + 0.5) / 32 - 1
        ny = 2 * (j + 0.5) / 32 - 1
        d = fwd + nx * t * right + ny * t * up
        d /= np.linalg.norm(d)
        th, _ = scenegen.trace_one(L, d, f.scene.objects)
        expect = th if 0 < th < f.z_far else f.z_far
        assert f.sm[j, i] == np.float32(expect)
        # the light matrix maps that texel-centre ray back to the texel centre
        Pw = L + 2.0 * d
        clip = VP @ np.append(Pw, 1.0)
        np.testing.assert_allclose(clip[:2] / clip[3], [nx, ny], atol=1e-12)


def test_hard_visibility_unoccluded_ground_is_lit():
    scene = scenegen.Scene(objects=np.zeros((0, 5)), light_pos=np.array([0.5, 0.3, 3.0]), light_radius=0.0)
    f = scenegen.render_frame(scene, 32, 32, 64, 64)
    assert scenegen.hard_visibility(f).all()
    assert (scenegen.soft_visibility(f, spp_side=4, radius=0.2) == 1.0).all()


def test_sphere_over_plane_shadow_is_exact_conic():
    """Point light L, sphere (S, R) above the ground: a ground point P is in
    shadow iff the distance from S to the segment P-L is below R."""
    S = np.array([0.1, -0.2, 0.6])
    R = 0.3
    L = np.array([0.4, 0.5, 2.8])
    scene = scenegen.Scene(objects=np.array([[0.0, *S, R]]), light_pos=L, light_radius=0.0)
    f = scenegen.render_frame(scene, 64, 64, 64, 64)
    vis = scenegen.hard_visibility(f).astype(bool)
    P = f.pos4[..., :3].astype(np.float64)
    ground = (f.nrm4[..., 2] > 0.999) & (np.abs(f.pos4[..., 2]) < 1e-6)
    d = L - P
    tt = np.clip(np.sum((S - P) * d, axis=-1) / np.sum(d * d, axis=-1), 0, 1)
    closest = P + tt[..., None] * d
    dist = np.linalg.norm(closest - S, axis=-1)
    margin = np.abs(dist - R) > 1e-4
    expect_lit = dist >= R
    sel = ground & margin
    assert sel.sum() > 1000
    assert (~expect_lit[sel]).sum() > 50  # the shadow is in view
    np.testing.assert_array_equal(vis[sel], expect_lit[sel])


def test_soft_visibility_umbra_and_point_limit():
    # a big sphere straight above a ground point: umbra -> 0
    L = np.array([0.0, 0.0, 3.0])
    scene = scenegen.Scene(objects=np.array([[0.0, 0.0, 0.0, 1.5, 0.6]]), light_pos=L, light_radius=0.1)
    f = scenegen.render_frame(scene, 32, 32, 64, 64)
    P = f.pos4[..., :3]
    ground = (f.nrm4[..., 2] > 0.999) & (np.abs(f.pos4[..., 2]) < 1e-6)
    near = ground & (np.hypot(P[..., 0], P[..., 1]) < 0.2)
    if near.any():
        v = scenegen.soft_visibility(f, spp_side=8)
        assert (v[near] == 0.0).all()
    # r = 0: Monte-Carlo visibility equals the brute-force hard visibility
    f2 = scenegen.hard_frame(32, 32, 64, 64, 8, 2)
    v0 = scenegen.soft_visibility(f2, spp_side=4, radius=0.0)
    np.testing.assert_array_equal(v0, scenegen.hard_visibility(f2).astype(np.float32))


def _segment_fraction(h, r):
    """Visible fraction of a disk of radius r cut by a straight edge at signed
    distance h from its centre (the part beyond the edge is hidden)."""
    if h >= r:
        return 1.0
    if h <= -r:
        return 0.0
    seg = r * r * math.acos(h / r) - h * math.sqrt(r * r - h * h)  # area beyond the edge
    return 1.0 - seg / (math.pi * r * r)


def _single_pixel_frame(P, n, L, r, objects):
    pos4 = np.zeros((1, 1, 4), np.float32)
    pos4[0, 0, :3] = P
    pos4[0, 0, 3] = 1.0
    nrm4 = np.zeros((1, 1, 4), np.float32)
    nrm4[0, 0, :3] = n
    return scenegen.Frame(H=1, W=1, pos4=pos4, nrm4=nrm4, mask=np.ones((1, 1), np.uint8),
                          sm=np.zeros((1, 1), np.float32), view_proj=np.eye(4, dtype=np.float32),
                          light_pos=np.asarray(L, np.float32), light_radius=r, r_hat=0.0,
                          cam_pos=np.zeros(3, np.float32), z_far=100.0, bias=0.0, tan_half_fov=1.0,
                          scene=scenegen.Scene(objects=np.asarray(objects, np.float64), light_pos=np.asarray(L),
                                               light_radius=r))


def test_soft_visibility_straight_edge_closed_form():
    """Ground point P = 0 below an emitter disk of radius r centred at
    L = (0, 0, 2) (the disk is perpendicular to L - P, i.e. horizontal).  A
    huge box filling x >= e, z >= 0.9 blocks exactly the rays towards disk
    points with x_d > e (a ray reaches x = e at height 2 e / x_d < 2).  The
    visible fraction is therefore one minus the circular segment beyond the
    chord x = e; the mirrored box checks the other half of the disk.  This
    pins the stratification and the uniform (area-preserving) concentric
    mapping of the samples."""
    L = np.array([0.0, 0.0, 2.0])
    r = 0.2
    for e in [0.0, 0.05, 0.12]:
        expect = _segment_fraction(e, r)
        for side in (+1.0, -1.0):
            cx = side * (e + 50.0)
            box = [[1.0, cx, 0.0, 50.9, 50.0]]
            fr = _single_pixel_frame([0, 0, 0], [0, 0, 1], L, r, box)
            v = scenegen.soft_visibility(fr, spp_side=128)[0, 0]
            assert abs(v - expect) < 2e-3, (e, side, v, expect)
    # with 32 x 32 samples (the default) the estimate stays within a few 1e-3
    fr = _single_pixel_frame([0, 0, 0], [0, 0, 1], L, r, [[1.0, 50.05, 0.0, 50.9, 50.0]])
    assert abs(scenegen.soft_visibility(fr)[0, 0] - _segment_fraction(0.05, r)) < 5e-3
