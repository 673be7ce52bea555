"""Pins for the oracle's shadow-map lookup, hard depth test, features,
blocker search and penumbra model (Sec. 3.1, 3.2, 3.6, suppl. Sec. 4)."""
import math

import numpy as np
import pytest

import scenegen
from oracle import gather as G

F32 = np.float32


def test_projection_known_indices():
    """A hand-built clip matrix with ndc = (x, y) (w = 1): texel i = floor((x/2+1/2) Ws)."""
    M = np.eye(4, dtype=F32)
    M[2, :] = 0
    Ws, Hs = 8, 4
    P = np.array([[0.0, 0.0, 5.0],      # centre -> (4, 2)
                  [-1.0, -1.0, 0.0],    # corner -> (0, 0)
                  [0.999, 0.999, 0.0],  # -> (7, 3)
                  [1.0, 0.0, 0.0],      # u = 1 -> i = 8, outside
                  [-0.75, 0.5, 0.0],    # u = 0.125 -> i = 1 exactly on a boundary; v = 0.75 -> j = 3
                  [-1.0000001, 0.0, 0.0]], F32)
    i, j, inside, _ = G.project_fp32(P, M, Ws, Hs)
    assert list(inside) == [True, True, True, False, True, False]
    assert list(i[inside]) == [4, 0, 7, 1]
    assert list(j[inside]) == [2, 0, 3, 3]


def test_projection_behind_light_is_outside():
    M = np.zeros((4, 4), F32)
    M[0, 0] = M[1, 1] = 1
    M[3, 2] = -1  # w = -z (looking down -z)
    P = np.array([[0.1, 0.1, -1.0], [0.1, 0.1, 1.0], [0.1, 0.1, 0.0]], F32)
    _, _, inside, cw = G.project_fp32(P, M, 16, 16)
    assert list(inside) == [True, False, False]


def test_projection_binary32_order_matters_and_fp64_agrees_elsewhere():
    f = scenegen.hard_frame(96, 128, 512, 512, 8, 1)
    P = f.pos4[..., :3]
    i, j, inside, _ = G.project_fp32(P, f.view_proj, 512, 512)
    tex32 = np.where(inside, j * 512 + i, -1)
    tex64 = G.project_fp64_index(P, f.view_proj, 512, 512)
    diff = tex32 != tex64
    assert diff.mean() < 1e-3  # only pixels that sit on a texel boundary
    # where they differ, the two choices are neighbouring texels
    if diff.any():
        a, b = tex32[diff], tex64[diff]
        both = (a >= 0) & (b >= 0)
        assert (np.abs(a[both] % 512 - b[both] % 512) <= 1).all()
        assert (np.abs(a[both] // 512 - b[both] // 512) <= 1).all()


def test_depth_test_binary32_definition():
    zf = np.array([1.0, 1.0, 2.0, 3.0], F32)
    z = np.array([1.0, 0.99, 1.9, 100.0], F32)
    beta = 0.01
    hard = G.depth_test_fp32(zf, z, beta)
    # 1 <= 1 + 0.01; 1 <= 0.99 + 0.01 (= 1.0 in binary32); 2 <= 1.9 + 0.02 false; far -> lit
    assert list(hard) == [True, F32(0.99) + F32(0.01) * F32(1.0) >= F32(1.0), False, True]


def _ambiguity(f, tex, zf):
    """Pixels whose hard bit is not decided at the map's resolution: the
    decision differs among the 3x3 texels around the chosen one, or the exact
    light ray meets an occluder within the bias distance of the pixel."""
    Hs, Ws = f.sm.shape
    ins = tex >= 0
    j = np.where(ins, tex // Ws, 0)
    i = np.where(ins, tex % Ws, 0)
    dec = []
    for dj in (-1, 0, 1):
        for di in (-1, 0, 1):
            jj = np.clip(j + dj, 0, Hs - 1)
            ii = np.clip(i + di, 0, Ws - 1)
            dec.append(G.depth_test_fp32(zf, f.sm[jj, ii], f.bias))
    dec = np.stack(dec)
    amb = ~(dec.all(0) | (~dec).all(0))
    ze = scenegen.light_depth_exact(f)
    zf64 = np.linalg.norm(f.pos4[..., :3].astype(np.float64) - f.scene.light_pos, axis=-1)
    contact = (zf64 - ze > 1e-6 * zf64) & (zf64 - ze <= 1.01 * f.bias * zf64)
    return amb | contact


@pytest.mark.parametrize("seed", [2, 4])
def test_hard_bit_matches_brute_force_shadow_rays(seed):
    """Shadow-map hard visibility vs brute-force shadow rays on a tiny scene:
    identical wherever the map resolution decides the answer."""
    f = scenegen.hard_frame(128, 128, 1024, 1024, 12, seed)
    vis = scenegen.hard_visibility(f).astype(bool)
    tex, z, hard = G.lookup_and_test(f.pos4, f.sm, f.view_proj, f.light_pos, f.z_far, f.bias)
    zf = G.emitter_distance_fp32(f.pos4[..., :3], f.light_pos)
    ins = tex >= 0
    amb = _ambiguity(f, tex, zf)
    decided = ins & ~amb
    assert decided.sum() > 0.6 * ins.sum()
    assert (~vis[decided]).sum() > 100 and vis[decided].sum() > 100
    np.testing.assert_array_equal(hard[decided], vis[decided])
    # and the disagreements are rare overall
    assert (hard != vis)[ins].mean() < 0.02


def test_hard_bit_sphere_over_plane_conic():
    S = np.array([0.1, -0.2, 0.6])
    R = 0.3
    L = np.array([0.4, 0.5, 2.8])
    scene = scenegen.Scene(objects=np.array([[0.0, *S, R]]), light_pos=L, light_radius=0.0)
    f = scenegen.render_frame(scene, 96, 96, 2048, 2048)
    tex, z, hard = G.lookup_and_test(f.pos4, f.sm, f.view_proj, f.light_pos, f.z_far, f.bias)
    zf = G.emitter_distance_fp32(f.pos4[..., :3], f.light_pos)
    P = f.pos4[..., :3].astype(np.float64)
    d = L - P
    tt = np.clip(np.sum((S - P) * d, axis=-1) / np.sum(d * d, axis=-1), 0, 1)
    dist = np.linalg.norm(P + tt[..., None] * d - S, axis=-1)
    ground = (f.nrm4[..., 2] > 0.999) & (np.abs(f.pos4[..., 2]) < 1e-6) & (tex >= 0)  # the plane, not the sphere top
    amb = _ambiguity(f, tex, zf)
    sel = ground & ~amb
    assert (dist[sel] < R).sum() > 100
    np.testing.assert_array_equal(hard[sel], dist[sel] >= R)


def test_features_closed_form_single_pixel():
    """P on the ground straight below the light, camera above: c_e = n.(L-P)/|L-P| = 1."""
    Lp = np.array([0.0, 0.0, 2.0], F32)
    Cp = np.array([0.0, -3.0, 4.0], F32)
    pos4 = np.array([[[0.0, 0.0, 0.0, 2.5]]], F32)
    nrm4 = np.array([[[0.0, 0.0, 1.0, 0.0]]], F32)
    sm = np.full((4, 4), 1.5, F32)
    M = np.eye(4, dtype=F32)
    M[2, :] = 0
    feat, tex, hard = G.features(pos4, nrm4, sm, M, Lp, Cp, 2.0, 100.0, 0.0)
    zf = 2.0
    ce = 1.0
    cc = 4.0 / 5.0
    np.testing.assert_allclose(feat[:, 0, 0], [ce + 2.0, 1.5 / zf, 1.5 - zf, cc / 2.5], rtol=0, atol=1e-15)
    assert tex[0, 0] == 2 * 4 + 2 and not hard[0, 0]


def test_features_invariants_on_rendered_frame():
    f = scenegen.hard_frame(64, 96, 256, 256, 8, 7)
    feat, tex, hard = G.features(f.pos4, f.nrm4, f.sm, f.view_proj, f.light_pos, f.cam_pos,
                                 f.r_hat, f.z_far, f.bias)
    assert feat.shape == (4, 64, 96)
    assert (np.abs(feat[0]) <= 1 + 1e-6).all()          # cosine, point light r_hat = 0
    assert (feat[3] > 0).all()                            # surfaces face the camera, d > 0
    out = tex < 0
    np.testing.assert_allclose(feat[2][out] + np.linalg.norm(
        f.pos4[..., :3][out].astype(np.float64) - f.light_pos, axis=-1), f.z_far, rtol=1e-12)
    # lit pixels inside the map: z close to z_f -> z/z_f near 1
    lit = hard & ~out
    assert np.median(np.abs(feat[1][lit] - 1.0)) < 5e-3
    # the emitter size is a DC offset on c_e only
    feat2, _, _ = G.features(f.pos4, f.nrm4, f.sm, f.view_proj, f.light_pos, f.cam_pos,
                             3.25, f.z_far, f.bias)
    np.testing.assert_allclose(feat2[0] - feat[0], 3.25, atol=1e-12)
    np.testing.assert_array_equal(feat2[1:], feat[1:])


def test_emitter_size_feature_scale():
    assert scenegen.emitter_size_feature(0.0) == 0.0
    assert scenegen.emitter_size_feature(0.25) == pytest.approx(4.0)   # 50 cm diameter -> 4
    assert scenegen.emitter_size_feature(0.125) == pytest.approx(2.0)
    assert scenegen.emitter_size_feature(1.0) == 4.0


def test_blocker_search_brute_force_tiny():
    rng = np.random.default_rng(0)
    Hs = Ws = 16
    sm = rng.uniform(1.0, 3.0, (Hs, Ws)).astype(F32)
    M = np.eye(4, dtype=F32)
    M[2, :] = 0
    pos = rng.uniform(-0.95, 0.95, (5, 7, 3)).astype(F32)
    pos4 = np.concatenate([pos, np.ones((5, 7, 1), F32)], axis=-1)
    L = np.array([0.0, 0.0, 2.5], F32)
    r, th, beta = 0.3, 0.5, 0.01
    zmin, zmax, found = G.blocker_search(pos4, sm, M, L, r, th, 100.0, beta, kmax=32)
    i, j, inside, _ = G.project_fp32(pos4[..., :3], M, Ws, Hs)
    zf = G.emitter_distance_fp32(pos4[..., :3], L)
    for idx in np.ndindex(5, 7):
        k = math.ceil(float(F32(r) * F32(8.0) / (zf[idx] * F32(th))))
        vals = [sm[b, a] for b in range(Hs) for a in range(Ws)
                if abs(a - i[idx]) <= k and abs(b - j[idx]) <= k and sm[b, a] < zf[idx] - F32(beta) * zf[idx]]
        assert found[idx] == bool(vals)
        if vals:
            assert zmin[idx] == min(vals) and zmax[idx] == max(vals)


def test_blocker_search_special_cases():
    Hs = Ws = 8
    sm = np.full((Hs, Ws), 5.0, F32)
    sm[3, 3] = 1.0
    M = np.eye(4, dtype=F32)
    M[2, :] = 0
    # pixel projecting to texel (3,3): x = (3.5/8)*2-1
    x = (3.5 / 8) * 2 - 1
    pos4 = np.array([[[x, x, 0.0, 1.0], [x + 0.5, x, 0.0, 1.0]]], F32)
    L = np.array([0.0, 0.0, 3.0], F32)
    # point light: k = 0 -> only the own texel
    zmin, zmax, found = G.blocker_search(pos4, sm, M, L, 0.0, 0.5, 100.0, 0.0)
    assert found[0, 0] and zmin[0, 0] == 1.0 and zmax[0, 0] == 1.0
    assert not found[0, 1] and zmin[0, 1] == 0.0
    # big emitter: the window reaches the blocker from the second pixel as well
    zmin, zmax, found = G.blocker_search(pos4, sm, M, L, 1.0, 0.5, 100.0, 0.0)
    assert found[0, 1] and zmin[0, 1] == 1.0


def _footprint_texels(VP64, L, fwd, right, up, z_f, r, Ws, Hs):
    """Half-separation, in texels, of the light-space images of a segment of
    half-length r centred on a receiver that sits on the light's view axis at
    distance z_f and lies perpendicular to that axis (along the map's right
    and up axes).  Projective geometry through the light's own FP64
    world->clip matrix; nothing here uses a window formula."""
    P = np.asarray(L, np.float64) + z_f * fwd

    def uv(Q):
        c = VP64 @ np.append(Q, 1.0)
        return (c[0] / c[3] * 0.5 + 0.5) * Ws, (c[1] / c[3] * 0.5 + 0.5) * Hs

    (xa, _), (xb, _) = uv(P - r * right), uv(P + r * right)
    (_, ya), (_, yb) = uv(P - r * up), uv(P + r * up)
    return 0.5 * abs(xb - xa), 0.5 * abs(yb - ya)


@pytest.mark.parametrize("light_dist,Ws", [(3.0, 2048), (3.0, 512), (5.0, 1024), (8.0, 4096)])
def test_blocker_window_is_emitter_footprint_in_texels(light_dist, Ws):
    """The window half-size is the emitter radius, carried to the receiver's
    depth and measured in shadow-map texels through the light's projection
    (the PCSS search region of the penumbra model, suppl. Sec. 4): project the
    receiver's two points at +-r along the map axes and take half their
    separation, rounded up and capped at 32.  Several light distances change
    the light frustum's fov (fov = 2 asin(2/|L|)), so tan(fov/2) against
    tan(fov), and Ws/2 against Ws, give different windows."""
    rng = np.random.default_rng(int(light_dist * 10) + Ws)
    checked = 0
    for _ in range(40):
        d = rng.normal(size=3)
        d[2] = abs(d[2]) + 0.5
        L = light_dist * d / np.linalg.norm(d)
        fwd, right, up, t, VP = scenegen.light_frustum(L)
        z_f = float(rng.uniform(0.5, 1.0) * light_dist)
        r = float(rng.uniform(0.005, 0.3))
        hx, hy = _footprint_texels(VP, L, fwd, right, up, z_f, r, Ws, Ws)
        assert hx == pytest.approx(hy, rel=1e-9)          # square texels, square window
        frac = hx - math.floor(hx)
        if min(frac, 1.0 - frac) < 1e-3:                  # too close to an integer to judge ceil
            continue
        want = min(32, math.ceil(hx))
        got = int(G.blocker_window_half(F32(z_f), r, Ws, t))
        assert got == want, (L, z_f, r, hx)
        checked += 1
    assert checked >= 30


def test_blocker_window_distinguishes_scale_errors():
    """A hand-picked case where the footprint is well below the cap: a light at
    distance 3 (tan(fov/2) = 2/sqrt(5)), Ws = 512, r = 0.05, receiver at 2.5.
    The footprint is r (Ws/2) / (z_f tan(fov/2)) = 5.72 texels -> k = 6; a
    window built on Ws (11.4 -> 12), on tan(fov) (0.57 -> 1) or on the
    diameter (11.4 -> 12) would differ."""
    L = np.array([0.0, -1.0, 2.8284271247461903])
    fwd, right, up, t, VP = scenegen.light_frustum(L)
    assert t == pytest.approx(2.0 / math.sqrt(5.0), rel=1e-12)
    hx, _ = _footprint_texels(VP, L, fwd, right, up, 2.5, 0.05, 512, 512)
    assert hx == pytest.approx(5.7243340, rel=1e-6)
    assert int(G.blocker_window_half(F32(2.5), 0.05, 512, t)) == 6
    # the cap: a large emitter close to the light reaches 32
    assert int(G.blocker_window_half(F32(0.2), 0.3, 512, t)) == 32


def test_penumbra_model_closed_forms():
    zf = np.array([2.0, 3.0, 5.0])
    zmin = np.array([1.0, 1.5, 2.0])
    zmax = np.array([1.4, 1.5, 3.0])
    # r_e = 0: theta = 0 -> x_a = -x_b -> zero width
    xa, xb = G.penumbra_width(zf, zmin, zmax, 0.0)
    np.testing.assert_allclose(xa + xb, 0.0, atol=1e-12)
    # r_s = 0 (z_min = z_max): x_a = x_b = r_e (z_f - z_m) / z_m (similar triangles)
    re = 0.25
    xa, xb = G.penumbra_width(zf, zmin, zmin, re)
    np.testing.assert_allclose(xa, re * (zf - zmin) / zmin, rtol=1e-12)
    np.testing.assert_allclose(xb, xa, rtol=1e-12)
    # the width grows with the receiver distance
    xa, xb = G.penumbra_width(np.array([2.0, 4.0]), np.array([1.0, 1.0]), np.array([1.2, 1.2]), 0.2)
    assert (xa + xb)[1] > (xa + xb)[0]


def test_receptive_field_rule(golden_counts):
    for l, rf in golden_counts["receptive_field"]["values"].items():
        assert G.receptive_field(int(l)) == rf
        assert G.levels_for_penumbra(rf) == pytest.approx(int(l))


@pytest.fixture(scope="module")
def golden_counts():
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_network_counts.json")) as fh:
        return json.load(fh)
