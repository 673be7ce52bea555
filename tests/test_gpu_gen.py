"""GPU scene generation (ray-cast G-buffer, shadow map, Monte-Carlo
visibility) against the FP64 C ray caster on the same seeded scenes.  The GPU
casts in FP32, so decisions may differ on silhouette edges: hit masks agree on
>= 99.9% of pixels, positions / depths where both hit agree to FP32 precision,
and Monte-Carlo visibilities (same SplitMix64-keyed stratified samples, jitter
rounded to 24 bits) agree on >= 98% of pixels with a mean difference <= 2e-3."""
import numpy as np
import pytest

import scenegen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2301_05262_gb300 as nsm  # noqa: E402


def _gpu_gbuffer(scene, H, W):
    pos = torch.empty((H, W, 4), device="cuda")
    nrm = torch.empty((H, W, 4), device="cuda")
    mask = torch.empty((H, W), dtype=torch.uint8, device="cuda")
    nsm.gen_gbuffer(H, W, scenegen.camera_vector(scene, H, W), scene.objects, pos, nrm, mask)
    torch.cuda.synchronize()
    return pos, nrm, mask


@pytest.mark.parametrize("seed,n_obj", [(1, 8), (21, 32), (5, 64)])
def test_gbuffer_matches_ray_caster(seed, n_obj):
    scene = scenegen.random_scene(seed, n_obj, soft=True)
    H, W = 192, 256
    f = scenegen.render_frame(scene, H, W, 64, 64)
    pos, nrm, mask = (t.cpu().numpy() for t in _gpu_gbuffer(scene, H, W))
    assert (mask == f.mask).mean() >= 0.999
    both = (mask == 1) & (f.mask == 1)
    dp = np.abs(pos[..., :3] - f.pos4[..., :3]).max(axis=-1)
    same = dp <= 1e-3  # same surface hit; elsewhere a silhouette decided differently
    assert same[both].mean() >= 0.999
    # FP32 hit distances: ~1e-7 typically, larger where the ray grazes the ground plane
    assert np.median(dp[both & same]) <= 1e-6
    assert np.percentile(dp[both & same], 99) <= 1e-4
    dd = np.abs(pos[..., 3] - f.pos4[..., 3])[both & same]
    assert np.percentile(dd, 99) <= 1e-4
    # sphere normals are (P - C) / r: the position error divided by the radius
    dn = np.abs(nrm - f.nrm4)[both & same].max(axis=-1)
    assert np.median(dn) <= 1e-6
    assert np.percentile(dn, 99.9) <= 1e-3


@pytest.mark.parametrize("seed,n_obj,S", [(1, 8, 256), (21, 32, 512), (5, 64, 300)])
def test_shadowmap_matches_ray_caster(seed, n_obj, S):
    scene = scenegen.random_scene(seed, n_obj, soft=False)
    f = scenegen.render_frame(scene, 8, 8, S, S)
    depth = torch.empty((S, S), device="cuda")
    nsm.gen_shadowmap(S, S, scenegen.light_camera_vector(scene), scenegen.Z_FAR, scene.objects, depth)
    torch.cuda.synchronize()
    d = depth.cpu().numpy()
    rel = np.abs(d - f.sm) / f.sm
    assert (rel <= 1e-5).mean() >= 0.999
    assert ((d == scenegen.Z_FAR) == (f.sm == scenegen.Z_FAR)).mean() >= 0.999


@pytest.mark.parametrize("soft", [False, True])
def test_visibility_matches_ray_caster(soft):
    scene = scenegen.random_scene(21, 24, soft=soft)
    f = scenegen.render_frame(scene, 96, 128, 64, 64)
    spp = 8
    ref = scenegen.soft_visibility(f, spp_side=spp, seed=7) if soft else scenegen.hard_visibility(f).astype(np.float32)
    pos = torch.from_numpy(f.pos4).cuda()
    nrm = torch.from_numpy(f.nrm4).cuda()
    mask = torch.from_numpy(f.mask).cuda()
    vis = torch.empty((f.H, f.W), device="cuda")
    nsm.gen_visibility(f.H, f.W, pos, nrm, mask, scene.light_pos, f.light_radius if soft else 0.0,
                       spp if soft else 1, 7, scenegen.SHADOW_EPS, scene.objects, vis)
    torch.cuda.synchronize()
    v = vis.cpu().numpy()
    assert (v == ref).mean() >= (0.98 if soft else 0.999)
    assert np.abs(v - ref).mean() <= 2e-3
    assert ((v >= 0) & (v <= 1)).all()


def test_generator_rejects_bad_arguments():
    with pytest.raises(nsm.NSMError):
        nsm.gen_shadowmap(8, 8, np.zeros(13), -1.0, np.zeros((0, 5)), torch.empty((8, 8), device="cuda"))
    with pytest.raises(nsm.NSMError):
        nsm.gen_gbuffer(4, 4, np.zeros(14), np.zeros((300, 5)), torch.empty((4, 4, 4), device="cuda"),
                        torch.empty((4, 4, 4), device="cuda"), torch.empty((4, 4), dtype=torch.uint8, device="cuda"))
