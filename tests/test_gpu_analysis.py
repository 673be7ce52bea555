"""GPU parity of the frame-analysis calls against the oracle: the Eq. 3
temporal-instability terms (accepted-pixel counts exact: reprojection and the
depth / normal tests are binary32 on both sides; sums within binary32
rounding of exp) and the Sec. 3.6 penumbra histogram (per-pixel widths are
binary32 on the GPU and FP64 in the oracle, so a pixel whose width lies
within rounding of a bin edge may land in the neighbouring bin)."""
import numpy as np
import pytest

import scenegen
from oracle import gather as G
from oracle import temporal as TM

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2301_05262_gb300 as nsm  # noqa: E402
from gpu_helpers import DeviceFrame, run_features  # noqa: E402


def _images(frames, seed):
    """Seeded test images: each frame's ray-cast hard visibility blended with noise."""
    rng = np.random.default_rng(seed)
    return [(0.7 * scenegen.hard_visibility(f) + 0.3 * rng.random((f.H, f.W))).astype(np.float32) for f in frames]


def _gpu_pair(I1, I0, f1, f0, cam0):
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    s = torch.zeros(1, dtype=torch.float64, device="cuda")
    c = torch.zeros(1, dtype=torch.int64, device="cuda")
    nsm.temporal_instability(d(I1), d(I0), d(f1.pos4), d(f1.nrm4), d(f0.pos4), d(f0.nrm4), cam0, s, c)
    torch.cuda.synchronize()
    return float(s.item()), int(c.item())


def test_instability_moving_light_and_objects():
    H, W = 96, 128
    frames = scenegen.temporal_sequence(H, W, 128, 128, 16, 21, n_frames=4)
    imgs = _images(frames, 3)
    cam = scenegen.camera_vector(frames[0].scene, H, W)
    for t in range(1, 4):
        s, c = _gpu_pair(imgs[t], imgs[t - 1], frames[t], frames[t - 1], cam)
        rs, rc = TM.instability_pair(imgs[t], imgs[t - 1], frames[t].pos4, frames[t].nrm4, frames[t - 1].pos4,
                                     frames[t - 1].nrm4, cam)
        assert c == rc
        assert s == pytest.approx(rs, rel=1e-6)
        assert 0.9 * H * W < c < H * W  # moving objects lose a few pixels


@pytest.mark.parametrize("seed", [4, 17])
def test_instability_moving_camera(seed):
    H, W = 120, 200
    s1 = scenegen.random_scene(seed, 24)
    s0 = scenegen.perturbed(s1, scenegen.SplitMix64(seed))
    f1, f0 = scenegen.render_frame(s1, H, W, 64, 64), scenegen.render_frame(s0, H, W, 64, 64)
    I1, I0 = _images([f1, f0], seed)
    cam0 = scenegen.camera_vector(s0, H, W)
    s, c = _gpu_pair(I1, I0, f1, f0, cam0)
    rs, rc = TM.instability_pair(I1, I0, f1.pos4, f1.nrm4, f0.pos4, f0.nrm4, cam0)
    assert c == rc and c > 0.5 * H * W
    assert s == pytest.approx(rs, rel=1e-6)


def test_instability_identical_frames_and_empty():
    f = scenegen.render_frame(scenegen.random_scene(2, 8), 64, 64, 64, 64)
    I = _images([f], 1)[0]
    s, c = _gpu_pair(I, I, f, f, scenegen.camera_vector(f.scene, 64, 64))
    assert s == 0.0 and c == 64 * 64
    z = torch.zeros(1, dtype=torch.float64, device="cuda")
    n = torch.zeros(1, dtype=torch.int64, device="cuda")
    e = torch.empty((0, 4), device="cuda")
    nsm.temporal_instability(torch.empty((0, 5), device="cuda"), torch.empty((0, 5), device="cuda"), e, e, e, e,
                             np.zeros(14), z, n)
    torch.cuda.synchronize()
    assert z.item() == 0.0 and n.item() == 0


@pytest.mark.parametrize("seed,S", [(21, 256), (7, 512)])
def test_penumbra_histogram_and_depth(seed, S):
    H, W = 96, 160
    f = scenegen.soft_frame(H, W, S, S, 24, seed)
    df = DeviceFrame(f)
    _, _, _, blk = run_features(df, blocker=True)
    th = scenegen.camera_vector(f.scene, H, W)[12]
    bin_px, nbins = 0.5, 256
    hist = torch.zeros(nbins, dtype=torch.int32, device="cuda")
    nsm.penumbra_histogram(blk, df.pos4, th, bin_px, hist)
    nsm.penumbra_histogram(blk, df.pos4, th, bin_px, hist)  # accumulates
    torch.cuda.synchronize()
    h = hist.cpu().numpy().astype(np.int64)
    # oracle: exact blocker search, FP64 penumbra model, FP64 projection
    zmin, zmax, found = G.blocker_search(f.pos4, f.sm, f.view_proj, f.light_pos, f.light_radius, f.tan_half_fov,
                                         f.z_far, f.bias)
    zf = np.linalg.norm(f.light_pos.astype(np.float64) - f.pos4[..., :3].astype(np.float64), axis=-1)
    xa, xb = G.penumbra_width(zf[found], zmin[found], zmax[found], f.light_radius)
    w = TM.screen_width_px(xa + xb, f.pos4[..., 3][found], H, th)
    ref = 2 * TM.penumbra_histogram(w, bin_px, nbins)
    assert h.sum() == ref.sum() == 2 * int(found.sum()) > 0
    q = w / bin_px
    near = np.abs(q - np.round(q)) <= 1e-4 * np.maximum(1.0, np.abs(q))
    assert np.abs(h - ref).sum() <= 2 * 2 * int(near.sum())
    p_gpu, l_gpu = nsm.depth_for_penumbra(h, bin_px)
    p_ref = TM.p95_from_histogram(ref, bin_px)
    assert abs(p_gpu - p_ref) <= bin_px
    assert l_gpu == TM.depth_for_width(p_gpu)


def test_analysis_rejects_bad_arguments():
    x = torch.zeros((4, 4), device="cuda")
    with pytest.raises(nsm.NSMError):
        nsm.penumbra_histogram(torch.zeros((3, 4, 4), device="cuda"), torch.zeros((4, 4, 4), device="cuda"), 0.0,
                               0.5, torch.zeros(8, dtype=torch.int32, device="cuda"))
    with pytest.raises(nsm.NSMError):
        nsm.temporal_instability(x, x, torch.zeros((4, 4, 4)), x, x, x, np.zeros(14),
                                 torch.zeros(1, dtype=torch.float64, device="cuda"),
                                 torch.zeros(1, dtype=torch.int64, device="cuda"))
