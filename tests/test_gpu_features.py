"""GPU parity of the feature gather (nsm_features) against the oracle:
texel indices and hard bits bit-exact, features within FP32 rounding,
blocker search exact (window minima / maxima are texel values)."""
import numpy as np
import pytest

import scenegen
from oracle import gather as G

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
from gpu_helpers import DeviceFrame, run_features, unpack_hard_bits  # noqa: E402


def _check_frame(f, blocker=False, sample=None):
    df = DeviceFrame(f)
    feat, tex, hard, blk = run_features(df, blocker=blocker)
    feat = feat.cpu().numpy()
    tex = tex.cpu().numpy()
    hard = unpack_hard_bits(hard.cpu().numpy().view(np.uint32), f.H * f.W).reshape(f.H, f.W)
    ofeat, otex, ohard = G.features(f.pos4, f.nrm4, f.sm, f.view_proj, f.light_pos, f.cam_pos,
                                    f.r_hat, f.z_far, f.bias)
    # bit-exact: texel choice and hard depth test
    np.testing.assert_array_equal(tex, otex.astype(np.int32))
    np.testing.assert_array_equal(hard, ohard)
    # features: FP32 evaluation vs FP64 from the same inputs
    err = np.abs(feat - ofeat)
    scale = np.maximum(1.0, np.abs(ofeat))
    assert (err / scale).max() < 2e-6, (err / scale).max()
    if blocker:
        blk = blk.cpu().numpy()
        idx = sample if sample is not None else np.s_[:, :]
        sub = f.pos4[idx]
        zmin, zmax, found = G.blocker_search(sub, f.sm, f.view_proj, f.light_pos, f.light_radius,
                                             f.tan_half_fov, f.z_far, f.bias)
        np.testing.assert_array_equal(blk[0][idx], zmin)
        np.testing.assert_array_equal(blk[1][idx], zmax)
        zf = G.emitter_distance_fp32(sub[..., :3], f.light_pos)
        xa, xb = G.penumbra_width(zf, np.where(found, zmin, 1.0), np.where(found, zmax, 1.0), f.light_radius)
        width = np.where(found, xa + xb, 0.0)
        np.testing.assert_allclose(blk[2][idx], width, rtol=2e-4, atol=2e-5)
        assert found.mean() > 0.0
    return tex, hard


def test_features_config1_256():
    f = scenegen.hard_frame(256, 256, 512, 512, 8, 1)
    tex, hard = _check_frame(f)
    assert (tex >= 0).mean() > 0.5 and (~hard).sum() > 100


def test_features_ragged_sizes_and_tail_word():
    # H*W not a multiple of 32 (last hard-bit word partly used), odd sizes
    f = scenegen.soft_frame(37, 53, 333, 129, 8, 4)
    _check_frame(f, blocker=True)


def test_features_soft_blocker_search():
    f = scenegen.soft_frame(64, 96, 512, 512, 16, 21)
    _check_frame(f, blocker=True)


def test_features_1080p_full_size():
    f = scenegen.hard_frame(1080, 1920, 2048, 2048, 64, 11)
    _check_frame(f)


def test_features_1080p_blocker_sampled_rows():
    # 16-row bands of blocker CTAs (windows up to 65 texels, both table levels), top and bottom edges
    f = scenegen.soft_frame(1080, 1920, 2048, 2048, 64, 21)
    for rows in (np.s_[496:512, :], np.s_[1064:1080, :], np.s_[0:2, :]):
        _check_frame(f, blocker=True, sample=rows)


def test_features_hard_blocker_point_light_windows():
    # point light: k = 0, one-texel windows (the direct-scan branch)
    f = scenegen.hard_frame(128, 160, 256, 256, 8, 3)
    _check_frame(f, blocker=True)


def test_features_blocker_wide_texel_spacing():
    # few pixels over a large map: neighbouring windows barely overlap
    f = scenegen.soft_frame(48, 64, 2048, 2048, 16, 22)
    _check_frame(f, blocker=True)


def test_features_empty_frame():
    import paper_2301_05262_gb300 as nsm
    f = scenegen.hard_frame(4, 4, 8, 8, 2, 1)
    df = DeviceFrame(f)
    df.frame.H = 0
    feat = torch.empty((4, 1), device="cuda")
    nsm.nsm_features(df.frame, feat)  # nothing to do, no error


def test_features_rejects_host_pointer():
    import paper_2301_05262_gb300 as nsm
    f = scenegen.hard_frame(8, 8, 8, 8, 2, 1)
    fr = nsm.make_frame(f.pos4, f.nrm4, f.sm, __import__("gpu_helpers").light_desc(f), f.cam_pos)
    feat = torch.empty((4, 8, 8), device="cuda")
    with pytest.raises(nsm.NSMError) as ei:
        nsm.nsm_features(fr, feat)
    assert ei.value.status == 1


def test_features_blocker_map_smaller_than_a_square():
    # a 7 x 6 map: every 8 x 8 / 4 x 4 table entry near the edges is clipped; windows < 8 texels
    f = scenegen.soft_frame(24, 40, 6, 7, 6, 24)
    _check_frame(f, blocker=True)


def test_features_2160p_4096_map_blocker_sampled_rows():
    # the largest configuration: 256 MiB of table scratch, windows on a denser texel grid
    f = scenegen.soft_frame(2160, 3840, 4096, 4096, 64, 31)
    for rows in (np.s_[1072:1088, :], np.s_[2144:2160, :]):
        _check_frame(f, blocker=True, sample=rows)


def test_features_blocker_with_caller_workspace():
    # the no-allocation entry point gives the same bits as the pooled one
    import paper_2301_05262_gb300 as nsm
    f = scenegen.soft_frame(64, 96, 512, 512, 16, 21)
    df = DeviceFrame(f)
    _, _, _, blk = run_features(df, blocker=True)
    feat = torch.empty((4, f.H, f.W), device="cuda")
    blk2 = torch.empty_like(blk)
    ws = torch.empty((nsm.nsm_features_workspace_bytes(512, 512),), dtype=torch.uint8, device="cuda")
    nsm.nsm_features_ws(df.frame, feat, None, None, blk2, ws)
    torch.cuda.synchronize()
    assert torch.equal(blk, blk2)
    with pytest.raises(nsm.NSMError) as ei:
        nsm.nsm_features_ws(df.frame, feat, None, None, blk2, ws[: ws.numel() // 2])
    assert ei.value.status == 8
