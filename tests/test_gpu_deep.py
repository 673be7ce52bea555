"""GPU parity of the deeper networks (Sec. 3.6: 2 to 7 levels) against the
FP64 oracle forward with the same number of levels: the FP32 form within
1e-4 max-abs on visibility; the 3-level result equals the fused FP32 form's
to rounding (both FP32: within the sum of their distances to FP64); the
tensor-core form (compensated BF16, 3 to 7 levels) within 2e-3 max-abs and
1e-8 MSE, under the 1e-2 / 1e-4 bar of the BF16 inference; the three-term
FP8 form within that 1e-2 / 1e-4 bar, on the trained 3-level weights too."""
import numpy as np
import pytest

import scenegen
from oracle import gather as G
from oracle import network as N

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2301_05262_gb300 as nsm  # noqa: E402
from gpu_helpers import DeviceFrame, run_infer  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = nsm.Context()
    yield c
    c.check()
    c.close()


def _deep(ctx, df, theta, L, precision=None):
    f = df.f
    ws = torch.empty((nsm.nsm_infer_deep_workspace_bytes(f.H, f.W, L, precision),), dtype=torch.uint8, device="cuda")
    vis = torch.empty((f.H, f.W), device="cuda")
    nsm.nsm_infer_deep(ctx, df.frame, torch.from_numpy(theta).cuda(), L, ws, vis, precision=precision)
    torch.cuda.synchronize()
    ctx.check()
    return vis.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("L,H,W", [(2, 68, 132), (3, 96, 128), (4, 64, 200), (5, 128, 192), (6, 128, 192),
                                   (7, 128, 192)])
def test_deep_forward_matches_oracle(ctx, L, H, W):
    f = scenegen.soft_frame(H, W, 256, 256, 16, 40 + L)
    theta = scenegen.he_init_weights(L, N.layer_table(L)).astype(np.float32)
    vis = _deep(ctx, DeviceFrame(f), theta, L)
    feat, _, _ = G.features(f.pos4, f.nrm4, f.sm, f.view_proj, f.light_pos, f.cam_pos, f.r_hat, f.z_far, f.bias)
    ref = N.forward(feat, theta.astype(np.float64), levels=L)
    err = np.abs(vis - ref)
    print(f"L={L} {H}x{W}: max {err.max():.2e}")
    assert np.isfinite(vis).all() and err.max() <= 1e-4, err.max()


@pytest.mark.parametrize("L,H,W", [(3, 96, 136), (5, 128, 192), (5, 256, 656), (6, 128, 256), (7, 128, 192),
                                   (7, 192, 576), (5, 832, 1280)])
def test_deep_bf16_forward_matches_oracle(ctx, L, H, W):
    """Levels 0 and 1 on the BF16 stage kernels, levels 2 .. L-1 on the tcgen05
    layers: at 256 x 656 the level-2 rows are 164 = 128 + 36 pixels (two
    M tiles, ragged); 7 levels reach 1024 channels (the bottleneck's 3x3 has
    32 input chunks of 16 and 16 output blocks of 64).  At 832 x 1280 (152
    SMs) the 3x3 layers take tiles of 4 image rows at level 2, 2 at level 3
    and 1 at level 4 (the largest row count that still gives every SM a
    tile), so every tile height is checked against the oracle."""
    f = scenegen.soft_frame(H, W, 256, 256, 16, 60 + L)
    theta = scenegen.he_init_weights(L, N.layer_table(L)).astype(np.float32)
    vis = _deep(ctx, DeviceFrame(f), theta, L, nsm.NSM_BF16)
    feat, _, _ = G.features(f.pos4, f.nrm4, f.sm, f.view_proj, f.light_pos, f.cam_pos, f.r_hat, f.z_far, f.bias)
    ref = N.forward(feat, theta.astype(np.float64), levels=L)
    err = np.abs(vis - ref)
    mse = float(np.mean(err ** 2))
    print(f"BF16 L={L} {H}x{W}: max {err.max():.2e}, MSE {mse:.2e}")
    assert np.isfinite(vis).all() and err.max() <= 2e-3 and mse <= 1e-8, (err.max(), mse)


@pytest.mark.parametrize("kind,H,W,S,n,seed", [("hard", 256, 256, 512, 8, 1), ("soft", 256, 256, 512, 8, 3),
                                                ("hard", 200, 320, 1024, 64, 5), ("soft", 200, 320, 1024, 64, 7)])
def test_fp8_three_term_trained_network_meets_the_bar(ctx, kind, H, W, S, n, seed):
    """The three-term E4M3 form of the trained 3-level network against the FP64
    forward: within the 1e-2 max-abs / 1e-4 MSE bar (the oracle's rounding of
    the same recipe at every storage point gives 1.2e-3 / 7e-10 on these
    frames; the single-term E4M3 form misses the bar by two orders)."""
    f = (scenegen.hard_frame if kind == "hard" else scenegen.soft_frame)(H, W, S, S, n, seed)
    theta = scenegen.trained_weights()
    vis = _deep(ctx, DeviceFrame(f), theta, 3, nsm.NSM_FP8)
    feat, _, _ = G.features(f.pos4, f.nrm4, f.sm, f.view_proj, f.light_pos, f.cam_pos, f.r_hat, f.z_far, f.bias)
    ref = N.forward(feat, theta.astype(np.float64))
    err = np.abs(vis - ref)
    mse = float(np.mean(err ** 2))
    print(f"FP8x3 trained {kind} {H}x{W}: max {err.max():.2e}, MSE {mse:.2e}")
    assert np.isfinite(vis).all() and err.max() <= 1e-2 and mse <= 1e-4, (err.max(), mse)
    assert err.max() <= 5e-3 and mse <= 1e-8, (err.max(), mse)


@pytest.mark.parametrize("L,H,W", [(2, 68, 132), (3, 96, 136), (5, 128, 192), (7, 128, 192)])
def test_fp8_three_term_deep_forward_matches_oracle(ctx, L, H, W):
    f = scenegen.soft_frame(H, W, 256, 256, 16, 80 + L)
    theta = scenegen.he_init_weights(L, N.layer_table(L)).astype(np.float32)
    vis = _deep(ctx, DeviceFrame(f), theta, L, nsm.NSM_FP8)
    feat, _, _ = G.features(f.pos4, f.nrm4, f.sm, f.view_proj, f.light_pos, f.cam_pos, f.r_hat, f.z_far, f.bias)
    ref = N.forward(feat, theta.astype(np.float64), levels=L)
    err = np.abs(vis - ref)
    mse = float(np.mean(err ** 2))
    print(f"FP8x3 L={L} {H}x{W}: max {err.max():.2e}, MSE {mse:.2e}")
    assert np.isfinite(vis).all() and err.max() <= 1e-2 and mse <= 1e-4, (err.max(), mse)


def test_deep_bf16_rejects_two_levels(ctx):
    f = scenegen.hard_frame(64, 64, 64, 64, 4, 2)
    theta = scenegen.he_init_weights(2, N.layer_table(2)).astype(np.float32)
    ws = torch.empty((1 << 20,), dtype=torch.uint8, device="cuda")
    with pytest.raises(nsm.NSMError) as ei:
        nsm.nsm_infer_deep(ctx, DeviceFrame(f).frame, torch.from_numpy(theta).cuda(), 2, ws,
                           torch.empty((64, 64), device="cuda"), precision=nsm.NSM_BF16)
    assert ei.value.status == 7  # NSM_ERR_UNSUPPORTED


def test_deep_three_levels_equals_the_fused_form(ctx):
    f = scenegen.hard_frame(128, 256, 512, 512, 8, 1)
    theta = scenegen.trained_weights()
    df = DeviceFrame(f)
    w = nsm.Weights(ctx, theta)
    fused = run_infer(ctx, w, df, nsm.NSM_FP32).cpu().numpy().astype(np.float64)
    # two FP32 evaluations of the same network with different summation and
    # contraction orders, each within ~5e-6 of FP64 at these sizes (the parity
    # tests above): their distance is bounded by the sum, 1e-5
    d = np.abs(_deep(ctx, df, theta, 3) - fused)
    print(f"deep vs fused 3-level: max {d.max():.3e}, mean {d.mean():.3e}")
    assert d.max() <= 1e-5


def test_deep_rejects_bad_shapes(ctx):
    f = scenegen.hard_frame(40, 64, 64, 64, 4, 2)   # 40 is not a multiple of 16
    df = DeviceFrame(f)
    theta = scenegen.he_init_weights(5, N.layer_table(5)).astype(np.float32)
    ws = torch.empty((nsm.nsm_infer_deep_workspace_bytes(40, 64, 5),), dtype=torch.uint8, device="cuda")
    with pytest.raises(nsm.NSMError) as ei:
        nsm.nsm_infer_deep(ctx, df.frame, torch.from_numpy(theta).cuda(), 5, ws, torch.empty((40, 64), device="cuda"))
    assert ei.value.status == 2
    with pytest.raises(nsm.NSMError):
        nsm.nsm_infer_deep(ctx, df.frame, torch.from_numpy(theta).cuda(), 8, ws, torch.empty((40, 64), device="cuda"))


@pytest.mark.parametrize("precision,L,H,W", [(0, 2, 68, 132), (0, 5, 128, 192), (1, 3, 96, 136), (1, 5, 256, 656),
                                             (2, 3, 96, 136), (2, 7, 128, 192)])
def test_packed_weights_equal_the_per_call_packing(ctx, precision, L, H, W):
    """nsm_infer_deep_packed from weights packed once gives the same bits as
    nsm_infer_deep_ex, which packs the same vector per call, in every form
    (FP32 = 0, BF16 = 1, FP8 three-term = 2), with the smaller workspace;
    re-packing from a device vector (load_device) follows the new weights."""
    f = scenegen.soft_frame(H, W, 256, 256, 16, 80 + L)
    df = DeviceFrame(f)
    theta = scenegen.he_init_weights(L, N.layer_table(L)).astype(np.float32)
    ex = _deep(ctx, df, theta, L, precision)
    w = nsm.DeepWeights(ctx, theta, L, precision)
    ws = torch.empty((nsm.nsm_infer_deep_packed_workspace_bytes(H, W, L, precision),), dtype=torch.uint8,
                     device="cuda")
    vis = torch.empty((H, W), device="cuda")
    nsm.nsm_infer_deep_packed(ctx, df.frame, w, ws, vis)
    torch.cuda.synchronize()
    ctx.check()
    assert np.array_equal(vis.cpu().numpy().astype(np.float64), ex)
    theta2 = (theta * np.float32(0.75)).astype(np.float32)
    w.load_device(torch.from_numpy(theta2).cuda())
    nsm.nsm_infer_deep_packed(ctx, df.frame, w, ws, vis)
    torch.cuda.synchronize()
    ctx.check()
    assert np.array_equal(vis.cpu().numpy().astype(np.float64), _deep(ctx, df, theta2, L, precision))
    w.close()


def test_packed_weights_reject_bad_arguments(ctx):
    theta = scenegen.he_init_weights(3, N.layer_table(3)).astype(np.float32)
    with pytest.raises(nsm.NSMError) as ei:
        nsm.DeepWeights(ctx, theta[:-1], 3, nsm.NSM_FP32)
    assert ei.value.status == 2  # NSM_ERR_SHAPE
    with pytest.raises(nsm.NSMError) as ei:
        nsm.DeepWeights(ctx, scenegen.he_init_weights(2, N.layer_table(2)).astype(np.float32), 2, nsm.NSM_BF16)
    assert ei.value.status == 7  # NSM_ERR_UNSUPPORTED
    w = nsm.DeepWeights(ctx, theta, 3, nsm.NSM_BF16)
    f = scenegen.hard_frame(64, 64, 64, 64, 4, 2)
    need = nsm.nsm_infer_deep_packed_workspace_bytes(64, 64, 3, nsm.NSM_BF16)
    ws = torch.empty((need - 256,), dtype=torch.uint8, device="cuda")
    with pytest.raises(nsm.NSMError):
        nsm.nsm_infer_deep_packed(ctx, DeviceFrame(f).frame, w, ws, torch.empty((64, 64), device="cuda"))
    w.close()
