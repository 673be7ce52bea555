"""GPU parity of nsm_infer (gather fused into the network) against the FP64
oracle on the same seeded inputs.

FP32 form: max-abs <= 1e-4 on visibility against the FP64 forward.
BF16 form (compensated: every stored value a BF16 hi + lo pair): (a) against
the oracle forward rounded the same way at every storage point (features,
weights, the 3x3 -> 1x1 intermediate, every level output; the level-0 decoder
on the coarse grid with rounded effective weights and its outermost ring
exact): MSE <= 1e-8 and max-abs <= 1e-3 -- what is left is FP32 accumulation
order; (b) against the exact FP64 forward: MSE <= 1e-4 and max-abs <= 1e-2."""
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


def _features(f):
    feat, _, _ = G.features(f.pos4, f.nrm4, f.sm, f.view_proj, f.light_pos, f.cam_pos, f.r_hat, f.z_far, f.bias)
    return feat


def _theta(seed=3):
    return scenegen.he_init_weights(seed, N.layer_table(3)).astype(np.float32)


def _run(ctx, f, theta, precision):
    w = nsm.Weights(ctx, theta)
    vis = run_infer(ctx, w, DeviceFrame(f), precision).cpu().numpy().astype(np.float64)
    assert np.isfinite(vis).all() and (vis >= 0).all() and (vis <= 1).all()
    return vis


def _check(ctx, f, theta, precision):
    vis = _run(ctx, f, theta, precision)
    feat = _features(f)
    th64 = theta.astype(np.float64)
    ref = N.forward(feat, th64)
    err = np.abs(vis - ref)
    if precision == nsm.NSM_FP32:
        assert err.max() <= 1e-4, err.max()
    else:
        qref = N.forward_rounded(feat, th64, N.round_bf16_pair, rnd_in=N.round_bf16_pair, coarse_dec0=True)
        qerr = np.abs(vis - qref)
        assert float(np.mean(qerr ** 2)) <= 1e-8, float(np.mean(qerr ** 2))
        assert qerr.max() <= 1e-3, qerr.max()
        assert float(np.mean(err ** 2)) <= 1e-4
        assert err.max() <= 1e-2, err.max()
    return vis, err


@pytest.mark.parametrize("precision", [nsm.NSM_FP32, nsm.NSM_BF16])
def test_infer_config1_256(ctx, precision):
    f = scenegen.hard_frame(256, 256, 512, 512, 8, 1)
    _check(ctx, f, _theta(), precision)


@pytest.mark.parametrize("precision", [nsm.NSM_FP32, nsm.NSM_BF16])
def test_infer_ragged_tiles(ctx, precision):
    # sizes that leave partial tiles at every level (and an odd bottleneck size)
    _check(ctx, scenegen.soft_frame(68, 132, 300, 200, 8, 5), _theta(4), precision)
    _check(ctx, scenegen.soft_frame(4, 4, 16, 16, 3, 6), _theta(5), precision)
    _check(ctx, scenegen.hard_frame(260, 388, 256, 256, 8, 7), _theta(6), precision)


@pytest.mark.parametrize("precision", [nsm.NSM_FP32, nsm.NSM_BF16])
def test_infer_1080p_full_size(ctx, precision):
    f = scenegen.hard_frame(1080, 1920, 2048, 2048, 64, 11)
    _check(ctx, f, _theta(), precision)


def test_infer_bf16_vs_fp64(ctx):
    """Error of the BF16 form against the exact FP64 forward at 256^2, hard
    and soft shadows: max-abs within 1e-2 and MSE within 1e-4."""
    for f in (scenegen.hard_frame(256, 256, 512, 512, 8, 1), scenegen.soft_frame(256, 256, 512, 512, 8, 21)):
        theta = _theta(3)
        vis = _run(ctx, f, theta, nsm.NSM_BF16)
        ref = N.forward(_features(f), theta.astype(np.float64))
        err = np.abs(vis - ref)
        assert float(np.mean(err ** 2)) <= 1e-4
        assert err.max() <= 1e-2, err.max()


@pytest.mark.parametrize("precision", [nsm.NSM_FP32, nsm.NSM_BF16])
def test_infer_trained_weights(ctx, precision):
    """The seeded oracle-trained weights (saturating outputs, steep shadow
    edges): FP32 within 1e-4 of the FP64 forward, BF16 within its rounding
    model and within 1e-2 max-abs / 1e-4 MSE of the FP64 forward."""
    theta = scenegen.trained_weights()
    for f in (scenegen.hard_frame(256, 256, 512, 512, 8, 1), scenegen.soft_frame(256, 256, 512, 512, 8, 21),
              scenegen.soft_frame(68, 132, 300, 200, 8, 5)):
        _check(ctx, f, theta, precision)


def test_infer_trained_weights_1080p_soft_bf16(ctx):
    """Full-size 1080p soft frame with the trained weights, BF16 against FP64."""
    f = scenegen.soft_frame(1080, 1920, 2048, 2048, 64, 21)
    theta = scenegen.trained_weights()
    vis = _run(ctx, f, theta, nsm.NSM_BF16)
    err = np.abs(vis - N.forward(_features(f), theta.astype(np.float64)))
    assert err.max() <= 1e-2 and float(np.mean(err ** 2)) <= 1e-4, (err.max(), float(np.mean(err ** 2)))


@pytest.fixture(scope="module")
def frame_2160p():
    return scenegen.soft_frame(2160, 3840, 4096, 4096, 64, 31)


@pytest.mark.parametrize("precision", [nsm.NSM_FP32, nsm.NSM_BF16])
def test_infer_2160p_4096_map_bands(ctx, frame_2160p, precision):
    """The largest serving size (3840 x 2160 view, 4096^2 map, soft emitter,
    trained weights) against the FP64 oracle on row bands at the top, middle
    and bottom edge."""
    from gpu_helpers import oracle_band
    f = frame_2160p
    theta = scenegen.trained_weights()
    vis = _run(ctx, f, theta, precision)
    th64 = theta.astype(np.float64)
    for y0, y1 in ((0, 40), (1060, 1100), (2120, 2160)):
        err = np.abs(vis[y0:y1] - oracle_band(f, th64, y0, y1))
        if precision == nsm.NSM_FP32:
            assert err.max() <= 1e-4, (y0, err.max())
        else:
            assert err.max() <= 1e-2 and float(np.mean(err ** 2)) <= 1e-4, (y0, err.max())


def test_infer_fp8_trained_weights_follow_rounding_model(ctx):
    theta = scenegen.trained_weights()
    f = scenegen.soft_frame(256, 256, 512, 512, 8, 21)
    vis = _run(ctx, f, theta, nsm.NSM_FP8)
    q = _fp8_model(_features(f), theta)
    assert float(np.mean((vis - q) ** 2)) <= 1e-6


def test_infer_rejects_bad_shapes_and_workspace(ctx):
    f = scenegen.hard_frame(8, 8, 8, 8, 2, 1)
    df = DeviceFrame(f)
    w = nsm.Weights(ctx, _theta())
    vis = torch.empty((8, 8), device="cuda")
    small = torch.empty((16,), dtype=torch.uint8, device="cuda")
    with pytest.raises(nsm.NSMError) as ei:
        nsm.nsm_infer(ctx, df.frame, w, nsm.NSM_FP32, small, vis)
    assert ei.value.status == 8
    df.frame.W = 6
    with pytest.raises(nsm.NSMError) as ei:
        nsm.nsm_infer(ctx, df.frame, w, nsm.NSM_FP32, small, vis)
    assert ei.value.status == 2


@pytest.mark.parametrize("precision", [nsm.NSM_FP32, nsm.NSM_BF16])
def test_infer_host_entry_point_matches_device_call(ctx, precision):
    f = scenegen.soft_frame(64, 128, 256, 256, 8, 9)
    theta = _theta(7)
    w = nsm.Weights(ctx, theta)
    dev = run_infer(ctx, w, DeviceFrame(f), precision).cpu().numpy()
    from gpu_helpers import light_desc
    hf = nsm.make_frame(f.pos4, f.nrm4, f.sm, light_desc(f), f.cam_pos)
    stage = torch.empty((nsm.nsm_infer_host_stage_bytes(f.H, f.W, f.Hs, f.Ws),), dtype=torch.uint8, device="cuda")
    ws = torch.empty((nsm.nsm_infer_workspace_bytes(f.H, f.W, precision),), dtype=torch.uint8, device="cuda")
    out = np.empty((f.H, f.W), np.float32)
    nsm.nsm_infer_host(ctx, hf, w, precision, stage, ws, out)
    np.testing.assert_array_equal(out, dev)


def _fp8_model(feat, theta):
    """The oracle forward rounded as the FP8 form stores values: E4M3 features,
    3x3 -> 1x1 intermediates and level outputs (unit scale), E4M3 weights with
    one scale per output channel."""
    return N.forward_rounded(feat, theta.astype(np.float64), N.round_e4m3, rnd_in=N.round_e4m3,
                             rnd_w=N.round_e4m3_per_out_channel, rnd_mid=N.round_e4m3)


@pytest.mark.parametrize("case", ["hard256", "soft256", "ragged"])
def test_infer_fp8_follows_its_rounding_model(ctx, case):
    """FP8 form against the oracle with the same E4M3 storage points: what is
    left is FP32 accumulation order, which can move a stored value to the
    neighbouring E4M3 value (1/16 relative steps), so the bound is on the MSE
    with a looser max.  Against FP64 this form misses the 1e-2 / 1e-4 bar
    with He-init weights (~0.15 max-abs, ~4e-4 MSE; reported by bench.py);
    the test only checks it stays in that regime."""
    f = {"hard256": lambda: scenegen.hard_frame(256, 256, 512, 512, 8, 1),
         "soft256": lambda: scenegen.soft_frame(256, 256, 512, 512, 8, 21),
         "ragged": lambda: scenegen.soft_frame(68, 132, 300, 200, 8, 5)}[case]()
    theta = _theta(3)
    vis = _run(ctx, f, theta, nsm.NSM_FP8)
    feat = _features(f)
    q = _fp8_model(feat, theta)
    ref = N.forward(feat, theta.astype(np.float64))
    qerr = np.abs(vis - q)
    err = np.abs(vis - ref)
    print(f"fp8 {case}: vs model max {qerr.max():.3e} mse {np.mean(qerr ** 2):.3e}; "
          f"vs fp64 max {err.max():.3e} mse {np.mean(err ** 2):.3e}")
    assert float(np.mean(qerr ** 2)) <= 1e-6, float(np.mean(qerr ** 2))
    assert qerr.max() <= 0.1, qerr.max()
    assert float(np.mean(err ** 2)) <= 5e-3


def test_infer_soft_temporal_sequence_per_frame(ctx):
    """The soft temporal sequence (emitter orbiting 2 degrees / frame, 4 objects
    moving 0.01 / frame), 8 frames at 256^2: every frame's BF16 output within
    1e-2 max-abs / 1e-4 MSE of the FP64 forward, the FP8 output on its rounding
    model."""
    theta = _theta(3)
    for f in scenegen.temporal_sequence(256, 256, 512, 512, 12, 21):
        feat = _features(f)
        ref = N.forward(feat, theta.astype(np.float64))
        vb = _run(ctx, f, theta, nsm.NSM_BF16)
        e = np.abs(vb - ref)
        assert e.max() <= 1e-2 and float(np.mean(e ** 2)) <= 1e-4, (e.max(), float(np.mean(e ** 2)))
        v8 = _run(ctx, f, theta, nsm.NSM_FP8)
        assert float(np.mean((v8 - _fp8_model(feat, theta)) ** 2)) <= 1e-6

