"""GPU parity of nsm_infer (gather fused into the network) against the FP64
oracle forward on the same seeded inputs.  Tolerances: FP32 form max-abs
<= 1e-4 on visibility; BF16 / FP8 forms max-abs <= 1e-2 and MSE <= 1e-4."""
import numpy as np
import pytest

import scenegen
from oracle import gather as G
from oracle import network as N

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2301_05262_gb300 as nsm  # noqa: E402
from gpu_helpers import DeviceFrame, run_infer  # noqa: E402

TOL = {nsm.NSM_FP32: (1e-4, None), nsm.NSM_BF16: (1e-2, 1e-4), nsm.NSM_FP8: (1e-2, 1e-4)}


@pytest.fixture(scope="module")
def ctx():
    c = nsm.Context()
    yield c
    c.check()
    c.close()


def _oracle_vis(f, theta):
    feat, _, _ = G.features(f.pos4, f.nrm4, f.sm, f.view_proj, f.light_pos, f.cam_pos, f.r_hat, f.z_far, f.bias)
    return N.forward(feat, theta)


def _theta(seed=3):
    return scenegen.he_init_weights(seed, N.layer_table(3))


def _compare(ctx, f, theta, precision, report=None):
    w = nsm.Weights(ctx, theta.astype(np.float32))
    vis = run_infer(ctx, w, DeviceFrame(f), precision).cpu().numpy()
    ref = _oracle_vis(f, theta.astype(np.float32).astype(np.float64))
    err = np.abs(vis.astype(np.float64) - ref)
    mx, mse = err.max(), float(np.mean(err ** 2))
    if report is not None:
        report.append((f.H, f.W, precision, mx, mse))
    tol_max, tol_mse = TOL[precision]
    assert mx <= tol_max, (precision, mx)
    if tol_mse is not None:
        assert mse <= tol_mse, (precision, mse)
    assert np.isfinite(vis).all() and (vis >= 0).all() and (vis <= 1).all()
    return vis, ref


@pytest.mark.parametrize("precision", [nsm.NSM_FP32])
def test_infer_config1_256(ctx, precision):
    f = scenegen.hard_frame(256, 256, 512, 512, 8, 1)
    _compare(ctx, f, _theta(), precision)


@pytest.mark.parametrize("precision", [nsm.NSM_FP32])
def test_infer_ragged_tiles(ctx, precision):
    # sizes that leave partial tiles at every level (and an odd bottleneck size)
    f = scenegen.soft_frame(68, 132, 300, 200, 8, 5)
    _compare(ctx, f, _theta(4), precision)
    f = scenegen.soft_frame(4, 4, 16, 16, 3, 6)
    _compare(ctx, f, _theta(5), precision)


@pytest.mark.parametrize("precision", [nsm.NSM_FP32])
def test_infer_1080p_full_size(ctx, precision):
    f = scenegen.hard_frame(1080, 1920, 2048, 2048, 64, 11)
    _compare(ctx, f, _theta(), precision)


def test_infer_rejects_bad_shapes_and_workspace(ctx):
    f = scenegen.hard_frame(8, 8, 8, 8, 2, 1)
    df = DeviceFrame(f)
    w = nsm.Weights(ctx, _theta().astype(np.float32))
    vis = torch.empty((8, 8), device="cuda")
    small = torch.empty((16,), dtype=torch.uint8, device="cuda")
    with pytest.raises(nsm.NSMError) as ei:
        nsm.nsm_infer(ctx, df.frame, w, nsm.NSM_FP32, small, vis)
    assert ei.value.status == 8
    df.frame.W = 6
    with pytest.raises(nsm.NSMError) as ei:
        nsm.nsm_infer(ctx, df.frame, w, nsm.NSM_FP32, small, vis)
    assert ei.value.status == 2


def test_infer_host_entry_point_matches_device_call(ctx):
    f = scenegen.soft_frame(64, 128, 256, 256, 8, 9)
    theta = _theta(7)
    w = nsm.Weights(ctx, theta.astype(np.float32))
    dev = run_infer(ctx, w, DeviceFrame(f), nsm.NSM_FP32).cpu().numpy()
    from gpu_helpers import light_desc
    hf = nsm.make_frame(f.pos4, f.nrm4, f.sm, light_desc(f), f.cam_pos)
    stage = torch.empty((nsm.nsm_infer_host_stage_bytes(f.H, f.W, f.Hs, f.Ws),), dtype=torch.uint8, device="cuda")
    ws = torch.empty((nsm.nsm_infer_workspace_bytes(f.H, f.W, nsm.NSM_FP32),), dtype=torch.uint8, device="cuda")
    out = np.empty((f.H, f.W), np.float32)
    nsm.nsm_infer_host(ctx, hf, w, nsm.NSM_FP32, stage, ws, out)
    np.testing.assert_array_equal(out, dev)
