"""GPU parity of the space-to-depth topology (Sec. 3.5: level 0 removed, 2x2
squares flattened into 16 input channels, 4-channel head recombined at full
resolution) in the compensated BF16 form, against the FP64 oracle
`forward_s2d` on the same seeded inputs: max-abs <= 1e-3 and MSE <= 1e-8."""
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


def _theta(seed):
    return scenegen.he_init_weights(seed, N.layer_table_s2d(3)).astype(np.float32)


def _check(ctx, f, theta):
    w = nsm.Weights(ctx, theta, nsm.NSM_TOPO_S2D)
    vis = run_infer(ctx, w, DeviceFrame(f), nsm.NSM_BF16).cpu().numpy().astype(np.float64)
    feat, _, _ = G.features(f.pos4, f.nrm4, f.sm, f.view_proj, f.light_pos, f.cam_pos, f.r_hat, f.z_far, f.bias)
    ref = N.forward_s2d(feat, theta.astype(np.float64))
    err = np.abs(vis - ref)
    print(f"s2d {f.H}x{f.W}: max {err.max():.3e} mse {np.mean(err ** 2):.3e}")
    assert np.isfinite(vis).all() and (vis >= 0).all() and (vis <= 1).all()
    assert err.max() <= 1e-3, err.max()
    assert float(np.mean(err ** 2)) <= 1e-8
    return vis


def test_param_count_matches_the_oracle_table():
    n = sum(ci * co * k * k + co for (_, ci, co, k) in N.layer_table_s2d(3))
    assert nsm.nsm_param_count_topology(nsm.NSM_TOPO_S2D) == n == 36116


@pytest.mark.parametrize("case", ["hard256", "soft256", "ragged", "tiny"])
def test_s2d_bf16_matches_oracle(ctx, case):
    f = {"hard256": lambda: scenegen.hard_frame(256, 256, 512, 512, 8, 1),
         "soft256": lambda: scenegen.soft_frame(256, 256, 512, 512, 8, 21),
         "ragged": lambda: scenegen.soft_frame(68, 132, 300, 200, 8, 5),
         "tiny": lambda: scenegen.soft_frame(4, 8, 16, 16, 3, 6)}[case]()
    _check(ctx, f, _theta(7))


def test_s2d_bf16_1080p_full_frame(ctx):
    _check(ctx, scenegen.soft_frame(1080, 1920, 2048, 2048, 64, 21), _theta(8))


def test_s2d_weights_reject_other_forms_and_batches(ctx):
    f = scenegen.hard_frame(8, 8, 16, 16, 2, 1)
    w = nsm.Weights(ctx, _theta(9), nsm.NSM_TOPO_S2D)
    df = DeviceFrame(f)
    for prec in (nsm.NSM_FP32, nsm.NSM_FP8):
        with pytest.raises(nsm.NSMError) as ei:
            run_infer(ctx, w, df, prec)
        assert ei.value.status == 7
    views = nsm.make_views([df.frame], [torch.empty((8, 8), device="cuda")])
    ws = torch.empty((nsm.nsm_infer_batched_workspace_bytes(views),), dtype=torch.uint8, device="cuda")
    with pytest.raises(nsm.NSMError) as ei:
        nsm.nsm_infer_batched(ctx, views, w, ws)
    assert ei.value.status == 7
    with pytest.raises(nsm.NSMError):
        nsm.Weights(ctx, _theta(9)[:-1], nsm.NSM_TOPO_S2D)


@pytest.mark.parametrize("case", ["hard256", "soft256", "ragged"])
def test_s2d_bf16_trained_weights(ctx, case):
    """The seeded oracle-trained weights of the topology (steep shadow edges)."""
    f = {"hard256": lambda: scenegen.hard_frame(256, 256, 512, 512, 8, 1),
         "soft256": lambda: scenegen.soft_frame(256, 256, 512, 512, 8, 21),
         "ragged": lambda: scenegen.soft_frame(68, 132, 300, 200, 8, 5)}[case]()
    _check(ctx, f, scenegen.trained_weights_s2d())
