"""GPU parity of the feature sensitivity (Sec. 3.2, Eq. 1): the per-channel
feature moments against the oracle's features, and the absolute
sensitivities of nsm_sensitivity against the oracle's Eq. 1 with the FP64
forward as the network, on the same noise draws and sigma."""
import numpy as np
import pytest

import scenegen
from oracle import gather as G
from oracle import network as N
from oracle import sensitivity as SE

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2301_05262_gb300 as nsm  # noqa: E402
from gpu_helpers import DeviceFrame  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = nsm.Context()
    yield c
    c.check()
    c.close()


def _feat(f):
    return G.features(f.pos4, f.nrm4, f.sm, f.view_proj, f.light_pos, f.cam_pos, f.r_hat, f.z_far, f.bias)[0]


def test_feature_moments_match_the_oracle_features():
    frames = [scenegen.soft_frame(68, 132, 512, 512, 8, 21), scenegen.hard_frame(36, 52, 256, 256, 6, 22)]
    m = torch.zeros(8, dtype=torch.float64, device="cuda")
    for f in frames:
        nsm.feature_moments(DeviceFrame(f).frame, m)
    torch.cuda.synchronize()
    got = m.cpu().numpy()
    feats = [_feat(f) for f in frames]
    x = np.concatenate([ft.reshape(4, -1) for ft in feats], axis=1)
    np.testing.assert_allclose(got[:4], x.sum(axis=1), rtol=1e-5, atol=1e-3)
    np.testing.assert_allclose(got[4:], (x * x).sum(axis=1), rtol=1e-5)
    n = x.shape[1]
    sig = np.sqrt(got[4:] / n - (got[:4] / n) ** 2)
    np.testing.assert_allclose(sig, SE.feature_std(feats), rtol=1e-4)


@pytest.mark.parametrize("precision,rtol", [(nsm.NSM_FP32, 2e-3), (nsm.NSM_BF16, 3e-2)])
def test_sensitivity_matches_oracle_eq1(ctx, precision, rtol):
    f = scenegen.soft_frame(64, 96, 512, 512, 12, 23)
    th = scenegen.trained_weights()
    feat = _feat(f)
    sigma = SE.feature_std([feat])
    draws = 2
    noise = np.random.default_rng(24).standard_normal((draws, 4, f.H, f.W)).astype(np.float32)
    ref = SE.sensitivity(lambda x: N.forward(x, th.astype(np.float64)), [feat], sigma.astype(np.float32),
                         [list(noise)])
    df = DeviceFrame(f)
    w = nsm.Weights(ctx, th.astype(np.float32))
    ws = torch.empty(nsm.nsm_sensitivity_workspace_bytes(f.H, f.W), dtype=torch.uint8, device="cuda")
    s = torch.zeros(4, dtype=torch.float64, device="cuda")
    nsm.sensitivity(ctx, df.frame, w, precision, torch.from_numpy(noise).cuda(), sigma, ws, s)
    torch.cuda.synchronize()
    got = s.cpu().numpy() / (draws * f.H * f.W)
    print("S gpu", got, "oracle", ref, "relative", SE.relative(got))
    assert (ref > 0).all()
    np.testing.assert_allclose(got, ref, rtol=rtol)
    np.testing.assert_allclose(SE.relative(got), SE.relative(ref), atol=rtol)


def test_sensitivity_rejects_fp8_and_bad_sigma(ctx):
    f = scenegen.hard_frame(16, 16, 64, 64, 2, 25)
    df = DeviceFrame(f)
    w = nsm.Weights(ctx, scenegen.trained_weights().astype(np.float32))
    ws = torch.empty(nsm.nsm_sensitivity_workspace_bytes(16, 16), dtype=torch.uint8, device="cuda")
    s = torch.zeros(4, dtype=torch.float64, device="cuda")
    noise = torch.zeros((1, 4, 16, 16), device="cuda")
    with pytest.raises(nsm.NSMError) as ei:
        nsm.sensitivity(ctx, df.frame, w, nsm.NSM_FP8, noise, [1, 1, 1, 1], ws, s)
    assert ei.value.status == 7
    with pytest.raises(nsm.NSMError):
        nsm.sensitivity(ctx, df.frame, w, nsm.NSM_FP32, noise, [1, 0, 1, 1], ws, s)
