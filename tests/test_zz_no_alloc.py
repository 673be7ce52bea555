"""nsm_infer_fp32_static: the entry point for callers that may not allocate
device memory (a render loop or an engine plug-in that only owns its frame
buffers).  It must give the same visibility as nsm_infer (FP32) on two calls
in a row, with inputs that differ between the calls, and refuse views larger
than its fixed scratch array.  Kept in its own file, collected last."""
import numpy as np
import pytest

import scenegen
from oracle import network as N

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def nsm():
    from paper_2301_05262_gb300 import build as nsm_build
    nsm_build.build()
    import paper_2301_05262_gb300 as mod
    return mod


def _device_frame(nsm, f):
    from gpu_helpers import DeviceFrame
    return DeviceFrame(f)


def test_static_entry_matches_workspace_entry_twice(nsm):
    from gpu_helpers import run_infer
    ctx = nsm.Context()
    frames = [scenegen.hard_frame(256, 256, 512, 512, 8, 1), scenegen.soft_frame(512, 512, 1024, 1024, 16, 2)]
    thetas = [scenegen.he_init_weights(3, N.layer_table(3)).astype(np.float32),
              scenegen.he_init_weights(4, N.layer_table(3)).astype(np.float32)]
    dfs = [_device_frame(nsm, f) for f in frames]
    refs = [run_infer(ctx, nsm.Weights(ctx, th), df, nsm.NSM_FP32).cpu().numpy() for df, th in zip(dfs, thetas)]
    # two calls in a row on the static entry point, with different inputs
    outs = []
    for df, th in zip(dfs, thetas):
        params = torch.from_numpy(th).cuda()
        out = torch.full((df.f.H, df.f.W), float("nan"), device="cuda")
        nsm.nsm_infer_fp32_static(df.frame, params, out)
        outs.append((out, params))
    torch.cuda.synchronize()
    for (out, _), ref in zip(outs, refs):
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        assert np.abs(got - ref).max() <= 1e-4
    ctx.check()


def test_static_entry_rejects_views_over_the_limit(nsm):
    f = scenegen.hard_frame(516, 512, 64, 64, 2, 1)  # 264,192 pixels > 262,144
    df = _device_frame(nsm, f)
    params = torch.zeros(nsm.nsm_param_count(), device="cuda")
    out = torch.empty((f.H, f.W), device="cuda")
    with pytest.raises(nsm.NSMError) as ei:
        nsm.nsm_infer_fp32_static(df.frame, params, out)
    assert ei.value.status == 2
    assert "static scratch limit" in str(ei.value)
