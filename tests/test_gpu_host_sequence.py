"""The pipelined host-buffer entry point (nsm_infer_host_sequence): every
frame's visibility equals nsm_infer's on the same inputs bit for bit, for
frames of different sizes (an empty one among them), with 2 and 3 staging
slots, in the FP32 and BF16 forms."""
import numpy as np
import pytest

import scenegen
from oracle import network as N

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2301_05262_gb300 as nsm  # noqa: E402
from gpu_helpers import DeviceFrame, light_desc, run_infer  # noqa: E402

SIZES = [(64, 96, 256), (128, 64, 512), (96, 160, 300), (0, 32, 64), (64, 96, 256), (40, 200, 128), (128, 64, 512)]


@pytest.fixture(scope="module")
def setup():
    ctx = nsm.Context()
    th = scenegen.he_init_weights(3, N.layer_table(3)).astype(np.float32)
    w = nsm.Weights(ctx, th)
    frames = []
    for k, (H, W, S) in enumerate(SIZES):
        if H == 0:
            frames.append(None)
        else:
            frames.append((scenegen.soft_frame if k % 2 else scenegen.hard_frame)(H, W, S, S, 12, 30 + k))
    return ctx, w, frames


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("nslots", [2, 3])
def test_sequence_matches_single_frames(setup, prec, nslots):
    ctx, w, frames = setup
    precision = nsm.PRECISIONS[prec]
    pinned, hframes, outs, refs = [], [], [], []
    for (H, W, S), f in zip(SIZES, frames):
        if f is None:
            f0 = frames[0]
            p = [torch.from_numpy(x).pin_memory() for x in (f0.pos4, f0.nrm4, f0.sm)]
            pinned.append(p)
            fr = nsm.make_frame(p[0], p[1], p[2], light_desc(f0), f0.cam_pos)
            fr.H = 0  # an empty view: nothing is copied or computed
            hframes.append(fr)
            outs.append(torch.full((1,), -7.0).pin_memory())
            refs.append(None)
            continue
        p = [torch.from_numpy(x).pin_memory() for x in (f.pos4, f.nrm4, f.sm)]
        pinned.append(p)
        hframes.append(nsm.make_frame(p[0], p[1], p[2], light_desc(f), f.cam_pos))
        outs.append(torch.full((H, W), -7.0).pin_memory())
        refs.append(run_infer(ctx, w, DeviceFrame(f), precision).cpu().numpy())
    slot = max(nsm.nsm_infer_host_stage_bytes(H, W, S, S) for (H, W, S) in SIZES if H > 0)
    slot = (slot + 255) // 256 * 256
    stage = torch.empty((nslots * slot,), dtype=torch.uint8, device="cuda")
    ws = torch.empty((max(nsm.nsm_infer_workspace_bytes(H, W, precision) for (H, W, _) in SIZES),),
                     dtype=torch.uint8, device="cuda")
    nsm.nsm_infer_host_sequence(ctx, hframes, w, precision, stage, ws, outs)
    for o, r in zip(outs, refs):
        if r is None:
            assert o.item() == -7.0  # nothing written for an empty frame
        else:
            np.testing.assert_array_equal(o.numpy(), r)
    ctx.check()


def test_sequence_rejects_small_staging(setup):
    ctx, w, frames = setup
    f = frames[0]
    p = [torch.from_numpy(x).pin_memory() for x in (f.pos4, f.nrm4, f.sm)]
    hf = nsm.make_frame(p[0], p[1], p[2], light_desc(f), f.cam_pos)
    one = nsm.nsm_infer_host_stage_bytes(f.H, f.W, f.Hs, f.Ws)
    stage = torch.empty((one + 256,), dtype=torch.uint8, device="cuda")
    ws = torch.empty((nsm.nsm_infer_workspace_bytes(f.H, f.W, nsm.NSM_BF16),), dtype=torch.uint8, device="cuda")
    with pytest.raises(nsm.NSMError):
        nsm.nsm_infer_host_sequence(ctx, [hf, hf], w, nsm.NSM_BF16, stage, ws,
                                    [np.empty((f.H, f.W), np.float32), np.empty((f.H, f.W), np.float32)])
