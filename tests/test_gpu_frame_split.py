"""GPU: one frame computed as row bands with nsm_infer_rows (the unit of a
frame split across devices) equals nsm_infer on the whole frame bit for bit,
in the FP32 and the BF16 forms; bad bands are rejected."""
import numpy as np
import pytest

import scenegen
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


@pytest.mark.parametrize("precision", [nsm.NSM_FP32, nsm.NSM_BF16])
@pytest.mark.parametrize("world,halo", [(3, 16), (4, 32)])
def test_row_bands_equal_the_whole_frame(ctx, precision, world, halo):
    f = scenegen.soft_frame(264, 200, 512, 512, 12, 7)
    df = DeviceFrame(f)
    w = nsm.Weights(ctx, scenegen.trained_weights().astype(np.float32))
    whole = run_infer(ctx, w, df, precision).cpu().numpy()
    parts = []
    for r in range(world):
        y0, y1 = nsm.frame_rows(f.H, r, world)
        ws = torch.empty(nsm.nsm_infer_rows_workspace_bytes(f.H, f.W, y0, y1, halo, precision), dtype=torch.uint8,
                         device="cuda")
        out = torch.full((y1 - y0, f.W), float("nan"), device="cuda")
        nsm.nsm_infer_rows(ctx, df.frame, w, precision, y0, y1, halo, ws, out)
        parts.append(out)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(torch.cat(parts).cpu().numpy(), whole)


def test_row_bands_reject_unaligned_bounds(ctx):
    f = scenegen.hard_frame(64, 64, 128, 128, 4, 8)
    df = DeviceFrame(f)
    w = nsm.Weights(ctx, scenegen.he_init_weights(3, N.layer_table(3)).astype(np.float32))
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    out = torch.empty((64, 64), device="cuda")
    for y0, y1, halo in ((2, 32, 16), (0, 30, 16), (0, 32, 6), (32, 32, 16), (0, 68, 16)):
        with pytest.raises(nsm.NSMError) as ei:
            nsm.nsm_infer_rows(ctx, df.frame, w, nsm.NSM_FP32, y0, y1, halo, ws, out)
        assert ei.value.status == 2
