"""nsm_infer_fp32_static: the entry point for callers that may not allocate
device memory (a render loop or an engine plug-in that only owns its frame
buffers).  It must give the same visibility as nsm_infer (FP32) on two calls
in a row, with inputs that differ between the calls, and refuse views larger
than its fixed scratch array or frames that nsm_infer refuses.  Kept in its
own file, collected last."""
import math

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
    """Same kernels, same grids as nsm_infer: the results are bit-identical.
    The larger view runs first, so the second (smaller) call reads the array
    right after it held the first call's activations."""
    from gpu_helpers import run_infer
    ctx = nsm.Context()
    frames = [scenegen.soft_frame(512, 512, 1024, 1024, 16, 2), scenegen.hard_frame(256, 256, 512, 512, 8, 1)]
    thetas = [scenegen.he_init_weights(3, N.layer_table(3)).astype(np.float32),
              scenegen.he_init_weights(4, N.layer_table(3)).astype(np.float32)]
    dfs = [_device_frame(nsm, f) for f in frames]
    refs = [run_infer(ctx, nsm.Weights(ctx, th), df, nsm.NSM_FP32).cpu().numpy() for df, th in zip(dfs, thetas)]
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
        np.testing.assert_array_equal(got, ref)
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


def test_static_entry_rejects_what_nsm_infer_rejects(nsm):
    """Non-finite light values, tan_half_fov = 0, and buffers whose allocation
    is too short: errors, no launch, the output left untouched."""
    f = scenegen.hard_frame(64, 64, 64, 64, 2, 1)
    df = _device_frame(nsm, f)
    params = torch.zeros(nsm.nsm_param_count(), device="cuda")
    out = torch.full((f.H, f.W), 7.0, device="cuda")
    df.frame.light.pos[0] = math.nan
    with pytest.raises(nsm.NSMError) as ei:
        nsm.nsm_infer_fp32_static(df.frame, params, out)
    assert ei.value.status == 1
    df.frame.light.pos[0] = float(f.light_pos[0])
    df.frame.light.tan_half_fov = 0.0
    with pytest.raises(nsm.NSMError):
        nsm.nsm_infer_fp32_static(df.frame, params, out)
    df.frame.light.tan_half_fov = float(f.tan_half_fov)
    # a parameter buffer one float short: the last bytes of an allocation of
    # its own (driver API, exact 2 MiB, so no allocator pool hides the end)
    import ctypes
    drv = ctypes.CDLL("libcuda.so.1")
    dptr = ctypes.c_uint64(0)
    assert drv.cuMemAlloc_v2(ctypes.byref(dptr), ctypes.c_size_t(2 << 20)) == 0
    try:
        start = dptr.value + (2 << 20) - 4 * (nsm.nsm_param_count() - 1)
        st = nsm.lib().nsm_infer_fp32_static(ctypes.byref(df.frame), ctypes.c_void_p(start),
                                             ctypes.c_void_p(out.data_ptr()), None)
        assert st == 1
        assert b"dev_params" in nsm.lib().nsm_last_error()
        torch.cuda.synchronize()
        assert (out == 7.0).all()                                  # nothing ran
        # the same buffer, long enough, is accepted
        start = dptr.value + (2 << 20) - 4 * nsm.nsm_param_count()
        assert drv.cuMemsetD8_v2(ctypes.c_uint64(start), 0, ctypes.c_size_t(4 * nsm.nsm_param_count())) == 0
        st = nsm.lib().nsm_infer_fp32_static(ctypes.byref(df.frame), ctypes.c_void_p(start),
                                             ctypes.c_void_p(out.data_ptr()), None)
        assert st == 0, nsm.lib().nsm_last_error()
        torch.cuda.synchronize()
        # zero weights and biases: every pre-activation is 0, the head gives sigmoid(0)
        assert (out == 0.5).all()
    finally:
        torch.cuda.synchronize()
        drv.cuMemFree_v2(dptr)
