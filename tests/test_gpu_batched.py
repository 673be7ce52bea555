"""Batched serving: one pass of the five persistent stage kernels over many
views of uneven size gives exactly the per-view nsm_infer result; the CUDA
graph path replays with new inputs; the autotuner's plan keeps parity."""
import numpy as np
import pytest

import scenegen
from oracle import gather as G
from oracle import network as N

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2301_05262_gb300 as nsm  # noqa: E402
from gpu_helpers import DeviceFrame, run_infer  # noqa: E402

SIZES = [(64, 96, 128), (128, 128, 256), (36, 52, 64), (256, 192, 512), (100, 68, 96), (4, 4, 16)]


@pytest.fixture(scope="module")
def ctx():
    c = nsm.Context()
    yield c
    c.check()
    c.close()


def _views(sizes, seed):
    dfs, outs = [], []
    for k, (H, W, S) in enumerate(sizes):
        mk = scenegen.soft_frame if k % 2 else scenegen.hard_frame
        dfs.append(DeviceFrame(mk(H, W, S, S, 8, seed + k)))
        outs.append(torch.full((H, W), float("nan"), device="cuda"))
    return dfs, outs


def _batched(ctx, w, dfs, outs):
    views = nsm.make_views([d.frame for d in dfs], outs)
    ws = torch.empty((nsm.nsm_infer_batched_workspace_bytes(views),), dtype=torch.uint8, device="cuda")
    nsm.nsm_infer_batched(ctx, views, w, ws)
    torch.cuda.synchronize()
    return [o.cpu().numpy() for o in outs]


def test_batched_matches_single_view_calls(ctx):
    theta = scenegen.he_init_weights(3, N.layer_table(3)).astype(np.float32)
    w = nsm.Weights(ctx, theta)
    dfs, outs = _views(SIZES, 10)
    got = _batched(ctx, w, dfs, outs)
    for df, g in zip(dfs, got):
        ref = run_infer(ctx, w, df, nsm.NSM_BF16).cpu().numpy()
        np.testing.assert_array_equal(g, ref)


def test_graph_replay_with_new_inputs(ctx):
    theta = scenegen.he_init_weights(4, N.layer_table(3)).astype(np.float32)
    w = nsm.Weights(ctx, theta)
    nsm.nsm_ctx_set_graph(ctx, True)
    try:
        for seed in (20, 30, 40):  # same plan (sizes), different scenes / buffers
            dfs, outs = _views(SIZES[:4], seed)
            got = _batched(ctx, w, dfs, outs)
            for df, g in zip(dfs, got):
                np.testing.assert_array_equal(g, run_infer(ctx, w, df, nsm.NSM_BF16).cpu().numpy())
        assert nsm.nsm_ctx_graph_replays(ctx) == 3
        # a different plan re-captures
        dfs, outs = _views(SIZES[2:5], 50)
        _batched(ctx, w, dfs, outs)
        assert nsm.nsm_ctx_graph_replays(ctx) == 1
    finally:
        nsm.nsm_ctx_set_graph(ctx, False)


def test_autotuned_plan_keeps_parity(ctx):
    theta = scenegen.he_init_weights(5, N.layer_table(3)).astype(np.float32)
    w = nsm.Weights(ctx, theta)
    dfs, outs = _views([(256, 256, 512), (128, 192, 256)], 60)
    views = nsm.make_views([d.frame for d in dfs], outs)
    ws = torch.empty((nsm.nsm_infer_batched_workspace_bytes(views),), dtype=torch.uint8, device="cuda")
    nsm.nsm_autotune(ctx, views, w, ws, reps=2)
    rows, ctas, ms = nsm.nsm_autotune_report(ctx)
    assert all(r in (1, 2, 4, 8) for r in rows) and all(c >= 1 for c in ctas) and all(m > 0 for m in ms)
    got = _batched(ctx, w, dfs, outs)
    for df, g in zip(dfs, got):
        f = df.f
        feat, _, _ = G.features(f.pos4, f.nrm4, f.sm, f.view_proj, f.light_pos, f.cam_pos, f.r_hat, f.z_far, f.bias)
        q = N.forward_rounded(feat, theta.astype(np.float64), N.round_bf16_pair, rnd_in=N.round_bf16_pair,
                              coarse_dec0=True)
        assert float(np.mean((g - q) ** 2)) <= 1e-8
        assert np.abs(g - q).max() <= 1e-3
        np.testing.assert_array_equal(g, run_infer(ctx, w, df, nsm.NSM_BF16).cpu().numpy())


def test_batched_rejects_too_many_views(ctx):
    theta = scenegen.he_init_weights(3, N.layer_table(3)).astype(np.float32)
    w = nsm.Weights(ctx, theta)
    f = DeviceFrame(scenegen.hard_frame(8, 8, 16, 16, 2, 1))
    outs = [torch.empty((8, 8), device="cuda") for _ in range(33)]
    views = nsm.make_views([f.frame] * 33, outs)
    ws = torch.empty((1 << 20,), dtype=torch.uint8, device="cuda")
    with pytest.raises(nsm.NSMError) as ei:
        nsm.nsm_infer_batched(ctx, views, w, ws)
    assert ei.value.status == 2


def test_every_stage_variant_matches_the_default_plan():
    """Each tile variant of each tensor-core stage (tile height, warp roles, K
    slices, MMA schedule) gives the default plan's visibility on a ragged soft
    frame, to FP32 accumulation-order noise (K slices change the order)."""
    c = nsm.Context()
    f = scenegen.soft_frame(100, 300, 256, 256, 8, 5)
    w = nsm.Weights(c, scenegen.trained_weights())
    df = DeviceFrame(f)
    ref = run_infer(c, w, df, nsm.NSM_BF16).cpu().numpy()
    for stage in range(5):
        n = nsm.nsm_plan_variants(stage)
        assert n >= 2
        for v in range(n):
            nsm.nsm_plan_set(c, stage, v, 1)
            out = run_infer(c, w, df, nsm.NSM_BF16).cpu().numpy()
            assert np.abs(out - ref).max() <= 1e-4, (stage, v, np.abs(out - ref).max())
        nsm.nsm_plan_set(c, stage, 0, 0)
    assert nsm.nsm_plan_variants(5) == 0
    with pytest.raises(nsm.NSMError):
        nsm.nsm_plan_set(c, 0, 99, 0)
    c.check()


def test_batched_with_a_2160p_view_matches_single_view_calls(ctx):
    """The largest serving view (3840 x 2160, 4096^2 map) in one batch with
    small ones: every view equals its own nsm_infer call bit for bit."""
    w = nsm.Weights(ctx, scenegen.trained_weights())
    dfs = [DeviceFrame(scenegen.soft_frame(2160, 3840, 4096, 4096, 64, 31)),
           DeviceFrame(scenegen.hard_frame(68, 132, 300, 300, 8, 5)),
           DeviceFrame(scenegen.soft_frame(540, 960, 1024, 1024, 16, 6))]
    outs = [torch.full((d.f.H, d.f.W), float("nan"), device="cuda") for d in dfs]
    got = _batched(ctx, w, dfs, outs)
    for df, g in zip(dfs, got):
        np.testing.assert_array_equal(g, run_infer(ctx, w, df, nsm.NSM_BF16).cpu().numpy())


@pytest.mark.parametrize("graph", [False, True])
def test_per_view_completion_records(ctx, graph):
    """With view timing on, every view of a batch gets a completion time after
    the batch's start and no later than the batch's end (host wall clock
    around the synchronised call), the outputs are unchanged, and a second
    batch overwrites the records."""
    import time
    theta = scenegen.he_init_weights(5, N.layer_table(3)).astype(np.float32)
    w = nsm.Weights(ctx, theta)
    rec = torch.zeros(65, dtype=torch.int64, device="cuda")
    nsm.nsm_ctx_set_graph(ctx, graph)
    try:
        dfs, outs = _views(SIZES, 60)
        ref = _batched(ctx, w, dfs, outs)
        nsm.nsm_ctx_set_view_timing(ctx, rec)
        first = None
        for rep in range(2):
            dfs2, outs2 = _views(SIZES, 60)
            t0 = time.perf_counter()
            got = _batched(ctx, w, dfs2, outs2)
            wall_ns = (time.perf_counter() - t0) * 1e9
            r = rec.cpu().numpy()
            lat = r[1:1 + len(SIZES)] - r[0]
            assert r[0] > 0 and (lat > 0).all(), r
            assert lat.max() <= wall_ns, (lat.max(), wall_ns)
            for a, b in zip(got, ref):
                np.testing.assert_array_equal(a, b)
            if first is not None:
                assert r[0] > first
            first = r[0]
            # the counters reached each view's unit count exactly once
            assert (r[1 + 32:1 + 32 + len(SIZES)] > 0).all()
    finally:
        nsm.nsm_ctx_set_view_timing(ctx, None)
        nsm.nsm_ctx_set_graph(ctx, False)
