"""One frame split across devices by rows (multi-GPU inference, each device
recomputing a halo of rows, no exchange): the band bounds, the halo that
reproduces the whole-frame network exactly (the oracle forward on row bands),
and two gloo ranks that each compute their band with the oracle and gather
the whole frame."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import paper_2301_05262_gb300 as nsm  # noqa: E402


def test_frame_rows_partition():
    for H in (4, 8, 100, 1080, 2160):
        for world in (1, 2, 3, 4, 8):
            bands = [nsm.frame_rows(H, r, world) for r in range(world)]
            assert bands[0][0] == 0 and bands[-1][1] == H
            for (a0, a1), (b0, b1) in zip(bands, bands[1:]):
                assert a1 == b0
            assert all(y0 % 4 == 0 and y1 % 4 == 0 and y0 <= y1 for y0, y1 in bands)
            sizes = [y1 - y0 for y0, y1 in bands]
            assert max(sizes) - min(sizes) <= 4


def _band(feat, th, y0, y1, halo):
    from oracle import network as N
    a, b = max(0, y0 - halo), min(feat.shape[1], y1 + halo)
    return N.forward(feat[:, a:b], th)[y0 - a:y1 - a]


def test_halo_of_16_rows_is_exact_and_12_is_not():
    """The receptive field of the 3-level network reaches fewer than 16 rows
    (bands aligned to the 4-row pooling grid): a band recomputed with a 16-row
    halo equals the whole-frame forward; 12 rows do not suffice."""
    import scenegen
    from oracle import gather as G
    from oracle import network as N
    f = scenegen.soft_frame(160, 64, 256, 256, 8, 3)
    feat, _, _ = G.features(f.pos4, f.nrm4, f.sm, f.view_proj, f.light_pos, f.cam_pos, f.r_hat, f.z_far, f.bias)
    th = scenegen.trained_weights().astype(np.float64)
    full = N.forward(feat, th)
    for y0, y1 in ((64, 96), (0, 40), (120, 160)):
        np.testing.assert_array_equal(_band(feat, th, y0, y1, 16), full[y0:y1])
    assert np.abs(_band(feat, th, 64, 96, 12) - full[64:96]).max() > 1e-4


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import scenegen
    from oracle import gather as G
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        f = scenegen.hard_frame(72, 48, 256, 256, 8, 5)
        feat, _, _ = G.features(f.pos4, f.nrm4, f.sm, f.view_proj, f.light_pos, f.cam_pos, f.r_hat, f.z_far, f.bias)
        th = scenegen.trained_weights().astype(np.float64)
        y0, y1 = nsm.frame_rows(f.H, rank, world)
        mine = torch.from_numpy(_band(feat, th, y0, y1, 32).copy())
        sizes = [nsm.frame_rows(f.H, r, world) for r in range(world)]
        parts = [torch.empty((b - a, f.W), dtype=torch.float64) for a, b in sizes]
        parts[rank].copy_(mine)
        for r in range(world):  # bands may differ in size: one broadcast per band
            dist.broadcast(parts[r], src=r)
        q.put((rank, torch.cat(parts).numpy()))
    finally:
        dist.destroy_process_group()


def test_two_ranks_compute_one_frame():
    """Two gloo ranks each compute their band (32-row halo) with the oracle and
    gather the whole frame: equal to the whole-frame forward."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted((q.get(timeout=300) for _ in range(2)), key=lambda t: t[0])
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    import scenegen
    from oracle import gather as G
    from oracle import network as N
    f = scenegen.hard_frame(72, 48, 256, 256, 8, 5)
    feat, _, _ = G.features(f.pos4, f.nrm4, f.sm, f.view_proj, f.light_pos, f.cam_pos, f.r_hat, f.z_far, f.bias)
    full = N.forward(feat, scenegen.trained_weights().astype(np.float64))
    for _, whole in got:
        np.testing.assert_array_equal(whole, full)
