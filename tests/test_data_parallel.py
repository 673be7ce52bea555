"""Data-parallel training's exchange step on CPU: two gloo ranks over
127.0.0.1, each holding part of a batch (2 + 1 items: the split is uneven on
purpose).  Each rank's gradient and loss are the oracle's (the mean over its
own items); after GradientExchange they equal the oracle's full-batch
gradient and loss, and the Adam step taken with them equals the oracle's
full-batch training step."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _batch():
    """3 items x T = 2 instances of 16 x 16 features (seeded scenes and one
    perturbation each) with ray-cast targets; oracle features."""
    sys.path.insert(0, ROOT)
    import scenegen
    from oracle import gather as G
    rng = scenegen.SplitMix64(77)
    feats, targets = [], []
    for b in range(3):
        base = scenegen.random_scene(500 + b, 6, soft=True)
        insts = []
        for sc in (base, scenegen.perturbed(base, rng)):
            f = scenegen.render_frame(sc, 16, 16, 64, 64)
            insts.append(G.features(f.pos4, f.nrm4, f.sm, f.view_proj, f.light_pos, f.cam_pos, f.r_hat, f.z_far,
                                    f.bias)[0])
        feats.append(insts)
        f0 = scenegen.render_frame(base, 16, 16, 64, 64)
        targets.append(scenegen.soft_visibility(f0, spp_side=4).astype(np.float64))
    return feats, targets


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import scenegen
    from oracle import network as N
    from paper_2301_05262_gb300.data_parallel import GradientExchange
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        feats, targets = _batch()
        theta = scenegen.he_init_weights(3, N.layer_table(3))
        mine = [0, 1] if rank == 0 else [2]
        zeros = np.zeros_like(theta)
        _, _, _, loss, grad = N.train_step([feats[i] for i in mine], [targets[i] for i in mine], theta, zeros, zeros,
                                           1)
        g = torch.from_numpy(grad.copy())
        lo = torch.tensor([loss], dtype=torch.float64)
        GradientExchange().reduce(g, lo, len(mine))
        q.put((rank, g.numpy(), float(lo.item())))
    finally:
        dist.destroy_process_group()


def test_exchange_gives_the_full_batch_gradient_and_step():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    # drain the queue before joining: a child holding a large queued item
    # cannot exit until it has been read
    got = sorted((q.get(timeout=300) for _ in range(2)), key=lambda t: t[0])
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    sys.path.insert(0, ROOT)
    import scenegen
    from oracle import network as N
    feats, targets = _batch()
    theta = scenegen.he_init_weights(3, N.layer_table(3))
    zeros = np.zeros_like(theta)
    th_full, m_full, v_full, loss_full, grad_full = N.train_step(feats, targets, theta, zeros, zeros, 1, lr=1e-3)
    for rank, g, lo in got:
        np.testing.assert_allclose(g, grad_full, rtol=1e-12, atol=1e-15)
        assert lo == pytest.approx(loss_full, rel=1e-12)
        # the Adam step every replica takes with the exchanged gradient
        th, _, _ = N.adam_update(theta, g, zeros, zeros, 1, lr=1e-3)
        np.testing.assert_allclose(th, th_full, rtol=1e-12, atol=1e-15)


def test_exchange_is_the_identity_on_one_rank():
    sys.path.insert(0, ROOT)
    from paper_2301_05262_gb300.data_parallel import GradientExchange
    g = torch.arange(5, dtype=torch.float64)
    lo = torch.tensor([2.5], dtype=torch.float64)
    GradientExchange().reduce(g, lo, 7)
    assert g.tolist() == [0.0, 1.0, 2.0, 3.0, 4.0] and lo.item() == 2.5


class _FakeState:
    """Stands in for TrainState on CPU: grad() writes a rank-specific mean
    gradient and loss, apply() records the gradient it was given."""

    def __init__(self, rank, n=7):
        self.n = n
        self.rank = rank
        self.g = torch.zeros(n)
        self.applied = None

    def grad(self, batch, alpha, loss_out, stream=None):
        self.g = torch.arange(self.n, dtype=torch.float32) * (self.rank + 1) + 10 * self.rank
        loss_out.fill_(1.5 + self.rank)

    def read(self, k, out, stream=None):
        out.copy_(self.g)

    def write(self, k, src, stream=None):
        self.g = src.clone()

    def apply(self, **kw):
        self.applied = self.g.clone()


def _rank_trainer(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    from types import SimpleNamespace
    from paper_2301_05262_gb300.data_parallel import DataParallelTrainer
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        st = _FakeState(rank)
        tr = DataParallelTrainer(st, device=torch.device("cpu"))
        loss = tr.step(SimpleNamespace(B=2 if rank == 0 else 1))
        q.put((rank, st.applied.numpy(), float(loss.item())))
    finally:
        dist.destroy_process_group()


def test_trainer_exchanges_one_packed_buffer():
    """The trainer's packed [grad | loss | count] exchange on two gloo ranks
    with 2 + 1 items: the applied gradient and the loss are the item-weighted
    means on both ranks."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_trainer, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted((q.get(timeout=300) for _ in range(2)), key=lambda t: t[0])
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    a = np.arange(7, dtype=np.float64)
    want = (2 * a + (2 * a + 10)) / 3
    for _, g, lo in got:
        np.testing.assert_allclose(g, want, rtol=1e-6)
        assert lo == pytest.approx((2 * 1.5 + 2.5) / 3, rel=1e-6)
