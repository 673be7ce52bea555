"""Data-parallel training over torch.distributed ranks, one process per GPU.

Each rank holds a replica of the training state and a share of every batch.
A step is: nsm_train_grad on the local items (the mean gradient of those
items), the exchange, and nsm_train_apply with the exchanged gradient on every
rank, so the replicas' weights stay identical.  The exchange is the method's
one communication step (the gradient of the temporal-window loss of Eq. 2 is
a mean over items): each rank scales its gradient and loss by its item count,
the ranks all-reduce (sum) them together with the counts, and divide, which
gives the full batch's mean whatever the split.  One all-reduce of the
39,521-float gradient (plus the loss and the count) per step.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


class GradientExchange:
    """The exchange step on its own: item-weighted mean of a gradient vector
    and a loss over the ranks of a process group (any backend).  With no
    initialised process group, or one rank, it is the identity."""

    def __init__(self, group=None):
        self.group = group

    def world(self) -> int:
        if not (dist.is_available() and dist.is_initialized()):
            return 1
        return dist.get_world_size(self.group)

    def reduce(self, grad: torch.Tensor, loss: torch.Tensor, items: int):
        """In place: grad, loss <- sum_r items_r x_r / sum_r items_r."""
        if self.world() == 1:
            return grad, loss
        w = float(items)
        n = torch.tensor([w], dtype=grad.dtype, device=grad.device)
        grad.mul_(w)
        loss.mul_(w)
        dist.all_reduce(grad, group=self.group)
        dist.all_reduce(loss, group=self.group)
        dist.all_reduce(n, group=self.group)
        grad.div_(n)
        loss.div_(n)
        return grad, loss


class DataParallelTrainer:
    """nsm_train_grad -> GradientExchange -> nsm_train_apply on one replica.

    state: the rank's TrainState (same initial weights on every rank); the
    gradient travels through a device buffer of the state's size."""

    def __init__(self, state, group=None, device=None):
        self.state = state
        self.exchange = GradientExchange(group)
        device = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.gbuf = torch.empty(state.n, dtype=torch.float32, device=device)
        self.loss = torch.zeros(1, dtype=torch.float32, device=device)

    def step(self, batch, lr=1e-3, alpha=0.9, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        """One data-parallel step on this rank's share `batch`; returns the
        device loss tensor (the full batch's mean once exchanged)."""
        self.state.grad(batch, alpha=alpha, loss_out=self.loss, stream=stream)
        self.state.read(1, self.gbuf, stream=stream)
        if self.exchange.world() > 1:
            torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
            self.exchange.reduce(self.gbuf, self.loss, int(batch.B))
            self.state.write(1, self.gbuf, stream=stream)
        self.state.apply(lr=lr, beta1=beta1, beta2=beta2, eps=eps, stream=stream)
        return self.loss
