"""Data-parallel training over torch.distributed ranks, one process per GPU.

Each rank holds a replica of the training state and a share of every batch.
A step is: nsm_train_grad on the local items (the mean gradient of those
items), the exchange, and nsm_train_apply with the exchanged gradient on every
rank, so the replicas' weights stay identical.  The exchange is the method's
one communication step (the gradient of the temporal-window loss of Eq. 2 is
a mean over items): each rank scales its gradient and loss by its item count,
the ranks all-reduce (sum) them together with the counts, and divide, which
gives the full batch's mean whatever the split.  Gradient, loss and count
travel in one packed buffer [grad | loss | count]: one all-reduce of 39,523
floats per step, issued on the training stream with no host synchronisation
(NCCL orders it after the gradient kernels and the Adam step after it).
"""
from __future__ import annotations

import contextlib

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

    def reduce_packed(self, buf: torch.Tensor, items: int):
        """In place on buf = [x_0 .. x_{k-1} | slot]: every x_i becomes
        sum_r items_r x_i,r / sum_r items_r (the slot ends up holding the total
        item count).  One all-reduce."""
        if self.world() == 1:
            return buf
        w = float(items)
        buf[:-1].mul_(w)
        buf[-1:].fill_(w)
        dist.all_reduce(buf, group=self.group)
        buf[:-1].div_(buf[-1:])
        return buf

    def reduce(self, grad: torch.Tensor, loss: torch.Tensor, items: int):
        """In place: grad, loss <- sum_r items_r x_r / sum_r items_r, through
        one packed all-reduce."""
        if self.world() == 1:
            return grad, loss
        n, m = grad.numel(), loss.numel()
        buf = torch.empty(n + m + 1, dtype=grad.dtype, device=grad.device)
        buf[:n].copy_(grad.reshape(-1))
        buf[n:n + m].copy_(loss.reshape(-1))
        self.reduce_packed(buf, items)
        grad.copy_(buf[:n].view_as(grad))
        loss.copy_(buf[n:n + m].view_as(loss))
        return grad, loss


class DataParallelTrainer:
    """nsm_train_grad -> GradientExchange -> nsm_train_apply on one replica.

    state: the rank's TrainState (same initial weights on every rank).  The
    gradient and the loss land in views of one packed device buffer
    [grad | loss | count], which is exchanged as it is."""

    def __init__(self, state, group=None, device=None):
        self.state = state
        self.exchange = GradientExchange(group)
        device = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.packed = torch.zeros(state.n + 2, dtype=torch.float32, device=device)
        self.gbuf = self.packed[:state.n]
        self.loss = self.packed[state.n:state.n + 1]

    def step(self, batch, lr=1e-3, alpha=0.9, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        """One data-parallel step on this rank's share `batch`; returns the
        device loss tensor (the full batch's mean once exchanged)."""
        self.state.grad(batch, alpha=alpha, loss_out=self.loss, stream=stream)
        self.state.read(1, self.gbuf, stream=stream)
        if self.exchange.world() > 1:
            with torch.cuda.stream(stream) if stream is not None else contextlib.nullcontext():
                self.exchange.reduce_packed(self.packed, int(batch.B))
            self.state.write(1, self.gbuf, stream=stream)
        self.state.apply(lr=lr, beta1=beta1, beta2=beta2, eps=eps, stream=stream)
        return self.loss
