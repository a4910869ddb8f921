"""Data-parallel gradient step: one batch of scan positions split over ranks, one GPU per rank.

The paper spreads a batch over several GPUs (Sec. "Feature comparison with other open-source
packages", multi-GPU through `accelerate`) and, equivalently, accumulates gradients over
sub-batches (Sec. "Computation speed and convergence").  Positions are independent until the loss:
Eq. 5 and 6 divide by <I_meas^p> of the whole batch, and the Gaussian form takes a square root of
the whole batch's mean squared residual.  So one step is

  1. every rank: this rank's loss statistics {S, Q, D B} (`Ptycho.loss_stats`);
  2. all-reduce (sum) of those three numbers;
  3. every rank: loss and gradients of its positions against the whole batch's statistics
     (`Ptycho.loss_grad(..., whole_stats=...)`, i.e. pty_loss_grad_part);
  4. all-reduce (sum) of the loss share and of every gradient array (object amplitude and phase,
     probe, positions, tilts, dz); position and local-tilt gradients are zero outside a rank's own
     positions, so the sum assembles them;
  5. every rank: the same Adam update on the same parameters and gradients (pty_adam_update), so
     the replicas stay identical with no parameter broadcast.

The collectives are torch.distributed all-reduces on each rank's own tensors (NCCL between GPUs,
gloo on the CPU); this module only orders the calls.  Every number is computed by the library's
kernels.
"""
from __future__ import annotations

import torch

from . import _lib
from .ptycho import Adam, Params, Ptycho

GRAD_NAMES = ("amp", "phase", "probe", "pos", "tilt", "dz")


def _as_real(t: torch.Tensor) -> torch.Tensor:
    return torch.view_as_real(t) if t.is_complex() else t


def loss_grad(pt: Ptycho, params: Params, idx, I_meas: torch.Tensor, grads: Params, all_reduce):
    """Loss and gradients of the whole batch, of which this rank holds positions `idx`.

    all_reduce(tensor) sums a tensor over the ranks in place (e.g. torch.distributed.all_reduce).
    Returns (loss, grads); both hold the whole batch's values on every rank."""
    stats = pt.loss_stats(params, idx, I_meas)
    all_reduce(stats)
    loss, grads = pt.loss_grad(params, idx, I_meas, grads=grads, whole_stats=stats)
    want = set(pt.geom.grads)
    for name in GRAD_NAMES:
        if name in want:
            all_reduce(_as_real(getattr(grads, name)))
    all_reduce(loss)
    return loss, grads


def step(pt: Ptycho, params: Params, grads: Params, adam: Adam, idx, I_meas: torch.Tensor, all_reduce):
    """One data-parallel Adam iteration: `loss_grad`, then the same pty_adam_update on every rank."""
    loss, grads = loss_grad(pt, params, idx, I_meas, grads, all_reduce)
    adam.t += 1
    _lib.pty_adam_update(pt.cg, *pt._param_ptrs(params), *pt._param_ptrs(grads), adam.c(), adam.t, pt._stream())
    return loss


def split(batch, rank: int, world: int):
    """This rank's contiguous share of a batch of positions (sizes differ by at most one)."""
    n = len(batch)
    lo = rank * n // world
    hi = (rank + 1) * n // world
    return list(batch[lo:hi])

