"""Partition of independent units across ranks, and the one reduction that joins their results.

The units of the path are independent (wavelength, structure) problems: the wavelengths of a spectrum, the
structures of a batch. Each rank takes a contiguous range of units (`unit_range`), solves its own on its own
GPU, and the ranks meet once at the end: one all-reduce (sum) that both adds the per-rank contributions to a
spectrum loss and to its gradients with respect to shared parameters (positions, permittivities), and
gathers per-unit quantities (cross sections, the gradient with respect to each wavelength) by summing
zero-filled copies of the full-length vector, in which each rank has filled only its own range. Host-side
logic over torch.distributed (NCCL for CUDA tensors, gloo for CPU ones); with one process every function is
the identity.
"""
from __future__ import annotations

from typing import Callable, Tuple

import torch
import torch.distributed as dist


def world():
    """(world_size, rank) of the default process group, (1, 0) without one."""
    if dist.is_available() and dist.is_initialized():
        return dist.get_world_size(), dist.get_rank()
    return 1, 0


def unit_range(n_units: int, world_size: int, rank: int) -> Tuple[int, int]:
    """Contiguous [lo, hi) of the units owned by `rank`: the first n_units % world_size ranks take one unit
    more than the others; a rank may own none when there are fewer units than ranks."""
    if world_size < 1 or not 0 <= rank < world_size or n_units < 0:
        raise ValueError("bad partition request")
    base, extra = divmod(n_units, world_size)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def weighted_unit_range(weights, world_size: int, rank: int) -> Tuple[int, int]:
    """Contiguous [lo, hi) of the units owned by `rank` when units cost unequal work (a batch of structures of
    uneven size: the LU costs (3N)^3): rank r's range ends at the first unit where the running sum of weights
    reaches (r + 1)/world_size of the total, so the ranges are contiguous, cover every unit once, and their
    sums differ by at most the largest single weight."""
    if world_size < 1 or not 0 <= rank < world_size:
        raise ValueError("bad partition request")
    w = [float(x) for x in weights]
    if any(x < 0 for x in w):
        raise ValueError("weights must be non-negative")
    total = sum(w)

    def end(r):
        if r + 1 >= world_size:
            return len(w)
        target = total * (r + 1) / world_size
        acc = 0.0
        for i, x in enumerate(w):
            if acc + 0.5 * x >= target:   # cut where the unit's midpoint passes the target
                return i
            acc += x
        return len(w)

    lo = 0 if rank == 0 else end(rank - 1)
    return lo, max(lo, end(rank))


def sum_over_ranks(t: torch.Tensor) -> torch.Tensor:
    """In-place sum of t over all ranks (returns t)."""
    ws, _ = world()
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t


def gather_units(local: torch.Tensor, lo: int, n_units: int) -> torch.Tensor:
    """Full (n_units, ...) tensor from each rank's rows [lo, lo + len(local)): zero-filled and summed."""
    full = torch.zeros((n_units,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    full[lo:lo + local.shape[0]] = local
    return sum_over_ranks(full)


def spectrum_loss_and_grads(unit_fn: Callable[[int, int], tuple], n_units: int):
    """Loss of a spectrum that is a sum over independent units, with its gradients, across the ranks.

    unit_fn(lo, hi) -> (loss, grad_pos, grad_eps, grad_units) over the units [lo, hi) of this rank: loss a
    0-d tensor, grad_pos and grad_eps the gradients with respect to the shared parameters, grad_units the
    (hi - lo,) gradient with respect to each unit's own parameter (its wavelength). Returns the totals over
    all units (loss and shared gradients summed, grad_units gathered), identical on every rank."""
    ws, rank = world()
    lo, hi = unit_range(n_units, ws, rank)
    loss, gpos, geps, gunits = unit_fn(lo, hi)
    loss = sum_over_ranks(torch.as_tensor(loss, dtype=torch.float64).reshape(1).clone())[0]
    gpos = sum_over_ranks(gpos.clone())
    geps = sum_over_ranks(geps.clone())
    gunits = gather_units(gunits, lo, n_units)
    return loss, gpos, geps, gunits
