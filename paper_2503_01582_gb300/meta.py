"""Reptile meta-training step (§III-A "Meta-learning", Eq. 1-2) on the library.

A meta step adapts every task of a meta-batch from the shared initialisation
with q inner training steps (Eq. 1; the inner optimiser is the library's Adam
step, and all tasks of a step train in one batched launch), then moves the
initialisation toward the tasks' mean (Eq. 2, batched over the meta-batch):

    theta <- theta + beta (mean_t theta_t^(q) - theta)

Across GPUs the tasks are split between ranks (one process per GPU); the only
exchange of the step is one all-reduce of the ranks' task sums (and of their
task counts) before the outer update.
"""

from __future__ import annotations

from typing import Sequence


def meta_step(ctx, meta: int, tasks: Sequence[int], inner_steps, opts, beta: float, loss=None, group=None,
              task_sum=None) -> int:
    """Runs one meta step; returns the number of tasks over all ranks.

    ctx          a Context (or an object with the same methods)
    meta         the object holding the meta-parameters theta
    tasks        this rank's task objects (same architecture as meta)
    inner_steps  q lists of ray batches; list j holds step j's batch of every task
                 (each batch dict names its task object in "obj")
    opts         training options of the inner steps (make_opts)
    beta         outer step size of Eq. 2
    loss         optional device buffer receiving each inner step's per-batch losses
    group        torch.distributed process group for a multi-GPU meta step, or None
    task_sum     device buffer of param_count floats for the multi-GPU sum (allocated
                 when None)
    """
    ctx.reptile_begin(meta, tasks)
    for batches in inner_steps:
        ctx.train_step(list(batches), opts, loss)
    if group is None:
        ctx.reptile_update(meta, tasks, beta)
        return len(tasks)
    import torch
    import torch.distributed as dist

    if task_sum is None:
        task_sum = torch.empty(ctx.param_count(meta), dtype=torch.float32, device="cuda")
    ctx.reptile_task_sum(tasks, task_sum)
    ctx.sync()  # the sum is complete before the collective reads it
    n = torch.tensor([float(len(tasks))], dtype=torch.float64, device=task_sum.device)
    dist.all_reduce(task_sum, group=group)
    dist.all_reduce(n, group=group)
    n_total = int(round(n.item()))  # also waits for both collectives
    ctx.reptile_apply(meta, task_sum, n_total, beta)
    return n_total


def split_tasks(n_tasks: int, world: int, rank: int):
    """Task indices of this rank when a meta-batch of equally sized tasks is split
    over the ranks (contiguous, sizes differing by at most one)."""
    if world < 1 or not 0 <= rank < world or n_tasks < 0:
        raise ValueError("split_tasks: bad world, rank or task count")
    base, extra = divmod(n_tasks, world)
    start = rank * base + min(rank, extra)
    return list(range(start, start + base + (1 if rank < extra else 0)))
