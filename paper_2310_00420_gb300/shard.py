"""EM with the tasks split across GPUs, one process and one context per GPU (Sec. 3.3).

The E-step of task t needs only Phi_t, y_t and every alpha_c (Eqs. 3, 7, 11), so each rank
holds a contiguous range of tasks and runs their E-step alone.  The M-step (Eq. 5) and the
log-likelihood (Sec. 2) are sums over all tasks: after every E-step the ranks exchange their
rows of per-task M-step terms (cmcs_mstep_terms) in one all-gather, and every rank applies the
same M-step to the rows of all tasks in global task order (cmcs_mstep_apply).  The sums then
run over the same numbers in the same order as on one GPU, so alpha, the priors and every
later E-step are bit-identical whatever the number of ranks.

This module does the partition and the exchange only; the arithmetic is in the library.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np


def partition(N: Sequence[int], world: int) -> List[Tuple[int, int]]:
    """Contiguous task ranges [t0, t1) for `world` ranks, balanced by sum N_t (the operator's
    cost per task is proportional to N_t D).  Every rank gets at least one task, so world must
    not exceed the number of tasks."""
    N = np.asarray(N, dtype=np.float64)
    T = int(N.shape[0])
    if world < 1 or world > T:
        raise ValueError(f"cannot split {T} tasks over {world} ranks")
    cum = np.concatenate([[0.0], np.cumsum(N)])
    bounds = [0]
    for r in range(1, world):
        # first boundary at or past r / world of the total work, leaving a task for every
        # later rank
        t = int(np.searchsorted(cum, cum[-1] * r / world, side="left"))
        t = max(t, bounds[-1] + 1)
        t = min(t, T - (world - r))
        bounds.append(t)
    bounds.append(T)
    return [(bounds[r], bounds[r + 1]) for r in range(world)]


class ShardedEM:
    """Drives a context that holds tasks [t0, t1) of a problem of T_total tasks through EM
    iterations whose M-steps see every task (torch.distributed all-gather of the term rows).

    ctx: an object with estep(), mstep_terms(device=...) -> [T_local][W] and
    mstep_apply(terms [T_total][W]) (a cmcs.Context created with task_offset = t0 and
    T_total).  ranges: the partition of every rank (from `partition`), identical on all ranks.
    device: True to exchange device tensors (NCCL), False for host arrays (gloo)."""

    def __init__(self, ctx, ranges: Sequence[Tuple[int, int]], rank: int, group=None,
                 device: bool = True):
        self.ctx = ctx
        self.ranges = [tuple(map(int, r)) for r in ranges]
        self.rank = int(rank)
        self.group = group
        self.device = device
        self.T_total = self.ranges[-1][1]
        t0, t1 = self.ranges[self.rank]
        self.t0, self.t1 = t0, t1
        self.rows_max = max(b - a for a, b in self.ranges)

    def _gather(self, local):
        """Rows of every rank stacked in global task order, [T_total][W]."""
        import torch
        import torch.distributed as dist
        world = len(self.ranges)
        if self.device:
            loc = local
        else:
            loc = torch.from_numpy(np.ascontiguousarray(local))
        W = int(loc.shape[1])
        if world == 1:
            full = loc
        else:
            pad = loc.new_zeros((self.rows_max, W))
            pad[: loc.shape[0]] = loc
            parts = [loc.new_empty((self.rows_max, W)) for _ in range(world)]
            dist.all_gather(parts, pad, group=self.group)
            full = torch.cat([parts[r][: b - a] for r, (a, b) in enumerate(self.ranges)], dim=0)
        full = full.contiguous()
        return full if self.device else full.numpy()

    def em_iter(self, n: int = 1):
        for _ in range(int(n)):
            self.ctx.estep()
            local = self.ctx.mstep_terms(device=self.device)
            self.ctx.mstep_apply(self._gather(local))
