"""One replica grid sharded over several engines, one per GPU (host-side driver).

Walkers are independent between exchanges: the multidimensional REMD module
of the paper exchanges conditions, never coordinates, between replicas.  So
an E x pH x T grid is split by walker: every engine is built from the same
systems, grid, run parameters and seed, and advances only its own walkers
(``Engine.set_local_walkers``).  Random numbers are keyed by global walker,
site and slot, so the sharded run is bitwise the single-engine run.

At an exchange step t every engine evaluates its walkers' energies and
exports one row per walker (total energy in fixed point, N_H, N_e and the two
sums of the semi-grand T-exchange energy, 40 bytes); the rows of all engines
are gathered (an all-gather over ``torch.distributed``, NCCL between GPUs or
gloo between CPU processes) and every engine runs the same exchange attempt
on the same rows and random numbers in its own kernel (eqs (3)-(5)), so all
condition maps stay identical without a broadcast.  The step itself then
finishes as usual (see ``cph_exchange_rows`` in ``cphremd.h``).

This module only sequences library calls and moves the rows: every step of
the path runs in the engine's kernels.
"""
from __future__ import annotations

from typing import Callable, List, Sequence

import numpy as np


def partition(sizes: Sequence[int], system_of_slot: Sequence[int], n_parts: int) -> List[List[int]]:
    """Walkers (slot indices at the start) split into n_parts lists of about
    equal pair work: walkers by decreasing cost N^2 (ties by index) each go to
    the part with the least work so far (ties by part index).  Deterministic;
    every part gets at least one walker when there are enough walkers."""
    if n_parts < 1:
        raise ValueError("n_parts must be >= 1")
    W = len(system_of_slot)
    if n_parts > W:
        raise ValueError(f"{n_parts} parts for {W} walkers")
    cost = [int(sizes[system_of_slot[w]]) ** 2 for w in range(W)]
    order = sorted(range(W), key=lambda w: (-cost[w], w))
    load = [0] * n_parts
    parts: List[List[int]] = [[] for _ in range(n_parts)]
    for w in order:
        k = min(range(n_parts), key=lambda p: (load[p], p))
        parts[k].append(w)
        load[k] += cost[w]
    return [sorted(p) for p in parts]


def torch_allgather(group=None) -> Callable[[object], list]:
    """All-gather of any picklable object over an initialised
    torch.distributed process group (one entry per rank, rank order)."""
    import torch.distributed as dist

    def gather(obj):
        out = [None] * dist.get_world_size(group)
        dist.all_gather_object(out, obj, group=group)
        return out

    return gather


class ShardedRun:
    """Drive one engine of a sharded grid through the step schedule.

    ``engine`` has ``get_step``, ``run``, ``mc_titrate``, ``exchange_rows``,
    ``exchange_apply`` and ``step_replicas`` (``cphremd.Engine``, with its
    local walkers set); ``allgather(rows)`` returns every engine's rows.  The
    schedule is the engine's (MC intervals and exchange interval as given):
    plain steps go through ``run`` in spans that stop before the next
    exchange step; an exchange step t runs the MC sweeps due at t, exports
    and gathers the rows, applies the attempt, then the MD step."""

    def __init__(self, engine, allgather: Callable[[object], list], mc_ph_every: int,
                 mc_redox_every: int, exchange_every: int, mc_ph_kind: int = 1,
                 mc_redox_kind: int = 2, dim_next: int = -1):
        self.eng = engine
        self.allgather = allgather
        self.mc_ph, self.mc_redox, self.eaf = mc_ph_every, mc_redox_every, exchange_every
        self.kind_ph, self.kind_redox, self.dim_next = mc_ph_kind, mc_redox_kind, dim_next
        self.exchange_steps = 0

    def _is_exchange(self, t: int) -> bool:
        return t > 0 and self.eaf > 0 and t % self.eaf == 0

    def _mc_kinds(self, t: int) -> int:
        k = 0
        if t > 0 and self.mc_ph > 0 and t % self.mc_ph == 0:
            k |= self.kind_ph
        if t > 0 and self.mc_redox > 0 and t % self.mc_redox == 0:
            k |= self.kind_redox
        return k

    def _steps_to_exchange(self, t: int) -> int:
        if self.eaf <= 0:
            return 1 << 62
        nxt = max(self.eaf, ((t + self.eaf - 1) // self.eaf) * self.eaf)
        return nxt - t

    def exchange_step(self) -> None:
        t = self.eng.get_step()
        kinds = self._mc_kinds(t)
        if kinds:
            self.eng.mc_titrate(kinds)
        rows = self.eng.exchange_rows()
        every = self.allgather(rows)
        self.eng.exchange_apply(self.dim_next, _concat(every))
        self.eng.step_replicas(1)
        self.exchange_steps += 1

    def run(self, n_steps: int) -> None:
        n = int(n_steps)
        while n > 0:
            t = self.eng.get_step()
            if self._is_exchange(t):
                self.exchange_step()
                n -= 1
            else:
                k = min(n, self._steps_to_exchange(t))
                self.eng.run(k)
                n -= k


def _concat(parts):
    if parts and isinstance(parts[0], np.ndarray):
        return np.concatenate(parts)
    out = []
    for p in parts:
        out.extend(p)
    return out
