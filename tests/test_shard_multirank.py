"""One replica grid sharded over ranks: the host-side driver
(paper_1809_07726_gb300/shard.py) run by two and by three gloo ranks on CPU, with the FP64
oracle standing in for each rank's engine (an adapter with the engine's
methods, advancing only the rank's walkers).  Each sharded run must give the
same condition map, site states, positions and velocities, bit for bit, as
the one-rank run of the same driver and as the oracle's own schedule (which
attempts its exchanges inside the step, every walker in one process)."""
import math
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_1809_07726_gb300 import shard, synth

MC_PH, MC_REDOX, EAF, N_STEPS, SEED = 2, 3, 4, 17, 5


def _systems_grid():
    systems = [synth.make_system(24, 61, n_ph=2, ph_atoms=(4, 6), ph_states=(2, 3), redox_atoms=6),
               synth.make_system(36, 62, n_ph=1, ph_atoms=(6, 6), redox_atoms=8)]
    nE, npH, nT = 2, 2, 3
    sos = np.zeros(nE * npH * nT, np.int32)
    for iT in range(nT):
        for ipH in range(npH):
            for iE in range(nE):
                sos[synth.slot_index(iE, ipH, iT, nE, npH)] = 0 if iT < 2 else 1
    grid = synth.Grid(np.array([-0.25, -0.15]), np.array([5.0, 6.0]), np.array([300.0, 320.0, 345.0]),
                      sos, order=("E", "pH", "T"))
    return systems, grid


class OracleShard:
    """The engine interface the driver uses, on the oracle, advancing only
    ``local`` walkers.  Rows carry each walker's total energy and site states
    (the oracle reads N_H and N_e from the states)."""

    def __init__(self, systems, grid, local):
        self.W = oracle.Walkers(systems, grid, seed=SEED, mc_ph=MC_PH, mc_redox=MC_REDOX,
                                exchange_every=EAF)
        self.local = list(local)

    def get_step(self):
        return self.W.t

    def run(self, k):
        oracle.run_schedule(self.W, k, walkers=self.local)  # never crosses an exchange step

    def mc_titrate(self, kinds):
        W, t = self.W, self.W.t
        R = {w: oracle.born(W.x[w], W.osys[W.sys_of[w]].rho, W.osys[W.sys_of[w]].screen, W.gb)[1]
             for w in self.local}
        if kinds & 1:
            for w in self.local:
                oracle.mc_sweep(W, w, "ph", t, R[w])
        if kinds & 2:
            for w in self.local:
                oracle.mc_sweep(W, w, "redox", t, R[w])

    def exchange_rows(self):
        W = self.W
        rows = []
        for w in self.local:
            terms = oracle.energy(W.osys[W.sys_of[w]], W.x[w], W.q[w], W.gb, forces=False)[0]
            rows.append((w, float(terms[5]), W.state[w].tolist()))
        return rows

    def exchange_apply(self, dim, rows):
        W = self.W
        for w, U, st in rows:
            W.U[w] = U
            W.state[w] = np.array(st, np.int64)
        d = W.grid.order[W.n_events % len(W.grid.order)]
        W.n_events += 1
        oracle.exchange_attempt(W, d, W.t)

    def step_replicas(self, n):
        """MD only for the local walkers at step t (energies and forces at x_t,
        one observables sample, Langevin), as the schedule's step t after its
        MC sweeps and exchange attempt."""
        assert n == 1
        W, t = self.W, self.W.t
        for w in self.local:
            o = W.osys[W.sys_of[w]]
            terms, F, R, _ = oracle.energy(o, W.x[w], W.q[w], W.gb)
            W.F[w] = F
        for w in self.local:
            s = int(W.slot_of[w])
            W.visits[w, s] += 1
            for k, st in enumerate(W.state[w]):
                W.occ[s][k, st] += 1
        W.n_obs += 1
        for w in self.local:
            o = W.osys[W.sys_of[w]]
            oracle.langevin(W.x[w], W.v[w], W.F[w], o.mass, W.dt, W.gamma, W.cond(w)[2], W.seed, w, t)
        W.t += 1

    def snapshot(self):
        W = self.W
        return {"slot_of": W.slot_of.copy(), "x": {w: W.x[w].copy() for w in self.local},
                "v": {w: W.v[w].copy() for w in self.local},
                "state": {w: W.state[w].copy() for w in self.local},
                "visits": {w: W.visits[w].copy() for w in self.local}}


def _run(rank_walkers, allgather):
    systems, grid = _systems_grid()
    eng = OracleShard(systems, grid, rank_walkers)
    drv = shard.ShardedRun(eng, allgather, MC_PH, MC_REDOX, EAF)
    drv.run(N_STEPS)
    return eng.snapshot(), drv.exchange_steps


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    systems, grid = _systems_grid()
    parts = shard.partition([s.n for s in systems], grid.system_of_slot, world)
    snap, nex = _run(parts[rank], shard.torch_allgather())
    out[rank] = (snap, nex, parts[rank])
    dist.barrier()
    dist.destroy_process_group()


def test_partition_balances_pair_work():
    sizes = [500, 2000, 8000]
    sos = np.repeat([0, 1, 2], 128)
    for n in (1, 2, 3, 8):
        parts = shard.partition(sizes, sos, n)
        flat = sorted(w for p in parts for w in p)
        assert flat == list(range(len(sos)))
        loads = [sum(sizes[sos[w]] ** 2 for w in p) for p in parts]
        assert max(loads) - min(loads) <= sizes[2] ** 2
    assert shard.partition(sizes, sos, 2) == shard.partition(sizes, sos, 2)  # deterministic


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_match_one_rank_and_the_oracle_schedule(world):
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn")
    systems, grid = _systems_grid()
    one, nex1 = _run(list(range(grid.n_slots)), lambda rows: [rows])
    assert nex1 == N_STEPS // EAF
    # the oracle's own schedule: every walker, exchanges inside the step
    ref = oracle.Walkers(systems, grid, seed=SEED, mc_ph=MC_PH, mc_redox=MC_REDOX, exchange_every=EAF)
    oracle.run_schedule(ref, N_STEPS)
    np.testing.assert_array_equal(one["slot_of"], ref.slot_of)
    seen = set()
    for rank in range(world):
        snap, nex, walkers = out[rank]
        assert nex == nex1
        np.testing.assert_array_equal(snap["slot_of"], one["slot_of"])
        for w in walkers:
            seen.add(w)
            for key in ("x", "v", "state", "visits"):
                np.testing.assert_array_equal(snap[key][w], one[key][w])
            np.testing.assert_array_equal(snap["x"][w], ref.x[w])
            np.testing.assert_array_equal(snap["state"][w], ref.state[w])
    assert seen == set(range(grid.n_slots))
    # exchanges did happen, along every dimension, and moved walkers
    assert sum(1 for e in ref.ex_log) > 0 and not np.array_equal(ref.slot_of, np.arange(grid.n_slots))
