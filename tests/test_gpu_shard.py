"""One replica grid sharded over two engines on one GPU, driven by
paper_1809_07726_gb300/shard.py with an in-process all-gather (two host
threads): the engines' local walkers, condition maps, acceptance counts and
observables must equal those of one engine over the whole grid, bit for bit.
Each engine computes only its own walkers; exchanges run from the gathered
per-walker rows in each engine's kernel."""
import threading

import numpy as np
import pytest

from paper_1809_07726_gb300 import build, cphremd, shard, synth

pytestmark = pytest.mark.gpu

KW = dict(mc_ph_every=3, mc_redox_every=4, exchange_every=5)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()


def _systems_grid(kind="ragged"):
    """ragged: three systems of 300, 130 and 45 atoms, one per T index (E and
    pH lines stay within a system; T pairs cross systems and are skipped);
    single: one 200-atom system at every slot (exchanges along all three
    dimensions)."""
    nE, npH, nT = 3, 2, 3
    sos = np.zeros(nE * npH * nT, np.int32)
    if kind == "ragged":
        systems = [synth.make_system(300, 71, n_ph=3, ph_atoms=(6, 10), ph_states=(2, 3)),
                   synth.make_system(130, 72, n_ph=2),
                   synth.make_system(45, 73, n_ph=1, redox_atoms=8)]
        for iT in range(nT):
            for ipH in range(npH):
                for iE in range(nE):
                    sos[synth.slot_index(iE, ipH, iT, nE, npH)] = iT
    else:
        systems = [synth.make_system(200, 74, n_ph=3, ph_atoms=(6, 8), ph_states=(2, 3))]
    grid = synth.Grid(np.array([-0.26, -0.2, -0.14]), np.array([4.5, 6.0]), np.array([300.0, 318.0, 337.0]),
                      sos, order=("E", "pH", "T"))
    return systems, grid


class _Gather:
    def __init__(self, n):
        self.b = threading.Barrier(n)
        self.slots = [None] * n

    def rank(self, r):
        def g(rows):
            self.slots[r] = rows
            self.b.wait()
            out = list(self.slots)
            self.b.wait()
            return out
        return g


@pytest.mark.parametrize("prec,kind", [(cphremd.PREC_FP32, "ragged"), (cphremd.PREC_FP64, "ragged"),
                                       (cphremd.PREC_FP32, "single")])
def test_two_sharded_engines_equal_one_engine_bitwise(prec, kind):
    systems, grid = _systems_grid(kind)
    n_steps = 23
    ref = cphremd.init_system(systems, grid, seed=9, precision=prec, **KW)
    ref.run(n_steps)
    parts = shard.partition([s.n for s in systems], grid.system_of_slot, 2)
    engs = [cphremd.init_system(systems, grid, seed=9, precision=prec, **KW) for _ in parts]
    for e, p in zip(engs, parts):
        e.set_local_walkers(p)
    gather = _Gather(2)
    errors = []

    def drive(r):
        try:
            shard.ShardedRun(engs[r], gather.rank(r), KW["mc_ph_every"], KW["mc_redox_every"],
                             KW["exchange_every"]).run(n_steps)
        except Exception as ex:  # pragma: no cover - reported below
            errors.append(ex)
            gather.b.abort()

    th = [threading.Thread(target=drive, args=(r,)) for r in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errors, errors
    xr, vr, sr = ref.positions(), ref.velocities(), ref.site_states()
    visits_ref = ref.visits()
    occ_sum = np.zeros_like(ref.occupancy()[0])
    stats_ref = ref.accept_stats()
    mc_sum = np.zeros(4, np.int64)
    for e, p in zip(engs, parts):
        assert e.get_step() == n_steps
        np.testing.assert_array_equal(e.condition_map(), ref.condition_map())
        np.testing.assert_array_equal(e.accept_stats()[:6], stats_ref[:6])  # exchange counts: global
        mc_sum += e.accept_stats()[6:]
        x, v, st, vis = e.positions(), e.velocities(), e.site_states(), e.visits()
        for w in p:
            sl = ref.walker_slice(w)
            np.testing.assert_array_equal(x[sl], xr[sl])
            np.testing.assert_array_equal(v[sl], vr[sl])
            so = slice(ref.site_offsets[w], ref.site_offsets[w + 1])
            np.testing.assert_array_equal(st[so], sr[so])
            np.testing.assert_array_equal(vis[w], visits_ref[w])
        occ, n = e.occupancy()
        assert n == n_steps
        occ_sum += occ
    np.testing.assert_array_equal(mc_sum, stats_ref[6:])
    np.testing.assert_array_equal(occ_sum, ref.occupancy()[0])
    assert stats_ref[1] + stats_ref[3] + stats_ref[5] > 0  # some swap was accepted
    if kind == "single":
        assert stats_ref[0] > 0 and stats_ref[2] > 0 and stats_ref[4] > 0  # pairs tried along E, pH, T


def test_sharded_engine_refuses_internal_exchanges():
    systems, grid = _systems_grid()
    e = cphremd.init_system(systems, grid, seed=9, **KW)
    e.set_local_walkers([0, 1, 2])
    e.run(4)  # steps 0..3: no exchange step
    with pytest.raises(cphremd.CphError) as err:
        e.run(2)  # would cross step 5
    assert err.value.code == cphremd.E_STATE
    assert e.get_step() == 4  # nothing ran
    with pytest.raises(cphremd.CphError) as err:
        e.attempt_exchanges()
    assert err.value.code == cphremd.E_STATE
    rows = e.exchange_rows()
    assert sorted(rows["walker"]) == [0, 1, 2]
    with pytest.raises(cphremd.CphError) as err:
        e.exchange_apply(cphremd.DIM_NEXT, rows)  # rows of three walkers for a grid of 18
    assert err.value.code == cphremd.E_INVALID
