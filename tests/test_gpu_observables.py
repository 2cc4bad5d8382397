"""Sampling observables on the GPU: the device counters against a host tally
of the states the engine reports, graph replay against single steps, the
titration fits of titratable ions against eqs (1) and (2), and the counters'
invariants on the 384-replica E x T x pH grid.  (Bit-exact agreement with the
oracle's counters is checked in the FP64 whole-schedule test.)"""
import numpy as np
import pytest

from paper_1809_07726_gb300 import cphremd, synth

pytestmark = pytest.mark.gpu


def _ragged():
    return [synth.make_system(700, 21, n_ph=3, ph_atoms=(6, 12), ph_states=(2, 4)),
            synth.make_system(130, 22, n_ph=1),
            synth.make_system(40, 23, n_ph=1, redox_atoms=8)]


def _grid(systems, per_system=3):
    sos = np.repeat(np.arange(len(systems)), per_system).astype(np.int32)
    return synth.Grid(np.linspace(-0.3, -0.1, len(sos)), np.array([7.0]), np.array([300.0]),
                      sos, order=("E",))


def _tally(eng, occ, visits):
    st, cm, so = eng.site_states(), eng.condition_map(), eng.site_offsets
    for w in range(eng.W):
        s = int(cm[w])
        visits[w, s] += 1
        for k in range(so[w + 1] - so[w]):
            occ[so[s] + k, st[so[w] + k]] += 1


def test_counters_equal_host_tally_and_graph_replay():
    """FP32 ragged batch, MC every 2 / 3 steps, exchange every 2: the sample of
    a step sees the states and condition map that the step leaves behind."""
    systems = _ragged()
    grid = _grid(systems)
    kw = dict(seed=5, mc_ph_every=2, mc_redox_every=3, exchange_every=2)
    a = cphremd.init_system(systems, grid, **kw)
    b = cphremd.init_system(systems, grid, **kw)
    occ = np.zeros((int(a.site_offsets[-1]), cphremd.MAX_STATES), np.int64)
    visits = np.zeros((a.W, a.W), np.int64)
    for _ in range(25):
        a.run(1)
        _tally(a, occ, visits)
    b.run(25)  # step 0 direct, then graph periods of 6
    got, n = a.occupancy()
    assert n == 25
    np.testing.assert_array_equal(got, occ)
    np.testing.assert_array_equal(a.visits(), visits)
    got_b, n_b = b.occupancy()
    assert n_b == 25
    np.testing.assert_array_equal(got_b, occ)
    np.testing.assert_array_equal(b.visits(), visits)
    assert np.count_nonzero(visits - np.diag(np.diag(visits))) > 0, "no exchange happened"
    # fractions are the documented reduction of the counts
    fr = a.fractions()
    so = a.site_offsets
    for s in range(a.W):
        sysd = systems[grid.system_of_slot[s]]
        for k, st in enumerate(sysd.sites):
            n_of = np.asarray(st.n_prot if st.kind == "ph" else st.n_elec, float)
            w = (n_of - n_of.min()) / (n_of.max() - n_of.min())
            want = (occ[so[s] + k, :len(w)] * w).sum() / 25
            assert fr[so[s] + k] == pytest.approx(want, rel=1e-14, abs=1e-300)


def test_reset_and_no_sample():
    ion = synth.titratable_ion("ph", 5.0)
    grid = synth.Grid(np.array([0.0]), np.array([4.0, 6.0]), np.array([300.0]),
                      np.zeros(2, np.int32), order=("pH",))
    eng = cphremd.init_system([ion], grid, seed=1, mc_ph_every=1, mc_redox_every=0,
                              exchange_every=2)
    with pytest.raises(cphremd.CphError) as e:
        eng.fractions()
    assert e.value.code == cphremd.E_STATE
    eng.step_replicas(3)   # plain MD steps are sampled too
    occ, n = eng.occupancy()
    assert n == 3 and (occ.sum(1) == 3).all() and (occ[:, 0] == 3).all()
    eng.reset_observables()
    occ, n = eng.occupancy()
    assert n == 0 and not occ.any() and not eng.visits().any()
    eng.run(4)
    occ, n = eng.occupancy()
    assert n == 4 and (occ.sum(1) == 4).all()


@pytest.mark.parametrize("kind,ref", [("ph", 4.85), ("redox", -0.203)])
def test_ion_titration_fit_recovers_the_reference(kind, ref):
    """Titratable ions along pH (or E) with exchanges: G(s) has no
    electrostatic part, so 40,000 samples per condition follow eq (1) / (2)
    with n = 1, and the native fit returns pKa_ref / E0_ref."""
    ion = synth.titratable_ion(kind, ref)
    if kind == "ph":
        xs = np.linspace(ref - 1.5, ref + 1.5, 7)
        grid = synth.Grid(np.array([0.0]), xs, np.array([300.0]), np.zeros(7, np.int32),
                          order=("pH",))
        eng = cphremd.init_system([ion], grid, seed=8, mc_ph_every=1, mc_redox_every=0,
                                  exchange_every=4)
        want = 1.0 / (1.0 + 10.0 ** (xs - ref))
    else:
        xs = np.linspace(ref - 0.09, ref + 0.09, 7)
        grid = synth.Grid(xs, np.array([7.0]), np.array([300.0]), np.zeros(7, np.int32),
                          order=("E",))
        eng = cphremd.init_system([ion], grid, seed=8, mc_ph_every=0, mc_redox_every=1,
                                  exchange_every=4)
        want = 1.0 / (1.0 + np.exp(23.0605 / (0.0019872041 * 300.0) * (xs - ref)))
    eng.run(40000)
    eng.status()
    f = eng.fractions()
    assert np.abs(f - want).max() < 0.015
    x0, n, _ = cphremd.fit_hill(cphremd.FIT_PH if kind == "ph" else cphremd.FIT_REDOX, xs, f,
                                300.0, 1.0)
    if kind == "ph":
        assert abs(x0 - ref) < 0.03 and abs(n - 1.0) < 0.04
    else:
        assert abs(x0 - ref) < 0.0015 and abs(n - 1.0) < 0.04
    v = eng.visits()
    assert (v.sum(0) == 40000).all() and (v.sum(1) == 40000).all() and (v > 0).all()


def test_counter_invariants_on_the_3d_grid():
    """384 walkers over 500/2000/8000-atom systems: walkers only visit slots
    of their own system and every count sums to the step count."""
    systems, grid = synth.config_c4()
    eng = cphremd.init_system(systems, grid, seed=4, mc_ph_every=2, mc_redox_every=2,
                              exchange_every=2)
    eng.run(12)
    occ, n = eng.occupancy()
    assert n == 12 and (occ.sum(1) == 12).all()
    v = eng.visits()
    assert (v.sum(0) == 12).all() and (v.sum(1) == 12).all()
    sos = np.asarray(grid.system_of_slot)
    assert not v[sos[:, None] != sos[None, :]].any()
    assert np.count_nonzero(v - np.diag(np.diag(v))) > 0
    f = eng.fractions()
    assert ((f >= 0) & (f <= 1)).all()
