"""GPU parity of the engine's hot path against the FP64 oracle, through the C ABI.

Bars (FP32 mode): force RMS relative error <= 1e-5 per walker, every energy
term within 1e-6 relative, Born radii within 5e-6 (see R_REL).  FP64: 1e-10.
With CPH_ERROR_LOG set, the achieved errors are appended there (errlog).
Sizes span several 128-atom tiles with ragged tails, several systems batched
in one launch, and the full 384-walker 3D grid (sampled walkers)."""
import numpy as np
import pytest

import errlog
import oracle
from paper_1809_07726_gb300 import build, cphremd, synth

pytestmark = pytest.mark.gpu

FORCE_RMS = 1e-5
ENERGY_REL = 1e-6
# Born radii are an intermediate with no bar of their own.  Their error floor
# is the FP32 rounding of the walker-relative coordinates the pair kernels
# read (half an ulp of up to 42 A, ~2e-6 A): with nothing else rounded, psi
# of the 8000-atom system moves by up to 1.1e-6 relative and R by up to
# 9.3e-7 (1/R = 1/rt - tanh(theta)/rho passes the relative error of psi on
# with the factor R (1 - tanh^2) theta' psi / rho <= 2.0 here).  The FP32 pair
# arithmetic adds rounding of the same order; 5e-6 is five times the input
# floor.
R_REL = 5e-6


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()


def _grid_for(systems, per_system=2):
    sos = np.repeat(np.arange(len(systems)), per_system).astype(np.int32)
    W = len(sos)
    return synth.Grid(np.linspace(-0.3, -0.1, W), np.array([7.0]), np.array([300.0]), sos,
                      order=("E",))


def _compare_walker(eng, w, sysd, x, q, tol_f, tol_e, tol_r, gb=None, case=None):
    o = oracle.OSystem(sysd)
    terms, Fo, Ro, _ = oracle.energy(o, x, q, gb or oracle.GBParams())
    sl = eng.walker_slice(w)
    F = eng.forces()[sl]
    R = eng.born_radii()[sl]
    E = eng.energies()[w]
    rms = np.sqrt(((F - Fo) ** 2).mean()) / np.sqrt((Fo ** 2).mean())
    if case:
        # relative error per energy term; absolute (kcal/mol) for a term that
        # vanishes at this geometry (bonds and angles at their rest values)
        ee = {(f"energy_rel_{cphremd.TERMS[t]}" if abs(terms[t]) > 1e-6 else f"energy_abs_{cphremd.TERMS[t]}"):
              abs(E[t] - terms[t]) / (abs(terms[t]) if abs(terms[t]) > 1e-6 else 1.0) for t in range(6)}
        errlog.record(case, walker=w, atoms=sysd.n, force_rms_rel=rms,
                      born_radius_max_rel=(np.abs(R - Ro) / np.abs(Ro)).max(), **ee)
    assert rms <= tol_f, f"walker {w}: force rms rel {rms:.3e}"
    np.testing.assert_allclose(R, Ro, rtol=tol_r)
    for t in range(6):
        assert abs(E[t] - terms[t]) <= tol_e * abs(terms[t]) + 1e-9, (t, E[t], terms[t])
    return rms


@pytest.fixture(scope="module")
def ragged_systems():
    return [synth.make_system(700, 21, n_ph=3, ph_atoms=(6, 12), ph_states=(2, 4)),
            synth.make_system(130, 22, n_ph=1),
            synth.make_system(40, 23, n_ph=1, redox_atoms=8)]


@pytest.mark.parametrize("prec,tf,te,tr,shapes", [
    (cphremd.PREC_FP32, FORCE_RMS, ENERGY_REL, R_REL, None),
    (cphremd.PREC_FP32, FORCE_RMS, ENERGY_REL, R_REL, (0, 1, 1)),  # mixed tile shapes in one launch
    (cphremd.PREC_FP32, FORCE_RMS, ENERGY_REL, R_REL, (1, 1, 1)),
    (cphremd.PREC_FP64, 1e-10, 1e-10, 1e-11, None)])
def test_evaluate_matches_oracle_ragged_batch(ragged_systems, prec, tf, te, tr, shapes):
    grid = _grid_for(ragged_systems)
    eng = cphremd.init_system(ragged_systems, grid, seed=3, precision=prec)
    for k, sh in enumerate(shapes or ()):
        eng.set_tile_shape(k, sh)
    if shapes:
        np.testing.assert_array_equal(eng.tile_shapes(), shapes)
    eng.evaluate()
    for w in range(grid.n_slots):
        s = ragged_systems[grid.system_of_slot[w]]
        _compare_walker(eng, w, s, s.x, s.q, tf, te, tr)


@pytest.mark.parametrize("shapes", [(0, 0, 0), (1, 0, 1)])
def test_batched_equals_per_replica_bitwise(ragged_systems, shapes):
    grid = _grid_for(ragged_systems)
    a = cphremd.init_system(ragged_systems, grid, seed=3)
    b = cphremd.init_system(ragged_systems, grid, seed=3)
    b.set_launch_mode(cphremd.LAUNCH_PER_REPLICA)
    c = cphremd.init_system(ragged_systems, grid, seed=3)
    c.set_launch_mode(cphremd.LAUNCH_PER_REPLICA)
    c.set_replica_streams(4)  # walkers on four streams, forked and joined per sequence
    for e in (a, b, c):
        for k, sh in enumerate(shapes):
            e.set_tile_shape(k, sh)
    a.run(25)
    b.run(25)
    c.run(25)
    for get in ("positions", "velocities", "forces", "born_radii", "site_states",
                "condition_map"):
        np.testing.assert_array_equal(getattr(a, get)(), getattr(b, get)())
        np.testing.assert_array_equal(getattr(a, get)(), getattr(c, get)())


def test_runs_are_deterministic(ragged_systems):
    grid = _grid_for(ragged_systems)
    a = cphremd.init_system(ragged_systems, grid, seed=5)
    b = cphremd.init_system(ragged_systems, grid, seed=5)
    a.run(30)
    b.run(30)
    np.testing.assert_array_equal(a.positions(), b.positions())
    np.testing.assert_array_equal(a.energies(), b.energies())


def test_graph_replay_equals_direct_steps(ragged_systems):
    """cph_run replays a captured CUDA graph for whole schedule periods; the
    same steps launched one by one give identical results."""
    grid = _grid_for(ragged_systems)
    a = cphremd.init_system(ragged_systems, grid, seed=9, mc_ph_every=5, mc_redox_every=5,
                            exchange_every=10)
    b = cphremd.init_system(ragged_systems, grid, seed=9, mc_ph_every=5, mc_redox_every=5,
                            exchange_every=10)
    a.run(41)            # step 0 direct, then 4 graph periods of 10
    for _ in range(41):  # one step per call: never a whole period
        b.run(1)
    for get in ("positions", "velocities", "site_states", "condition_map", "accept_stats"):
        np.testing.assert_array_equal(getattr(a, get)(), getattr(b, get)())


@pytest.mark.parametrize("shapes", [None, (1, 0, 0)])
def test_full_3d_grid_sampled_walkers(shapes):
    """The 384-walker E x T x pH grid over 500/2000/8000-atom systems in one
    batched launch: one walker of each system against the oracle (all
    systems on symmetric tiles, and the 500-atom one on one warp per atom)."""
    systems, grid = synth.config_c4()
    eng = cphremd.init_system(systems, grid, seed=4)
    for k, sh in enumerate(shapes or ()):
        eng.set_tile_shape(k, sh)
    eng.evaluate()
    for w in (0, 2 * 64 + 5, 5 * 64 + 63):
        s = systems[grid.system_of_slot[w]]
        _compare_walker(eng, w, s, s.x, s.q, FORCE_RMS, ENERGY_REL, R_REL,
                        case="3D grid, 384 walkers (FP32" + (", shapes %s)" % (shapes,) if shapes else ")"))


def test_reference_energies_match_oracle(ragged_systems):
    grid = _grid_for(ragged_systems)
    eng = cphremd.init_system(ragged_systems, grid, seed=1)
    got = eng.reference_energies()
    want = np.concatenate([np.concatenate(oracle.reference_energies(oracle.OSystem(s), s,
                                                                    oracle.GBParams()))
                           for s in ragged_systems])
    np.testing.assert_allclose(got, want, rtol=1e-11, atol=1e-11)


def _band(x, prec):
    # decisions closer to the threshold than the exponent's error bound are
    # logged, not failed: FP64 1e-9 max(1,|x|); FP32 2e-4 max(1,|x|) (the
    # rounding of a dU summed from ~1e5 FP32 pair terms, with a 10x margin)
    return (1e-9 if prec == cphremd.PREC_FP64 else 2e-4) * max(1.0, abs(x))


@pytest.mark.parametrize("prec", [cphremd.PREC_FP32, cphremd.PREC_FP64])
@pytest.mark.parametrize("kappa,rgbmax", [(0.0, 0.0), (0.1, 0.0), (0.0, 10.0)])
def test_mc_sweep_matches_oracle(prec, kappa, rgbmax):
    """One protonation + redox sweep on the 2400-atom system with 20 pH sites:
    dU against the oracle's full recomputation, identical decisions; without
    salt, with Debye-Hueckel screening (kappa = 0.1 / A), and with a 10 A
    Born-radius cutoff (which the sites' reference compounds see too)."""
    _mc_sweep_vs_oracle(prec, kappa, rgbmax)


def test_mc_sweep_on_the_warp_per_atom_shape_matches_oracle():
    """The same in FP32 with the system on one warp per atom: the per-site
    kernel then reads its partners from the FP64 master arrays instead of the
    symmetric tiles' FP32 staging."""
    _mc_sweep_vs_oracle(cphremd.PREC_FP32, 0.0, 0.0, warp=True)


def _mc_sweep_vs_oracle(prec, kappa, rgbmax, warp=False):
    systems, grid = synth.config_c3()
    grid = synth.Grid(grid.E[[0, 3, 5, 7]], grid.pH[[0, 4]], grid.T, np.zeros(8, np.int32),
                      order=("E", "pH"))
    gb = cphremd.GBParams(1.0, 78.5, 0.09, 0.8, 0.0, 2.909125, kappa, 0.0, 1.4, rgbmax)
    eng = cphremd.init_system(systems, grid, seed=11, precision=prec, gb=gb)
    if warp:
        eng.set_tile_shape(0, cphremd.SHAPE_WARP_PER_ATOM)
    eng.set_step(10)
    eng.mc_titrate(cphremd.MC_BOTH)
    recs = eng.mc_records()
    W = oracle.Walkers(systems, grid, seed=11, gb=oracle.GBParams(kappa=kappa, rgbmax=rgbmax))
    for w in range(grid.n_slots):
        oracle.mc_sweep(W, w, "ph", 10)
        oracle.mc_sweep(W, w, "redox", 10)
    by_w = {}
    for (w, k, a, b, dU, x, lnu, acc) in W.mc_log:
        by_w.setdefault(w, []).append((k, a, b, dU, x, lnu, acc))
    n_checked = n_band = 0
    so = eng.site_offsets
    for w, lst in by_w.items():
        for (k, a, b, dU, x, lnu, acc) in lst:
            r = recs[so[w] + k]
            assert (r.walker, r.site, r.frm, r.to) == (w, k, a, b)
            tol = (1e-9 if prec == cphremd.PREC_FP64 else 2e-6) * max(1.0, abs(dU)) + \
                  (1e-9 if prec == cphremd.PREC_FP64 else 1e-4)
            assert abs(r.dU - dU) <= tol, (w, k, r.dU, dU)
            assert r.lnu == lnu
            n_checked += 1
            if abs(lnu - x) <= _band(x, prec):
                n_band += 1
                break  # later sites of this walker see different charges
            assert bool(r.accepted) == bool(acc), (w, k, r.x, x, lnu)
    assert n_checked >= 100 and n_band <= 2


@pytest.mark.parametrize("prec,tex", [(cphremd.PREC_FP64, "potential"), (cphremd.PREC_FP32, "potential"),
                                      (cphremd.PREC_FP64, "semigrand"), (cphremd.PREC_FP32, "semigrand")])
def test_exchange_attempts_match_oracle(prec, tex):
    """pH and E exchanges (integer counts: exact exponents) and T exchanges
    (energies from the engine vs the oracle) on an 4 x 2 x 3 grid, in both
    precision modes.  The T exponent (1/kT_i - 1/kT_j)(U_i - U_j) carries the
    mode's energy bar: |dx| <= |1/kT_i - 1/kT_j| e (S_i + S_j), e = 1e-6 (FP32)
    or 1e-10 (FP64), S = sum of the magnitudes of a walker's energy terms; a decision inside
    that band (or the MC band 2e-4 max(1,|x|), whichever is wider) is counted,
    and the oracle then follows the engine's condition map.  "semigrand" runs
    eq (5) on U - sum U_ref + sum_redox F N_e (E - E0_ref) (CPH_TEX_SEMIGRAND)
    against the oracle's exchange_energy of the same reading."""
    s = synth.make_system(300, 31, n_ph=6, ph_atoms=(6, 8), ph_states=(2, 3))
    grid = synth.Grid(np.linspace(-0.28, -0.16, 4), np.array([4.0, 6.0]),
                      np.array([300.0, 330.0, 363.0]), np.zeros(24, np.int32),
                      order=("E", "pH", "T"))
    tex_code = cphremd.TEX_SEMIGRAND if tex == "semigrand" else cphremd.TEX_POTENTIAL
    eng = cphremd.init_system([s], grid, seed=13, precision=prec, t_exchange_energy=tex_code)
    rng = np.random.default_rng(0)
    so = eng.site_offsets
    states = np.zeros(int(so[-1]), np.int32)
    for w in range(24):
        for k, st in enumerate(s.sites):
            states[so[w] + k] = rng.integers(len(st.q))
    eng.set_site_states(states)
    x = eng.positions()
    for w in range(24):
        x[eng.walker_slice(w)] += rng.normal(0, 0.05, size=(s.n, 3))
    eng.set_positions(x)
    W = oracle.Walkers([s], grid, seed=13, t_energy=tex)
    scale = np.zeros(24)
    for w in range(24):
        W.state[w] = states[so[w]:so[w + 1]].astype(np.int64)
        q = s.q.copy()
        for k, st in enumerate(s.sites):
            q[st.atoms] = st.q[W.state[w][k]]
        W.q[w] = q
        W.x[w] = np.ascontiguousarray(x[eng.walker_slice(w)])
        terms = oracle.energy(W.osys[0], W.x[w], q, forces=False)[0]
        W.U[w] = terms[5]
        scale[w] = np.abs(terms[:5]).sum()
    eng.set_step(100)
    seen = n_band = 0
    worst = 0.0
    for dim in ("E", "pH", "T", "E", "pH", "T"):
        eng.attempt_exchanges(cphremd.DIM_NAMES[dim])
        recs = [r for r in eng.exchange_records() if r.accepted >= 0]
        n0 = len(W.ex_log)
        oracle.exchange_attempt(W, dim, 100)
        ol = W.ex_log[n0:]
        assert len(recs) == len(ol)
        key = {(e[1], e[2]): e for e in ol}
        resync = False
        for r in recs:
            e = key[(r.slot_lo, r.slot_hi)]
            assert (r.walker_lo, r.walker_hi) == (e[3], e[4])
            assert r.lnu == e[6]
            tol = 1e-9 * max(1.0, abs(e[5]))
            if dim == "T":  # the energy bar of the mode, carried through eq (5)
                Ti, Tj = W.grid.T[r.slot_lo // 8], W.grid.T[r.slot_hi // 8]
                dbeta = abs(1.0 / (oracle.KB * Ti) - 1.0 / (oracle.KB * Tj))
                ebar = ENERGY_REL if prec == cphremd.PREC_FP32 else 1e-10
                tol = max(tol, dbeta * ebar * (scale[e[3]] + scale[e[4]]))
            assert abs(r.x - e[5]) <= tol, (dim, r.x, e[5], tol)
            worst = max(worst, abs(r.x - e[5]))
            seen += 1
            band = max(tol, _band(e[5], prec))
            if abs(e[6] - e[5]) <= band:
                n_band += 1
                resync = resync or bool(r.accepted) != bool(e[7])
                continue
            assert bool(r.accepted) == bool(e[7])
        if resync:  # a decision inside the band went the other way: follow the engine
            W.slot_of[:] = eng.condition_map()
            W.walker_at[W.slot_of] = np.arange(24)
        np.testing.assert_array_equal(eng.condition_map(), W.slot_of)
    errlog.record(f"exchange exponents ({'FP32' if prec == cphremd.PREC_FP32 else 'FP64'}, {tex})",
                  pairs=seen, max_abs_x_err=worst, decisions_in_band=n_band)
    assert seen > 20 and n_band <= 2


def test_fp64_whole_schedule_matches_oracle():
    """160-atom system, 8 walkers along E, FP64 mode: 120 steps of the full
    schedule (MC every 10, exchange every 20) agree with the oracle to 1e-9 A."""
    systems, grid = synth.config_c2()
    eng = cphremd.init_system(systems, grid, seed=2, precision=cphremd.PREC_FP64,
                              mc_ph_every=10, mc_redox_every=10, exchange_every=20)
    W = oracle.Walkers(systems, grid, seed=2, mc_ph=10, mc_redox=10, exchange_every=20)
    n = 120
    eng.run(n)
    oracle.run_schedule(W, n)
    x = eng.positions()
    for w in range(grid.n_slots):
        np.testing.assert_allclose(x[eng.walker_slice(w)], W.x[w], rtol=0, atol=1e-9)
    np.testing.assert_array_equal(eng.condition_map(), W.slot_of)
    np.testing.assert_array_equal(eng.site_states(), np.concatenate(W.state))
    # sampling observables: identical decisions give identical integer counts
    occ, n_samples = eng.occupancy()
    assert n_samples == W.n_obs == n
    for s in range(grid.n_slots):
        rows = occ[eng.site_offsets[s]:eng.site_offsets[s + 1]]
        np.testing.assert_array_equal(rows, W.occ[s])
    np.testing.assert_array_equal(eng.visits(), W.visits)
    np.testing.assert_allclose(eng.fractions(), np.concatenate(oracle.site_fractions(W)),
                               rtol=1e-14, atol=0)


def test_fp32_langevin_step_matches_oracle():
    """One MD step in FP32 mode from a shared state.  The step's velocity and
    displacement inherit the force error (RMS 1e-5 bar) and the FP32
    Box-Muller normals (~1e-7), so both are held to RMS relative 1e-5."""
    s = synth.make_system(260, 41, n_ph=1)
    grid = synth.Grid(np.array([-0.2]), np.array([7.0]), np.array([310.0]), np.zeros(1, np.int32))
    eng = cphremd.init_system([s], grid, seed=17)
    eng.set_step(7)
    eng.step_replicas(1)
    W = oracle.Walkers([s], grid, seed=17)
    W.t = 7
    oracle.run_schedule(W, 1)

    def rel_rms(a, b):
        return np.sqrt(((a - b) ** 2).mean()) / np.sqrt((b ** 2).mean())

    assert rel_rms(eng.velocities(), W.v[0]) <= FORCE_RMS
    assert rel_rms(eng.positions() - s.x, W.x[0] - s.x) <= FORCE_RMS


def test_nonfinite_state_is_reported_not_hidden():
    """Two non-excluded atoms placed on the same point make the pair sums
    non-finite; the fixed-point accumulators must not hide that: cph_status
    reports CPH_E_NONFINITE (no fault, only arithmetic)."""
    s = synth.make_system(300, 51, n_ph=1)
    grid = synth.Grid(np.array([-0.2]), np.array([7.0]), np.array([300.0]), np.zeros(1, np.int32))
    eng = cphremd.init_system([s], grid, seed=1)
    eng.evaluate()
    eng.status()
    x = eng.positions()
    x[200] = x[20]
    eng.set_positions(x)
    eng.evaluate()
    with pytest.raises(cphremd.CphError) as ei:
        eng.status()
    assert ei.value.code == cphremd.E_NONFINITE


def test_autotuned_work_item_size_changes_nothing_but_speed(ragged_systems):
    """The symmetric tiles' work-item size only changes speed: fixed-point sums
    make the trajectory bitwise identical to the default size (the shapes held
    at symmetric after tuning)."""
    grid = _grid_for(ragged_systems)
    a = cphremd.init_system(ragged_systems, grid, seed=21)
    b = cphremd.init_system(ragged_systems, grid, seed=21)
    chunk = a.autotune()
    assert chunk in (8, 16, 24, 32, 48, 64, 96, 128)
    for k in range(len(ragged_systems)):
        a.set_tile_shape(k, cphremd.SHAPE_SYMMETRIC)
    a.run(20)
    b.run(20)
    np.testing.assert_array_equal(a.positions(), b.positions())
    np.testing.assert_array_equal(a.forces(), b.forces())


def test_autotuned_tile_shapes_meet_the_bars(ragged_systems):
    """Whatever per-system shapes the autotuner picks (smallest systems on one
    warp per atom up to a tuned size), the results meet the FP32 bars; the
    shapes it reports follow its size rule."""
    grid = _grid_for(ragged_systems)
    eng = cphremd.init_system(ragged_systems, grid, seed=3)
    eng.autotune()
    sh = eng.tile_shapes()
    sizes = np.array([s.n for s in ragged_systems])
    if sh.any():
        assert sizes[sh == 1].max() < sizes[sh == 0].min() if (sh == 0).any() else True
    eng.evaluate()
    for w in range(grid.n_slots):
        s = ragged_systems[grid.system_of_slot[w]]
        _compare_walker(eng, w, s, s.x, s.q, FORCE_RMS, ENERGY_REL, R_REL)


def test_checkpoint_restart_continues_bitwise(ragged_systems):
    """A run restored from a checkpoint continues exactly as the run that
    wrote it, whatever seed the restoring engine was built with; a checkpoint
    of another layout is refused."""
    grid = _grid_for(ragged_systems)
    kw = dict(mc_ph_every=3, mc_redox_every=4, exchange_every=5)
    a = cphremd.init_system(ragged_systems, grid, seed=13, **kw)
    a.run(23)
    ck = a.get_state()
    a.run(37)
    b = cphremd.init_system(ragged_systems, grid, seed=99, **kw)
    b.set_state(ck)
    assert b.get_step() == 23
    b.run(37)
    for get in ("positions", "velocities", "site_states", "condition_map", "accept_stats",
                "visits", "charges"):
        np.testing.assert_array_equal(getattr(a, get)(), getattr(b, get)())
    np.testing.assert_array_equal(a.occupancy()[0], b.occupancy()[0])
    assert a.get_step() == b.get_step() == 60
    small = ragged_systems[:2]
    c = cphremd.init_system(small, _grid_for(small), seed=13, **kw)
    with pytest.raises(cphremd.CphError) as err:
        c.set_state(ck)
    assert err.value.code == cphremd.E_INVALID


# OBC model II ("igb=5"), model I with other dielectric constants, model I with
# salt screening, model II with salt and the surface term, and Born-radius
# cutoffs (8 A cuts through all three ragged systems, 12 A through the largest
# with the other variants on): the GB variants are parameter sets of the same
# kernels (the cutoff selects the band-aware tile variant)
GB_VARIANTS = [dict(eps_in=1.0, eps_out=78.5, offset=0.09, alpha=1.0, beta=0.8, gamma=4.85, kappa=0.0),
               dict(eps_in=2.0, eps_out=80.0, offset=0.09, alpha=0.8, beta=0.0, gamma=2.909125, kappa=0.0),
               dict(eps_in=1.0, eps_out=78.5, offset=0.09, alpha=0.8, beta=0.0, gamma=2.909125,
                    kappa=0.1),  # Debye-Hueckel salt screening
               dict(eps_in=1.0, eps_out=78.5, offset=0.09, alpha=1.0, beta=0.8, gamma=4.85,
                    kappa=0.05, sa_gamma=0.005, sa_probe=1.4),  # + ACE surface term
               dict(eps_in=1.0, eps_out=78.5, offset=0.09, alpha=0.8, beta=0.0, gamma=2.909125,
                    kappa=0.0, rgbmax=8.0),  # Born-radius cutoff
               dict(eps_in=1.0, eps_out=78.5, offset=0.09, alpha=1.0, beta=0.8, gamma=4.85,
                    kappa=0.05, sa_gamma=0.005, sa_probe=1.4, rgbmax=12.0)]


def test_cutoff_beyond_every_pair_changes_nothing(ragged_systems):
    """A Born-radius cutoff farther than every pair separation plus s_max
    leaves the band-aware FP32 tiles on exactly the arithmetic of the plain
    ones (bitwise equal results); an 8 A cutoff does change the radii."""
    grid = _grid_for(ragged_systems)
    out = []
    for rc in (0.0, 1000.0, 8.0):
        gb = cphremd.default_gb()
        gb.rgbmax = rc
        eng = cphremd.init_system(ragged_systems, grid, seed=3, gb=gb)
        eng.evaluate()
        out.append((eng.born_radii(), eng.forces(), eng.energies()))
    for a, b in zip(out[0], out[1]):
        np.testing.assert_array_equal(a, b)
    # fewer descreening shells: smaller psi and so smaller radii
    R0, R8 = out[0][0], out[2][0]
    assert (R8 <= R0 * (1 + 1e-6)).all() and (R8 < R0 * (1 - 1e-4)).mean() > 0.5


@pytest.mark.parametrize("prec,tf,te,tr,warp", [(cphremd.PREC_FP32, FORCE_RMS, ENERGY_REL, R_REL, False),
                                                (cphremd.PREC_FP32, FORCE_RMS, ENERGY_REL, R_REL, True),
                                                (cphremd.PREC_FP64, 1e-10, 1e-10, 1e-11, False)])
@pytest.mark.parametrize("v", GB_VARIANTS)
def test_gb_variants_match_oracle(ragged_systems, v, prec, tf, te, tr, warp):
    """Every GB variant on both FP32 tile shapes (warp: every system on one
    warp per atom) and in FP64 mode."""
    grid = _grid_for(ragged_systems)
    gb = cphremd.GBParams(v["eps_in"], v["eps_out"], v["offset"], v["alpha"], v["beta"], v["gamma"],
                          v["kappa"], v.get("sa_gamma", 0.0), v.get("sa_probe", 1.4),
                          v.get("rgbmax", 0.0))
    eng = cphremd.init_system(ragged_systems, grid, seed=3, precision=prec, gb=gb)
    if warp:
        for k in range(len(ragged_systems)):
            eng.set_tile_shape(k, cphremd.SHAPE_WARP_PER_ATOM)
    eng.evaluate()
    og = oracle.GBParams(**v)
    for w in range(grid.n_slots):
        s = ragged_systems[grid.system_of_slot[w]]
        _compare_walker(eng, w, s, s.x, s.q, tf, te, tr, gb=og)
