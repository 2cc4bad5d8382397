"""GPU parity on the degenerate inputs of the method, batched with ordinary
systems in one launch: a lone titratable atom (no pair at all), two and three
atoms (fewer atoms than one tile), a system without sites, one without
bonded terms, a site at the 64-atom limit with four states, and
eps_in = eps_out (tau = 0: no GB energy).  Each is checked against the FP64
oracle: energies, forces and Born radii after an evaluation, and every MC
decision of a sweep."""
import copy

import numpy as np
import pytest

import oracle
from paper_1809_07726_gb300 import build, cphremd, synth

pytestmark = pytest.mark.gpu

FORCE_RMS = 1e-5
ENERGY_REL = 1e-6
R_REL = 5e-6


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()


def _no_bonded(s):
    s = copy.deepcopy(s)
    s.bonds = np.zeros((0, 2), np.int32)
    s.bond_k = np.zeros(0)
    s.bond_r0 = np.zeros(0)
    s.angles = np.zeros((0, 3), np.int32)
    s.angle_k = np.zeros(0)
    s.angle_t0 = np.zeros(0)
    return s


@pytest.fixture(scope="module")
def odd_systems():
    return [synth.titratable_ion("ph", 4.4),                                # 1 atom, 1 site
            synth.make_system(2, 41, n_redox=0),                             # 2 atoms, no site
            synth.make_system(3, 42, n_redox=0),                             # 3 atoms
            synth.make_system(200, 43, n_ph=1, ph_atoms=(64, 64), ph_states=(4, 4),
                              n_redox=0),                                    # 64-atom site
            _no_bonded(synth.make_system(50, 44, n_ph=2)),                   # no bonded terms
            synth.make_system(290, 45, n_ph=3, ph_atoms=(6, 12), ph_states=(2, 4))]


def _grid(systems):
    sos = np.repeat(np.arange(len(systems)), 2).astype(np.int32)
    return synth.Grid(np.linspace(-0.3, -0.1, len(sos)), np.array([5.0]), np.array([300.0]), sos,
                      order=("E",))


def _gb(eps_out):
    g = cphremd.default_gb()
    g.eps_out = eps_out
    return g


def _compare(eng, w, s, gb, tf, te, tr, scale_of=None):
    """Energies within te of |E| (or of scale_of[t], a term's condition
    number, where given); forces within tf of the oracle's RMS force, with an
    absolute floor of 1e-9 kcal/mol/A where every force is rounding noise."""
    terms, Fo, Ro, _ = oracle.energy(oracle.OSystem(s), s.x, s.q, gb)
    sl = eng.walker_slice(w)
    F, R, E = eng.forces()[sl], eng.born_radii()[sl], eng.energies()[w]
    np.testing.assert_allclose(R, Ro, rtol=tr)
    scale = np.sqrt((Fo ** 2).mean())
    assert np.sqrt(((F - Fo) ** 2).mean()) <= tf * scale + 1e-9
    bad = []
    comp = [max(abs(terms[t]), (scale_of or {}).get(t, 0.0)) for t in range(5)]
    for t in range(6):
        ref = max(abs(terms[t]), (scale_of or {}).get(t, 0.0))
        if t == 5 and scale_of:
            ref = max(ref, sum(comp))  # the total of cancelling components
        if not abs(E[t] - terms[t]) <= te * ref + 1e-9:
            bad.append((t, E[t], terms[t], ref))
    assert not bad, (w, bad)
    return terms


def _lj_abs_sum(s, x):
    """sum over non-excluded pairs of |4 eps_ij ((sig_ij/r)^12 - (sig_ij/r)^6)|
    (exclusions: 1-2 and 1-3 pairs of the bond graph, Lorentz-Berthelot
    mixing): the scale an FP32 sum of those terms is exact to."""
    n = s.n
    excl = np.zeros((n, n), bool)
    for i, j in s.bonds:
        excl[i, j] = excl[j, i] = True
    for i, _, k in s.angles:
        excl[i, k] = excl[k, i] = True
    iu = np.triu_indices(n, 1)
    keep = ~excl[iu]
    i, j = iu[0][keep], iu[1][keep]
    r = np.linalg.norm(x[i] - x[j], axis=1)
    sig = 0.5 * (s.sigma[i] + s.sigma[j])
    e = np.sqrt(s.eps[i] * s.eps[j])
    sr6 = (sig / r) ** 6
    return float(np.abs(4 * e * (sr6 * sr6 - sr6)).sum())


@pytest.mark.parametrize("prec,tf,te,tr", [(cphremd.PREC_FP32, FORCE_RMS, ENERGY_REL, R_REL),
                                           (cphremd.PREC_FP64, 1e-10, 1e-10, 1e-11)])
@pytest.mark.parametrize("eps_out", [78.5, 1.0])
def test_degenerate_systems_evaluate_matches_oracle(odd_systems, prec, tf, te, tr, eps_out):
    grid = _grid(odd_systems)
    eng = cphremd.init_system(odd_systems, grid, seed=2, precision=prec, gb=_gb(eps_out))
    eng.evaluate()
    og = oracle.GBParams(eps_out=eps_out)
    for w in range(grid.n_slots):
        s = odd_systems[grid.system_of_slot[w]]
        terms = _compare(eng, w, s, og, tf, te, tr)
        if eps_out == 1.0:
            assert terms[0] == 0.0 and eng.energies()[w][0] == 0.0  # tau = 0: no GB energy
    # the lone atom: Born's radius rho - offset, no pair term
    R0 = eng.born_radii()[eng.walker_slice(0)]
    assert R0[0] == pytest.approx(odd_systems[0].rho[0] - 0.09, rel=1e-12)


@pytest.mark.parametrize("prec", [cphremd.PREC_FP32, cphremd.PREC_FP64])
def test_degenerate_systems_mc_sweep_matches_oracle(odd_systems, prec):
    """Every walker's pH and redox sweep against the oracle's full
    recomputation: the same proposals, dU within the bar, the same decisions
    (decisions inside the exponent's error band are skipped, as in the main
    MC test); systems without sites produce no record."""
    grid = _grid(odd_systems)
    eng = cphremd.init_system(odd_systems, grid, seed=7, precision=prec)
    eng.set_step(20)
    eng.mc_titrate(cphremd.MC_BOTH)
    recs = eng.mc_records()
    W = oracle.Walkers(odd_systems, grid, seed=7, gb=oracle.GBParams())
    for w in range(grid.n_slots):
        oracle.mc_sweep(W, w, "ph", 20)
        oracle.mc_sweep(W, w, "redox", 20)
    so = eng.site_offsets
    n_checked = 0
    done = set()
    for (w, k, a, b, dU, x, lnu, acc) in W.mc_log:
        if w in done:
            continue
        r = recs[so[w] + k]
        assert (r.walker, r.site, r.frm, r.to) == (w, k, a, b)
        tol = (1e-9 if prec == cphremd.PREC_FP64 else 2e-6) * max(1.0, abs(dU)) + \
              (1e-9 if prec == cphremd.PREC_FP64 else 1e-4)
        assert abs(r.dU - dU) <= tol, (w, k, r.dU, dU)
        assert r.lnu == lnu
        n_checked += 1
        band = (1e-9 if prec == cphremd.PREC_FP64 else 2e-4) * max(1.0, abs(x))
        if abs(lnu - x) <= band:
            done.add(w)  # later sites of this walker see different charges
            continue
        assert bool(r.accepted) == bool(acc), (w, k, r.x, x, lnu)
    n_sites = sum(len(odd_systems[grid.system_of_slot[w]].sites) for w in range(grid.n_slots))
    assert n_checked >= n_sites - 4
    assert len(so) == grid.n_slots + 1


def test_site_less_batch_runs_with_mc_switched_on():
    """MC every step on walkers that have no site: nothing to sweep, the
    schedule still runs (MD, exchanges, observables) and stays finite."""
    systems = [synth.make_system(40, 51, n_redox=0), synth.make_system(3, 52, n_redox=0)]
    grid = _grid(systems)
    eng = cphremd.init_system(systems, grid, seed=3, mc_ph_every=1, mc_redox_every=1,
                              exchange_every=2)
    eng.run(12)
    eng.status()
    assert np.isfinite(eng.positions()).all()
    occ, n = eng.occupancy()
    assert n == 12 and occ.size == 0
    v = eng.visits()
    assert (v.sum(0) == 12).all() and (v.sum(1) == 12).all()


@pytest.mark.parametrize("prec,tf,te,tr,warp", [(cphremd.PREC_FP32, FORCE_RMS, ENERGY_REL, R_REL, False),
                                                (cphremd.PREC_FP32, FORCE_RMS, ENERGY_REL, R_REL, True),
                                                (cphremd.PREC_FP64, 1e-10, 1e-10, 1e-11, False)])
def test_perturbed_geometry_matches_oracle(prec, tf, te, tr, warp):
    """The synthetic chains start at their bond lengths and angles, where the
    bonded terms vanish; here every atom is displaced (0.1 A) and a few angles
    are opened to within ~3 degrees of linear, so bonds, angles (and their
    sine denominators) carry real energies and forces.  The strained contacts
    make the LJ sum cancel (sum |e_ij| ~ 100 |E_LJ|), and the total is a sum
    of components ~100 times larger than itself; FP32 coordinates and pair
    terms are exact to ~1e-7 of each term, so in FP32 E_LJ is held to 1e-6 of
    sum |e_ij| and the total to 1e-6 of the sum of its components' scales
    (every other term to 1e-6 of itself).  warp: both systems on one warp per
    atom (the ordered kernels, whose FP32 bonded terms are the mixed-precision
    form)."""
    systems = [synth.make_system(290, 45, n_ph=3, ph_atoms=(6, 12), ph_states=(2, 4)),
               synth.make_system(1100, 46, n_ph=4)]
    grid = _grid(systems)
    eng = cphremd.init_system(systems, grid, seed=2, precision=prec)
    if warp:
        for k in range(len(systems)):
            eng.set_tile_shape(k, cphremd.SHAPE_WARP_PER_ATOM)
    rng = np.random.default_rng(5)
    x = eng.positions()
    xs = []
    for w in range(grid.n_slots):
        s = systems[grid.system_of_slot[w]]
        xw = s.x + rng.normal(0.0, 0.1, size=(s.n, 3))
        for a in (10, 40, 77):  # nearly straight angle a-1, a, a+1
            xw[a + 1] = xw[a] + 1.5 * (xw[a] - xw[a - 1]) / np.linalg.norm(xw[a] - xw[a - 1]) \
                + rng.normal(0.0, 0.04, 3)
        x[eng.walker_slice(w)] = xw
        xs.append(xw)
    eng.set_positions(x)
    eng.evaluate()
    for w in range(grid.n_slots):
        s = systems[grid.system_of_slot[w]]
        s2 = copy.deepcopy(s)
        s2.x = xs[w]
        cond = {2: _lj_abs_sum(s, xs[w])} if prec == cphremd.PREC_FP32 else None
        terms = _compare(eng, w, s2, oracle.GBParams(), tf, te, tr, cond)
        assert terms[3] > 1.0 and terms[4] > 1.0  # bonds and angles are strained
