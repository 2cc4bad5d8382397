"""Sampling observables on the CPU.

- The oracle's Hill fit of eqs (1) and (2) is pinned to exact curves, to the
  two-point closed form, to local optimality on noisy data and to the
  curves' symmetries.
- The library's native fit (host code, no GPU) must agree with it.
- The oracle's per-step counters are pinned to their invariants and, on
  titratable ions whose free energy has no electrostatic part, to the
  populations eqs (1) and (2) predict.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1809_07726_gb300 import build, cphremd, synth

KB, FARADAY, LN10 = oracle.KB, oracle.FARADAY, oracle.LN10


@pytest.fixture(scope="module")
def native():
    build.build()
    return cphremd


def _noisy_ph(seed, n_pts=9, pka=4.85, n=0.9, sd=0.03):
    rng = np.random.default_rng(seed)
    x = np.linspace(2.5, 7.5, n_pts)
    f = np.clip(oracle.f_prot(x, pka, n) + rng.normal(0, sd, n_pts), 0.0, 1.0)
    return x, f


def _noisy_redox(seed, n_pts=8, e0=-0.203, T=300.0, v=1.0, n=1.0, sd=0.03):
    rng = np.random.default_rng(seed)
    x = np.linspace(-0.33, -0.08, n_pts)
    f = np.clip(oracle.f_red(x, e0, T, v, n) + rng.normal(0, sd, n_pts), 0.0, 1.0)
    return x, f


def _rss(kind, x, f, x0, n, T=300.0, v=1.0):
    m = oracle.f_prot(x, x0, n) if kind == "pH" else oracle.f_red(x, x0, T, v, n)
    return float(np.sum((f - m) ** 2))


# ---------------------------------------------------------------- oracle fit pins

@pytest.mark.parametrize("pka,n", [(4.85, 1.0), (4.4, 0.7), (6.1, 1.6)])
def test_oracle_fit_recovers_exact_eq1_curves(pka, n):
    x = np.linspace(2.0, 9.0, 15)
    x0, nh, rss = oracle.fit_hill("pH", x, oracle.f_prot(x, pka, n))
    assert x0 == pytest.approx(pka, abs=1e-9)
    assert nh == pytest.approx(n, rel=1e-9)
    assert rss < 1e-25


@pytest.mark.parametrize("e0,T,v,n", [(-0.203, 300.0, 1.0, 1.0), (-0.15, 350.0, 1.0, 0.8),
                                      (-0.25, 300.0, 2.0, 1.0)])
def test_oracle_fit_recovers_exact_eq2_curves(e0, T, v, n):
    x = np.linspace(e0 - 0.1, e0 + 0.1, 11)
    x0, nh, rss = oracle.fit_hill("redox", x, oracle.f_red(x, e0, T, v, n), T, v)
    assert x0 == pytest.approx(e0, abs=1e-11)
    assert nh == pytest.approx(n, rel=1e-9)
    assert rss < 1e-25


def test_oracle_fit_two_points_interpolate():
    """Two interior points fix the curve: the Hill plot is the line through
    (x_i, ln((1 - f_i)/f_i) / ln 10) with slope n and root pKa."""
    x, f = np.array([4.0, 6.0]), np.array([0.8, 0.15])
    z = np.log((1 - f) / f) / LN10
    n = (z[1] - z[0]) / (x[1] - x[0])
    pka = x[0] - z[0] / n
    x0, nh, rss = oracle.fit_hill("pH", x, f)
    assert (x0, nh) == (pytest.approx(pka, abs=1e-10), pytest.approx(n, rel=1e-10))
    assert rss < 1e-25


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_oracle_fit_is_the_least_squares_minimum(seed):
    x, f = _noisy_ph(seed)
    x0, n, rss = oracle.fit_hill("pH", x, f)
    assert rss == pytest.approx(_rss("pH", x, f, x0, n), rel=1e-12)
    # brute force over a neighbourhood: nothing lower
    for d0 in np.linspace(-0.2, 0.2, 21):
        for dn in np.linspace(-0.2, 0.2, 21):
            assert _rss("pH", x, f, x0 + d0, n + dn) >= rss - 1e-15
    # stationary: central differences of the residual sum vanish
    h = 1e-6
    g0 = (_rss("pH", x, f, x0 + h, n) - _rss("pH", x, f, x0 - h, n)) / (2 * h)
    g1 = (_rss("pH", x, f, x0, n + h) - _rss("pH", x, f, x0, n - h)) / (2 * h)
    assert abs(g0) < 1e-7 and abs(g1) < 1e-7


def test_oracle_fit_symmetries():
    """Shifting x shifts x0; reflecting f -> 1 - f negates the Hill slope."""
    x, f = _noisy_ph(4)
    x0, n, rss = oracle.fit_hill("pH", x, f)
    a0, an, arss = oracle.fit_hill("pH", x + 1.25, f)
    assert (a0, an, arss) == (pytest.approx(x0 + 1.25, abs=1e-9), pytest.approx(n, rel=1e-9),
                              pytest.approx(rss, rel=1e-9))
    b0, bn, brss = oracle.fit_hill("pH", x, 1.0 - f)
    assert (b0, bn, brss) == (pytest.approx(x0, abs=1e-9), pytest.approx(-n, rel=1e-9),
                              pytest.approx(rss, rel=1e-9))


# ---------------------------------------------------------------- native fit

@pytest.mark.parametrize("seed", range(6))
def test_native_fit_matches_oracle(native, seed):
    x, f = _noisy_ph(seed, n_pts=6 + seed, sd=0.02 + 0.01 * seed)
    want = oracle.fit_hill("pH", x, f)
    got = native.fit_hill(native.FIT_PH, x, f)
    assert got[0] == pytest.approx(want[0], abs=1e-8)
    assert got[1] == pytest.approx(want[1], rel=1e-7)
    assert got[2] == pytest.approx(want[2], rel=1e-9, abs=1e-20)
    T, v = (300.0, 1.0) if seed % 2 == 0 else (341.5, 2.0)
    x, f = _noisy_redox(seed, T=T, v=v)
    want = oracle.fit_hill("redox", x, f, T, v)
    got = native.fit_hill(native.FIT_REDOX, x, f, T, v)
    assert got[0] == pytest.approx(want[0], abs=1e-10)
    assert got[1] == pytest.approx(want[1], rel=1e-7)
    assert got[2] == pytest.approx(want[2], rel=1e-9, abs=1e-20)


def test_native_fit_with_saturated_points_matches_oracle(native):
    """Fractions of exactly 0 or 1 (conditions where a site never changed
    state) are left out of the Hill-plot start but kept in the fit."""
    x = np.linspace(0.0, 12.0, 25)
    f = oracle.f_prot(x, 4.4, 1.0)
    f[:2], f[-3:] = 1.0, 0.0
    want = oracle.fit_hill("pH", x, f)
    got = native.fit_hill(native.FIT_PH, x, f)
    assert got[0] == pytest.approx(want[0], abs=1e-9)
    assert got[1] == pytest.approx(want[1], rel=1e-8)


@pytest.mark.parametrize("x,f,kind,T,v", [
    ([1.0, 2.0], [1.0, 0.0], 1, 300.0, 1.0),          # no interior fraction
    ([3.0, 3.0, 3.0], [0.2, 0.5, 0.7], 1, 300.0, 1.0),  # one distinct x
    ([1.0, 2.0], [0.5, 1.2], 1, 300.0, 1.0),          # f outside [0, 1]
    ([1.0, 2.0], [0.4, 0.6], 2, 0.0, 1.0),            # T <= 0
    ([1.0, 2.0], [0.4, 0.6], 2, 300.0, 0.0),          # v <= 0
    ([1.0], [0.5], 1, 300.0, 1.0),                    # one point
    ([1.0, 2.0], [0.4, 0.6], 3, 300.0, 1.0),          # unknown kind
])
def test_native_fit_rejects_degenerate_input(native, x, f, kind, T, v):
    with pytest.raises(cphremd.CphError):
        native.fit_hill(kind, x, f, T, v)


# ---------------------------------------------------------------- oracle counters

@pytest.fixture(scope="module")
def c2_run():
    systems, grid = synth.config_c2()
    W = oracle.Walkers(systems, grid, seed=12, mc_ph=3, mc_redox=3, exchange_every=2)
    oracle.run_schedule(W, 30)
    return W


def test_oracle_counters_are_consistent(c2_run):
    """One sample per step: every site row and every visit row and column of
    the walker-by-slot table sums to the step count, and the table is a sum
    of permutation matrices whose last one is the current condition map."""
    W = c2_run
    assert W.n_obs == 30
    for s, occ in enumerate(W.occ):
        assert (occ.sum(1) == 30).all()
        nst = [len(st.n_prot) for st in W.systems[W.sys_of[s]].sites]
        for k, n in enumerate(nst):
            assert (occ[k, n:] == 0).all()
    assert (W.visits.sum(0) == 30).all() and (W.visits.sum(1) == 30).all()
    assert all(W.visits[w, W.slot_of[w]] >= 1 for w in range(len(W.slot_of)))
    assert np.count_nonzero(W.visits - np.diag(np.diag(W.visits))) > 0, "no exchange happened"
    fr = oracle.site_fractions(W)
    for s, occ in enumerate(W.occ):
        for k, st in enumerate(W.systems[W.sys_of[s]].sites):
            n = np.asarray(st.n_prot if st.kind == "ph" else st.n_elec, float)
            want = (occ[k, :len(n)] * (n - n.min())).sum() / (n.max() - n.min()) / 30
            assert fr[s][k] == pytest.approx(want, rel=1e-15)


def test_oracle_counters_without_exchange_or_mc():
    systems, grid = synth.config_c2()
    W = oracle.Walkers(systems, grid, seed=12, mc_ph=0, mc_redox=0, exchange_every=0)
    oracle.run_schedule(W, 7)
    assert (W.visits == 7 * np.eye(len(W.slot_of), dtype=np.int64)).all()
    for s, occ in enumerate(W.occ):
        for k, st in enumerate(W.systems[W.sys_of[s]].sites):
            assert occ[k, st.init_state] == 7 and occ[k].sum() == 7


def _ion_fit(kind, ref, steps, seed):
    ion = synth.titratable_ion(kind, ref)
    if kind == "ph":
        xs = np.linspace(ref - 1.5, ref + 1.5, 7)
        grid = synth.Grid(np.array([0.0]), xs, np.array([300.0]), np.zeros(7, np.int32),
                          order=("pH",))
        W = oracle.Walkers([ion], grid, seed=seed, mc_ph=1, mc_redox=0, exchange_every=4)
    else:
        xs = np.linspace(ref - 0.09, ref + 0.09, 7)
        grid = synth.Grid(xs, np.array([7.0]), np.array([300.0]), np.zeros(7, np.int32),
                          order=("E",))
        W = oracle.Walkers([ion], grid, seed=seed, mc_ph=0, mc_redox=1, exchange_every=4)
    oracle.run_schedule(W, steps)
    f = np.array([fr[0] for fr in oracle.site_fractions(W)])
    return W, xs, f


@pytest.mark.parametrize("kind,ref", [("ph", 4.85), ("redox", -0.203)])
def test_oracle_ion_titration_follows_eqs_1_and_2(kind, ref):
    """A titratable ion's G(s) reduces to the pH or E term, so the sampled
    fractions at every condition follow eq (1) / eq (2) with n = 1, and the
    fit returns the site's reference pKa / E0 (5000 samples per condition)."""
    W, xs, f = _ion_fit(kind, ref, 5000, seed=31)
    want = oracle.f_prot(xs, ref) if kind == "ph" else oracle.f_red(xs, ref, 300.0)
    assert np.abs(f - want).max() < 0.04
    x0, n, _ = oracle.fit_hill("pH" if kind == "ph" else "redox", xs, f, 300.0, 1.0)
    if kind == "ph":
        assert abs(x0 - ref) < 0.06 and abs(n - 1.0) < 0.08
    else:
        assert abs(x0 - ref) < 0.0035 and abs(n - 1.0) < 0.08
    assert (W.visits.sum(0) == 5000).all() and (W.visits > 0).all()
