"""Pins of the oracle's random numbers, integrator, Monte Carlo and exchanges:
Philox known answers, Henderson-Hasselbalch and Nernst titration of an isolated
site, a brute-force partition function for coupled sites together with the
paper's eqs (6)-(8), exact detailed balance of one exchange attempt along each
dimension, and equipartition of the Langevin integrator."""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from oracle import FARADAY, KB, LN10, GBParams
from paper_1809_07726_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(t, 16) for t in r]
        out = oracle.philox(v[0:4], v[4:6])
        assert out.tolist() == v[6:10]


def test_uniforms_and_normals_statistics():
    u = np.array([oracle.uniforms(12345, i, 3, 7, 1) for i in range(25000)]).ravel()
    assert u.min() > 0.0 and u.max() < 1.0
    counts, _ = np.histogram(u, bins=50, range=(0, 1))
    exp = len(u) / 50
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert chi2 < 100  # 49 dof: p ~ 3e-5
    z = np.array([oracle.normals3(99, i, 0, 5) for i in range(30000)]).ravel()
    n = len(z)
    assert abs(z.mean()) < 4 / math.sqrt(n)
    assert abs(z.var() - 1) < 4 * math.sqrt(2 / n)
    assert abs((z ** 4).mean() - 3) < 4 * math.sqrt(96 / n)


def test_counter_streams_are_distinct():
    a = oracle.uniforms(1, 0, 0, 0, 1)
    for args in [(1, 1, 0, 0, 1), (1, 0, 1, 0, 1), (1, 0, 0, 1, 1), (1, 0, 0, 0, 2),
                 (2, 0, 0, 0, 1), (1, 0, 0, 1 << 32, 1)]:
        assert not np.array_equal(a, oracle.uniforms(*args))


def test_paper_printed_differences_match_eq6_constants():
    """Eq (6) with v = 1 turns the printed pKa differences into E0_prot - E0_deprot;
    two-decimal rounding of the printed pKa values allows +-3 mV."""
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "paper_temperature_differences.txt"))
            if ln.strip() and not ln.startswith("#")]
    for T, de0, glu, prn in (map(float, r) for r in rows):
        pred = oracle.eq6_delta_e0([glu, prn, prn], [0, 0, 0], T) * 1000.0
        assert abs(pred - de0) < 3.0


# ------------------------------------------------------------------ Langevin

def _ho_run(gamma, T, steps, n=1500, k=10.0, m=12.0, seed=4):
    x = np.ascontiguousarray(np.random.default_rng(seed).normal(0, 0.1, size=(n, 3)))
    v = np.zeros_like(x)
    mass = np.full(n, m)
    xs, ke, etot = [], [], []
    for t in range(steps):
        F = -k * x
        v_old = v.copy()
        oracle.langevin(x, v, F, mass, 0.002, gamma, T, seed, 0, t)
        xs.append((x ** 2).mean())
        ke.append((0.5 * m * v ** 2 / 418.4).mean())
        vbar2 = 0.5 * (v_old ** 2 + v ** 2)
        etot.append((0.5 * k * (x - 0.002 * v) ** 2).sum() + (0.5 * m * vbar2 / 418.4).sum())
    return np.array(xs), np.array(ke), np.array(etot)


def test_langevin_equipartition_harmonic():
    """<x^2> = kT/k and <1/2 m v^2> = 1/2 kT per component (4 sigma, plus the
    O((omega dt)^2) leapfrog bias)."""
    T, k = 300.0, 10.0
    xs, ke, _ = _ho_run(10.0, T, 2500, k=k)
    xs, ke = xs[500:], ke[500:]
    kT = KB * T
    assert xs.mean() == pytest.approx(kT / k, rel=0.02)
    assert ke.mean() == pytest.approx(0.5 * kT, rel=0.02)


def test_langevin_without_friction_is_symplectic_leapfrog():
    """gamma = 0 and T = 0: plain leapfrog; the harmonic energy stays bounded
    (no drift) to O((omega dt)^2)."""
    _, _, e = _ho_run(0.0, 0.0, 3000, n=50)
    assert np.abs(e / e[0] - 1).max() < 2e-3
    assert abs(e[-500:].mean() / e[:500].mean() - 1) < 5e-4


# ---------------------------------------------------------------- Monte Carlo

def _lone_site_system(n_states, kind, ref, seed=0):
    """A system made of one site's atoms only, so U_el(s) - U_ref(s) = 0."""
    s = synth.make_system(6, seed, n_ph=0, n_redox=0)
    rng = np.random.default_rng(seed)
    atoms = np.arange(6, dtype=np.int32)
    base = s.q.copy()
    tot = 1.0 if kind == "ph" else -1.0
    rows = [base] + [base + tot * rng.dirichlet(np.ones(6)) for _ in range(n_states - 1)]
    if kind == "ph":
        site = synth.Site("ph", atoms, np.stack(rows), np.array([0] + [1] * (n_states - 1)),
                          np.zeros(n_states, int), ref)
    else:
        site = synth.Site("redox", atoms, np.stack(rows), np.zeros(2, int), np.array([0, 1]), ref)
    s.sites = [site]
    return s


def _batch_mean_sd(a, nb=40):
    a = np.asarray(a, float)
    b = a[: len(a) // nb * nb].reshape(nb, -1).mean(1)
    return a.mean(), b.std(ddof=1) / math.sqrt(nb)


@pytest.mark.parametrize("n_states,pH", [(2, 4.0), (2, 5.2), (3, 5.0)])
def test_mc_isolated_site_follows_henderson_hasselbalch(n_states, pH):
    """Eq (1) with n_prot = 1; n-1 protonated tautomers shift the macroscopic
    pKa to pKa_ref + log10(n-1)."""
    pka = 4.6
    s = _lone_site_system(n_states, "ph", pka)
    grid = synth.Grid(np.array([0.0]), np.array([pH]), np.array([300.0]), np.zeros(1, np.int32))
    W = oracle.Walkers([s], grid, seed=21)
    prot = []
    for t in range(1, 6001):
        oracle.mc_sweep(W, 0, "ph", t)
        prot.append(W.n_prot(0))
    m, sd = _batch_mean_sd(prot[200:])
    target = oracle.f_prot(pH, pka + math.log10(n_states - 1))
    assert abs(m - target) < 4 * sd + 1e-3
    # and the exponent equals the closed form exactly
    for (w, k, a, b, dU, xexp, lnu, acc) in W.mc_log[:50]:
        dn = s.sites[0].n_prot[b] - s.sites[0].n_prot[a]
        assert xexp == pytest.approx(-LN10 * dn * (pH - pka), abs=1e-9)
        assert acc == (lnu < xexp)


@pytest.mark.parametrize("E", [-0.23, -0.17])
def test_mc_isolated_site_follows_nernst(E):
    e0, T = -0.2, 300.0
    s = _lone_site_system(2, "redox", e0, seed=3)
    grid = synth.Grid(np.array([E]), np.array([7.0]), np.array([T]), np.zeros(1, np.int32))
    W = oracle.Walkers([s], grid, seed=5)
    red = []
    for t in range(1, 6001):
        oracle.mc_sweep(W, 0, "redox", t)
        red.append(W.n_elec(0))
    m, sd = _batch_mean_sd(red[200:])
    assert abs(m - oracle.f_red(E, e0, T)) < 4 * sd + 1e-3


@pytest.fixture(scope="module")
def coupled():
    """1 pH site + 1 redox site on a 30-atom chain, frozen geometry."""
    s = synth.make_system(30, 8, n_ph=1, ph_atoms=(6, 6), ph_pka=[5.0], redox_atoms=8)
    o = oracle.OSystem(s)
    gb = GBParams()
    uref = oracle.reference_energies(o, s, gb)
    _, R = oracle.born(s.x, s.rho, s.screen, gb)
    W = {}
    for sp, sr in itertools.product(range(2), range(2)):
        q = s.q.copy()
        q[s.sites[0].atoms] = s.sites[0].q[sp]
        q[s.sites[1].atoms] = s.sites[1].q[sr]
        W[(sp, sr)] = oracle.u_el(o, s.x, q, R, gb) - uref[0][sp] - uref[1][sr]
    return s, W


def _pi(s, W, E, pH, T):
    kT = KB * T
    G = {st: W[st] + kT * LN10 * st[0] * (pH - s.sites[0].ref)
         + FARADAY * st[1] * (E - s.sites[1].ref) for st in W}
    z = {st: math.exp(-(g - min(G.values())) / kT) for st, g in G.items()}
    Z = sum(z.values())
    return {st: v / Z for st, v in z.items()}


def test_mc_coupled_sites_sample_the_brute_force_distribution(coupled):
    s, Wel = coupled
    E, pH, T = -0.21, 5.3, 300.0
    pi = _pi(s, Wel, E, pH, T)
    grid = synth.Grid(np.array([E]), np.array([pH]), np.array([T]), np.zeros(1, np.int32))
    W = oracle.Walkers([s], grid, seed=77)
    _, R = oracle.born(s.x, s.rho, s.screen, GBParams())
    fp, fr = [], []
    for t in range(1, 8001):
        oracle.mc_sweep(W, 0, "ph", t, R)
        oracle.mc_sweep(W, 0, "redox", t, R)
        fp.append(W.n_prot(0))
        fr.append(W.n_elec(0))
    for series, target in [(fp, pi[(1, 0)] + pi[(1, 1)]), (fr, pi[(0, 1)] + pi[(1, 1)])]:
        m, sd = _batch_mean_sd(series[200:])
        assert abs(m - target) < 4 * sd + 1e-3


def test_coupled_sites_obey_eqs_6_to_8(coupled):
    """From the brute-force partition function: E0(pH) (f_red = 1/2) follows
    eq (7), the pKa(E) follows eq (8), and both reduce to eq (6)."""
    s, Wel = coupled
    T = 300.0
    kT = KB * T
    pka_ref, e0_ref = s.sites[0].ref, s.sites[1].ref
    # pKa of the pH site with the redox site held reduced / oxidised
    pka_red = pka_ref - (Wel[(1, 1)] - Wel[(0, 1)]) / (kT * LN10)
    pka_oxi = pka_ref - (Wel[(1, 0)] - Wel[(0, 0)]) / (kT * LN10)
    # E0 with the pH site held protonated / deprotonated
    e0_prot = e0_ref - (Wel[(1, 1)] - Wel[(1, 0)]) / FARADAY
    e0_deprot = e0_ref - (Wel[(0, 1)] - Wel[(0, 0)]) / FARADAY
    assert FARADAY * (e0_prot - e0_deprot) == pytest.approx(
        kT * LN10 * (pka_red - pka_oxi), rel=1e-10)

    def solve(f, lo, hi):
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if f(lo) * f(mid) <= 0:
                hi = mid
            else:
                lo = mid
        return 0.5 * (lo + hi)

    for pH in (3.0, 5.0, 6.5, 9.0):
        e0 = solve(lambda E: (lambda p: p[(0, 1)] + p[(1, 1)] - 0.5)(_pi(s, Wel, E, pH, T)),
                   -2.0, 2.0)
        assert e0 == pytest.approx(oracle.eq7_e0(pH, e0_prot, [pka_red], [pka_oxi], T),
                                   abs=1e-9)
    for E in (-0.4, -0.2, 0.1):
        pka = solve(lambda pH: (lambda p: p[(1, 0)] + p[(1, 1)] - 0.5)(_pi(s, Wel, E, pH, T)),
                    -20.0, 30.0)
        assert pka == pytest.approx(oracle.eq8_sum_pka(E, e0_prot, e0_deprot, [pka_red], T),
                                    abs=1e-8)


# ------------------------------------------------------------------ exchange

def _perm_matrix(dim, conds, walkers, parity):
    """Exact transition matrix of one attempt on one line of slots."""
    nslot = len(conds)
    perms = list(itertools.permutations(range(nslot)))  # perm[slot] = walker
    idx = {p: i for i, p in enumerate(perms)}
    P = np.zeros((len(perms), len(perms)))
    pairs = [(m, m + 1) for m in range(parity, nslot - 1, 2)]
    for p in perms:
        for choice in itertools.product([0, 1], repeat=len(pairs)):
            prob = 1.0
            q = list(p)
            for (a, b), c in zip(pairs, choice):
                wi, wj = p[a], p[b]
                x = oracle.exchange_exponent(dim, conds[a], conds[b], *[walkers[wi][0],
                                             walkers[wj][0], walkers[wi][1], walkers[wj][1],
                                             walkers[wi][2], walkers[wj][2]])
                acc = min(1.0, math.exp(x))
                prob *= acc if c else 1 - acc
                if c:
                    q[a], q[b] = q[b], q[a]
            P[idx[p], idx[tuple(q)]] += prob
    return perms, P


@pytest.mark.parametrize("dim", ["E", "pH", "T"])
def test_exchange_attempt_is_in_detailed_balance(dim):
    """pi P = pi for pi(perm) = prod_w exp(-beta_slot U_w) 10^(-pH_slot N_H,w)
    exp(-F E_slot N_e,w / kT_slot), restricted to the exchanged dimension."""
    rng = np.random.default_rng({"E": 1, "pH": 2, "T": 3}[dim])
    n = 4
    if dim == "E":
        conds = [(e, 7.0, 300.0) for e in np.linspace(-0.3, -0.15, n)]
    elif dim == "pH":
        conds = [(-0.2, p, 300.0) for p in np.linspace(4.0, 5.5, n)]
    else:
        conds = [(-0.2, 7.0, t) for t in 300.0 * 1.05 ** np.arange(n)]
    walkers = [(float(rng.normal(-500, 2.0)), int(rng.integers(0, 4)), int(rng.integers(0, 2)))
               for _ in range(n)]

    def weight(perm):
        lw = 0.0
        for slot, w in enumerate(perm):
            U, NH, Ne = walkers[w]
            E, pH, T = conds[slot]
            if dim == "T":
                lw += -U / (KB * T)
            elif dim == "pH":
                lw += -LN10 * pH * NH
            else:
                lw += -FARADAY * E * Ne / (KB * T)
        return lw

    for parity in (0, 1):
        perms, P = _perm_matrix(dim, conds, walkers, parity)
        lw = np.array([weight(p) for p in perms])
        pi = np.exp(lw - lw.max())
        pi /= pi.sum()
        np.testing.assert_allclose(pi @ P, pi, rtol=1e-10, atol=1e-14)
        np.testing.assert_allclose(P.sum(1), 1.0, rtol=1e-12)


def test_exchange_acceptance_rate_matches_min_one_exp():
    """Empirical swap rate of the Philox-driven attempt against min{1, e^x}."""
    s = synth.make_system(6, 0, n_ph=0, n_redox=0)
    grid = synth.Grid(np.array([-0.2]), np.array([7.0]), np.array([300.0, 310.0]),
                      np.zeros(2, np.int32), order=("T",))
    W = oracle.Walkers([s], grid, seed=9)
    acc = 0
    n = 4000
    for t in range(n):
        W.walker_at[:] = [0, 1]
        W.slot_of[:] = [0, 1]
        W.U[:] = [-100.0, -99.0]
        W.n_attempts["T"] = 0
        oracle.exchange_attempt(W, "T", t)
        acc += int(W.walker_at[0] == 1)
    x = (1 / (KB * 300.0) - 1 / (KB * 310.0)) * (-100.0 + 99.0)
    p = min(1.0, math.exp(x))
    assert abs(acc / n - p) < 4 * math.sqrt(p * (1 - p) / n)


def _t_line_matrix(conds, eps, parity):
    """Exact transition matrix of one T attempt on one line, walker w carrying
    the exchange energy eps[w]."""
    nslot = len(conds)
    perms = list(itertools.permutations(range(nslot)))
    idx = {p: i for i, p in enumerate(perms)}
    P = np.zeros((len(perms), len(perms)))
    pairs = [(m, m + 1) for m in range(parity, nslot - 1, 2)]
    for p in perms:
        for choice in itertools.product([0, 1], repeat=len(pairs)):
            prob = 1.0
            q = list(p)
            for (a, b), c in zip(pairs, choice):
                x = oracle.exchange_exponent("T", conds[a], conds[b], eps[p[a]], eps[p[b]], 0, 0, 0, 0)
                acc = min(1.0, math.exp(x))
                prob *= acc if c else 1 - acc
                if c:
                    q[a], q[b] = q[b], q[a]
            P[idx[p], idx[tuple(q)]] += prob
    return perms, P


@pytest.mark.parametrize("choice", ["potential", "semigrand"])
def test_t_exchange_energy_choices_detailed_balance(choice):
    """Walkers in different redox states and with different site reference
    energies along a T line at E != E0_ref.  The C(pH,E)MD weight of walker w
    at temperature T is exp(-(U - U_ref + F N_e (E - E0_ref)) / kT) (the pH
    factor is the same at every slot of a T line).  With the semi-grand
    exchange energy one attempt is in detailed balance with that weight; with
    the potential energy it is in detailed balance with exp(-U / kT) only, and
    not with the C(pH,E)MD weight."""
    rng = np.random.default_rng(11)
    E, e0_ref, n = -0.15, -0.2, 4
    conds = [(E, 7.0, t) for t in 300.0 * 1.06 ** np.arange(n)]
    U = rng.normal(-500.0, 1.5, n)
    uref = rng.normal(-40.0, 1.0, n)
    Ne = np.array([0, 1, 1, 0])
    full = U - uref + FARADAY * Ne * (E - e0_ref)
    eps = full if choice == "semigrand" else U

    def lw(perm, energy):
        return sum(-energy[w] / (KB * conds[slot][2]) for slot, w in enumerate(perm))

    for parity in (0, 1):
        perms, P = _t_line_matrix(conds, eps, parity)
        for energy, should_hold in ((full, choice == "semigrand"), (U, choice == "potential")):
            w = np.array([lw(p, energy) for p in perms])
            pi = np.exp(w - w.max())
            pi /= pi.sum()
            dev = np.abs(pi @ P - pi).max() / pi.max()
            assert (dev < 1e-10) == should_hold, (choice, parity, dev)


def test_semigrand_exchange_energy_of_a_walker():
    """exchange_energy: the potential energy, less the sites' reference
    energies, plus F N_e (E - E0_ref) per redox site."""
    s = synth.make_system(40, 12, n_ph=2, ph_atoms=(6, 6), redox_atoms=8)
    grid = synth.Grid(np.array([-0.1]), np.array([6.0]), np.array([300.0]), np.zeros(1, np.int32))
    W = oracle.Walkers([s], grid, seed=1, t_energy="semigrand")
    W.state[0][:] = [1, 0, 1]
    W.U[0] = -321.5
    ur = W.uref[0]
    red = [k for k, st in enumerate(s.sites) if st.kind == "redox"][0]
    want = -321.5 - sum(ur[k][W.state[0][k]] for k in range(len(s.sites))) \
        + FARADAY * s.sites[red].n_elec[W.state[0][red]] * (-0.1 - s.sites[red].ref)
    assert oracle.exchange_energy(W, 0) == pytest.approx(want, rel=1e-14)
    W.t_energy = "potential"
    assert oracle.exchange_energy(W, 0) == -321.5
