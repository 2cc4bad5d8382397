"""The library's eq (6)-(8) predictions (host calls, no GPU needed) against
the oracle's closed forms, and end to end against the brute-force partition
function of a coupled redox + pH system: E0 where the reduced fraction is
one half follows eq (7), the pKa where the protonated fraction is one half
follows eq (8), and their ends reduce to eq (6) (the paper's "Temperature
dependence in predicting E0 vs pH and pKa vs redox potential" section draws
Figure 6's solid lines from eqs (7) and (8))."""
import itertools
import math

import numpy as np
import pytest

import oracle
from oracle import FARADAY, KB, LN10, GBParams
from paper_1809_07726_gb300 import build, cphremd, synth


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()


CASES = [  # (pka_red, pka_oxi, E0_prot, E0_deprot offset, T, v)
    ([4.55], [4.40], -0.203, None, 300.0, 1.0),
    ([4.6, 5.1, 4.9], [4.45, 4.93, 4.78], -0.19, None, 280.0, 1.0),
    ([7.0, 3.2], [6.1, 3.0], 0.05, None, 380.0, 2.0),
]


@pytest.mark.parametrize("pka_red,pka_oxi,e0p,_,T,v", CASES)
def test_predictions_match_the_oracle_closed_forms(pka_red, pka_oxi, e0p, _, T, v):
    d = cphremd.predict_delta_e0(pka_red, pka_oxi, T, v)
    assert d == pytest.approx(oracle.eq6_delta_e0(pka_red, pka_oxi, T, v), rel=1e-13)
    e0d = e0p - d
    pH = np.linspace(0.0, 12.0, 25)
    got = cphremd.predict_e0(pH, e0p, pka_red, pka_oxi, T, v)
    want = np.array([oracle.eq7_e0(p, e0p, pka_red, pka_oxi, T, v) for p in pH])
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-14)
    E = np.linspace(-0.5, 0.3, 17)
    got = cphremd.predict_sum_pka(E, e0p, e0d, pka_red, T, v)
    want = np.array([oracle.eq8_sum_pka(e, e0p, e0d, pka_red, T, v) for e in E])
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)


def test_predictions_reach_the_limits_of_eq6():
    """Eq (7): E0 -> E0_prot at low pH and E0_prot - (eq 6) at high pH; eq (8):
    sum pKa -> sum pKa_red at very negative E and sum pKa_oxi at very positive E."""
    pr, po, T = [4.6, 5.1], [4.3, 4.9], 300.0
    e0p = -0.2
    d = cphremd.predict_delta_e0(pr, po, T)
    lo, hi = cphremd.predict_e0([-30.0, 40.0], e0p, pr, po, T)
    assert lo == pytest.approx(e0p, abs=1e-12)
    assert hi == pytest.approx(e0p - d, abs=1e-12)
    s_lo, s_hi = cphremd.predict_sum_pka([-40.0, 40.0], e0p, e0p - d, pr, T)
    assert s_lo == pytest.approx(sum(pr), abs=1e-10)
    assert s_hi == pytest.approx(sum(po), abs=1e-10)


def test_predictions_refuse_bad_arguments():
    with pytest.raises(cphremd.CphError):
        cphremd.predict_delta_e0([4.0], [4.0], 0.0)
    with pytest.raises(cphremd.CphError):
        cphremd.predict_e0([7.0], -0.2, [4.0], [3.9], 300.0, v=-1.0)
    with pytest.raises(cphremd.CphError):
        cphremd.predict_sum_pka([float("nan")], -0.2, -0.22, [4.0], 300.0)


@pytest.fixture(scope="module")
def coupled():
    """1 pH site + 1 redox site on a 30-atom chain, frozen geometry: the
    electrostatic free energy W(s_pH, s_redox) of all four states."""
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


def _bisect(f, lo, hi):
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if f(lo) * f(mid) <= 0:
            hi = mid
        else:
            lo = mid
    return 0.5 * (lo + hi)


def test_predictions_follow_the_brute_force_partition_function(coupled):
    s, Wel = coupled
    T = 310.0
    kT = KB * T
    pka_ref, e0_ref = s.sites[0].ref, s.sites[1].ref
    pka_red = pka_ref - (Wel[(1, 1)] - Wel[(0, 1)]) / (kT * LN10)
    pka_oxi = pka_ref - (Wel[(1, 0)] - Wel[(0, 0)]) / (kT * LN10)
    e0_prot = e0_ref - (Wel[(1, 1)] - Wel[(1, 0)]) / FARADAY
    e0_deprot = e0_ref - (Wel[(0, 1)] - Wel[(0, 0)]) / FARADAY
    assert cphremd.predict_delta_e0([pka_red], [pka_oxi], T) == pytest.approx(e0_prot - e0_deprot,
                                                                               rel=1e-9)
    pHs = np.array([2.0, 4.5, 5.0, 6.0, 9.5])
    pred = cphremd.predict_e0(pHs, e0_prot, [pka_red], [pka_oxi], T)
    for pH, e in zip(pHs, pred):
        e0 = _bisect(lambda E: (lambda p: p[(0, 1)] + p[(1, 1)] - 0.5)(_pi(s, Wel, E, pH, T)),
                     -2.0, 2.0)
        assert e == pytest.approx(e0, abs=1e-9)
    Es = np.array([-0.45, -0.2, 0.0, 0.15])
    pred = cphremd.predict_sum_pka(Es, e0_prot, e0_deprot, [pka_red], T)
    for E, pk in zip(Es, pred):
        pka = _bisect(lambda pH: (lambda p: p[(1, 0)] + p[(1, 1)] - 0.5)(_pi(s, Wel, E, pH, T)),
                      -20.0, 30.0)
        assert pk == pytest.approx(pka, abs=1e-8)
