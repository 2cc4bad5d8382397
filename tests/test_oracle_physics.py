"""Pins of the FP64 oracle's pair physics against facts outside the oracle:
geometric quadrature of the HCT integral, the Born equation, Coulomb and LJ
closed forms, finite differences of the energy, conservation laws and
rigid-motion invariance."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from oracle import GBParams, KCOUL
from paper_1809_07726_gb300 import synth


def shell_integral(r, rt, s, rc=None):
    """H(r, rt, s) from geometry alone: for each shell of radius t >= rt about
    atom i, the fraction of the shell inside sphere j (radius s, centre at
    distance r) is (1 - c0)/2 with c0 = clip((t^2 + r^2 - s^2)/(2 t r), -1, 1);
    H = 2 * (1/4pi) * int 4 pi t^2 frac / t^4 dt, over shells t <= rc when a
    cutoff rc is given."""
    def f(t):
        c0 = (t * t + r * r - s * s) / (2.0 * t * r)
        c0 = min(1.0, max(-1.0, c0))
        return (1.0 - c0) / (t * t)
    hi = r + s if rc is None else min(r + s, rc)
    if rt >= hi:
        return 0.0
    pts = [p for p in (abs(r - s), s - r) if rt < p < hi]
    val, err = integrate.quad(f, rt, hi, points=pts or None, epsabs=1e-14, epsrel=1e-12,
                              limit=200)
    return val


CASES = [
    # (r, rt, s, branch)
    (6.0, 1.4, 1.2, "disjoint"),
    (20.0, 1.9, 1.7, "far"),
    (2.0, 1.5, 1.3, "partial overlap, L = rt"),
    (1.0, 0.5, 2.0, "i inside j"),
    (0.3, 2.5, 1.0, "j swallowed by i"),
    (2.2, 1.0, 1.4, "disjoint, close"),
    (1.6, 1.2, 1.0, "partial overlap, r > s"),
    (0.8, 1.1, 1.5, "partial overlap, s > r"),
]


@pytest.mark.parametrize("r,rt,s,branch", CASES)
def test_hct_matches_shell_quadrature(r, rt, s, branch):
    h = oracle.hct(r, rt, s)
    ref = shell_integral(r, rt, s)
    assert h == pytest.approx(ref, rel=1e-10, abs=1e-13), branch


def test_hct_matches_3d_monte_carlo():
    """Brute-force 3D sampling of sphere j: (1/4pi) int |x|^-4 over sphere j
    outside the ball rt equals H/2."""
    rng = np.random.default_rng(0)
    for r, rt, s in [(2.0, 1.5, 1.3), (4.0, 1.2, 1.5)]:
        n = 2_000_000
        p = rng.normal(size=(n, 3))
        p *= (s * rng.uniform(size=n) ** (1 / 3) / np.linalg.norm(p, axis=1))[:, None]
        p[:, 0] += r
        d = np.linalg.norm(p, axis=1)
        w = np.where(d > rt, d ** -4, 0.0)
        vol = 4.0 / 3.0 * math.pi * s ** 3
        est = vol * w.mean() / (4 * math.pi)
        sd = vol * w.std() / (4 * math.pi) / math.sqrt(n)
        assert abs(2 * est - oracle.hct(r, rt, s)) < 5 * 2 * sd


@pytest.mark.parametrize("r,rt,s,branch", CASES[:4] + CASES[5:])
def test_hct_derivatives_match_finite_differences(r, rt, s, branch):
    h = 1e-6
    fd_r = (oracle.hct(r + h, rt, s) - oracle.hct(r - h, rt, s)) / (2 * h)
    fd_t = (oracle.hct(r, rt + h, s) - oracle.hct(r, rt - h, s)) / (2 * h)
    fd_s = (oracle.hct(r, rt, s + h) - oracle.hct(r, rt, s - h)) / (2 * h)
    assert oracle.hct_dr(r, rt, s) == pytest.approx(fd_r, rel=1e-6, abs=1e-9)
    assert oracle.hct_drt(r, rt, s) == pytest.approx(fd_t, rel=1e-6, abs=1e-9)
    assert oracle.hct_ds(r, rt, s) == pytest.approx(fd_s, rel=1e-6, abs=1e-9)


def test_hct_far_field_is_volume_over_r4():
    """Far from i, sphere j is a point volume: H -> 2/3 s^3 / r^4."""
    s, r = 1.3, 400.0
    assert oracle.hct(r, 1.5, s) == pytest.approx(2.0 / 3.0 * s ** 3 / r ** 4, rel=1e-4)


def _one_system(n, x, q, rho, screen=None, sigma=None, eps=None, bonds=None):
    s = synth.System(x=np.asarray(x, float), mass=np.full(n, 12.0), q=np.asarray(q, float),
                     rho=np.asarray(rho, float),
                     screen=np.full(n, 0.8) if screen is None else np.asarray(screen, float),
                     sigma=np.full(n, 2.0) if sigma is None else np.asarray(sigma, float),
                     eps=np.zeros(n) if eps is None else np.asarray(eps, float),
                     bonds=np.zeros((0, 2), np.int32) if bonds is None else bonds,
                     bond_k=np.zeros(0 if bonds is None else len(bonds)),
                     bond_r0=np.zeros(0 if bonds is None else len(bonds)),
                     angles=np.zeros((0, 3), np.int32), angle_k=np.zeros(0),
                     angle_t0=np.zeros(0))
    return s, oracle.OSystem(s)


def test_born_isolated_ion():
    """A lone ion has psi = 0, R = rho - offset, and the Born energy
    -1/2 k (1/eps_in - 1/eps_out) q^2 / R."""
    gb = GBParams()
    for q, rho in [(1.0, 1.5), (-0.7, 2.0)]:
        s, o = _one_system(1, [[0.3, -0.2, 0.1]], [q], [rho])
        terms, F, R, psi = oracle.energy(o, s.x, s.q, gb)
        Rb = rho - gb.offset
        assert psi[0] == 0.0 and R[0] == pytest.approx(Rb, rel=1e-15)
        born = -0.5 * KCOUL * (1 / gb.eps_in - 1 / gb.eps_out) * q * q / Rb
        assert terms[0] == pytest.approx(born, rel=1e-14)
        assert np.all(F == 0.0)
    # textbook Born with zero offset
    gb0 = GBParams(offset=0.0)
    s, o = _one_system(1, [[0, 0, 0]], [1.0], [2.0])
    t0 = oracle.energy(o, s.x, s.q, gb0)[0]
    assert t0[0] == pytest.approx(-0.5 * KCOUL * (1 - 1 / 78.5) / 2.0, rel=1e-14)


def test_pair_far_limit_is_screened_coulomb():
    """Two ions far apart: Coulomb + GB cross term -> k q1 q2 / (eps_out r)."""
    gb = GBParams()
    q1, q2 = 0.8, -0.6
    for r in (200.0, 2000.0):
        s, o = _one_system(2, [[0, 0, 0], [r, 0, 0]], [q1, q2], [1.5, 1.7])
        terms, _, R, _ = oracle.energy(o, s.x, s.q, gb)
        tau = 1 / gb.eps_in - 1 / gb.eps_out
        self_e = -0.5 * KCOUL * tau * (q1 * q1 / R[0] + q2 * q2 / R[1])
        pair = terms[0] + terms[1] - self_e
        target = KCOUL * q1 * q2 / (gb.eps_out * r)
        assert pair == pytest.approx(target, rel=5 * (R[0] * R[1]) / r ** 2)


def test_pair_zero_distance_merges_into_one_born_ion():
    """With R_i = R_j = R and r -> 0, f -> R: the GB energy of two excluded
    charges is that of one ion of charge q1 + q2."""
    gb = GBParams()
    q1, q2, R = 0.4, 0.3, 1.6
    s, o = _one_system(2, [[0, 0, 0], [1e-7, 0, 0]], [q1, q2], [1.5, 1.5])
    o.excl[0, 1] = o.excl[1, 0] = 1
    e = oracle.u_el(o, s.x, s.q, np.array([R, R]), gb)
    tau = 1 / gb.eps_in - 1 / gb.eps_out
    assert e == pytest.approx(-0.5 * KCOUL * tau * (q1 + q2) ** 2 / R, rel=1e-12)


def test_coulomb_and_lj_closed_forms():
    gb = GBParams(eps_out=1.0)  # tau = 0: no GB
    r = 3.7
    s, o = _one_system(2, [[0, 0, 0], [0, r, 0]], [0.5, -0.25], [1.5, 1.5],
                       sigma=[3.0, 3.4], eps=[0.1, 0.4])
    terms = oracle.energy(o, s.x, s.q, gb)[0]
    assert terms[0] == 0.0
    assert terms[1] == pytest.approx(KCOUL * 0.5 * -0.25 / r, rel=1e-14)
    sig, ep = 3.2, math.sqrt(0.04)
    assert terms[2] == pytest.approx(4 * ep * ((sig / r) ** 12 - (sig / r) ** 6), rel=1e-13)
    # LJ minimum: depth -eps at 2^(1/6) sigma, zero force there
    rm = 2 ** (1 / 6) * sig
    s2, o2 = _one_system(2, [[0, 0, 0], [rm, 0, 0]], [0, 0], [1.5, 1.5],
                         sigma=[3.0, 3.4], eps=[0.1, 0.4])
    t2, F2, _, _ = oracle.energy(o2, s2.x, s2.q, gb)
    assert t2[2] == pytest.approx(-ep, rel=1e-13)
    assert np.abs(F2).max() < 1e-12
    # excluded pair: no Coulomb, no LJ
    b = np.array([[0, 1]], np.int32)
    s3, o3 = _one_system(2, [[0, 0, 0], [0, r, 0]], [0.5, -0.25], [1.5, 1.5],
                         sigma=[3.0, 3.4], eps=[0.1, 0.4], bonds=b)
    t3 = oracle.energy(o3, s3.x, s3.q, gb)[0]
    assert t3[1] == 0.0 and t3[2] == 0.0


@pytest.fixture(scope="module")
def small_chain():
    s = synth.make_system(40, 11, n_ph=1, ph_atoms=(6, 6))
    rng = np.random.default_rng(3)
    x = s.x + rng.normal(0, 0.05, size=s.x.shape)  # off the growth lattice: bonds stretched
    return s, oracle.OSystem(s), x


def test_forces_match_central_differences(small_chain):
    s, o, x = small_chain
    gb = GBParams()
    terms, F, _, _ = oracle.energy(o, x, s.q, gb)
    h = 1e-5
    rng = np.random.default_rng(1)
    for i in rng.choice(s.n, 8, replace=False):
        for c in range(3):
            xp = x.copy()
            xm = x.copy()
            xp[i, c] += h
            xm[i, c] -= h
            ep = oracle.energy(o, xp, s.q, gb, forces=False)[0][5]
            em = oracle.energy(o, xm, s.q, gb, forces=False)[0][5]
            fd = -(ep - em) / (2 * h)
            assert F[i, c] == pytest.approx(fd, rel=2e-6, abs=2e-6 * np.abs(F).max())


def test_forces_sum_to_zero_and_no_torque(small_chain):
    s, o, x = small_chain
    _, F, _, _ = oracle.energy(o, x, s.q, GBParams())
    scale = np.abs(F).max()
    assert np.abs(F.sum(0)).max() < 1e-11 * scale * s.n
    torque = np.cross(x, F).sum(0)
    assert np.abs(torque).max() < 1e-10 * scale * s.n * np.abs(x).max()


def test_rigid_motion_invariance(small_chain):
    s, o, x = small_chain
    gb = GBParams()
    t0, F0, R0, _ = oracle.energy(o, x, s.q, gb)
    rng = np.random.default_rng(7)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] *= -1
    x2 = x @ Q.T + np.array([12.3, -4.5, 7.8])
    t1, F1, R1, _ = oracle.energy(o, x2, s.q, gb)
    np.testing.assert_allclose(t1, t0, rtol=1e-12, atol=1e-12 * np.abs(t0).max())
    np.testing.assert_allclose(R1, R0, rtol=1e-12)
    np.testing.assert_allclose(F1, F0 @ Q.T, rtol=0, atol=1e-10 * np.abs(F0).max())


def test_uel_is_a_quadratic_form(small_chain):
    """U_el(q) = 1/2 q^T A q: the parallelogram law holds exactly, and the
    full energy's Coulomb + GB equals U_el at the same Born radii."""
    s, o, x = small_chain
    gb = GBParams()
    terms, _, R, _ = oracle.energy(o, x, s.q, gb)
    assert oracle.u_el(o, x, s.q, R, gb) == pytest.approx(terms[0] + terms[1], rel=1e-13)
    rng = np.random.default_rng(5)
    a = rng.normal(0, 0.3, s.n)
    b = rng.normal(0, 0.3, s.n)
    lhs = oracle.u_el(o, x, a + b, R, gb) + oracle.u_el(o, x, a - b, R, gb)
    rhs = 2 * oracle.u_el(o, x, a, R, gb) + 2 * oracle.u_el(o, x, b, R, gb)
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_gb_gradient_matches_finite_differences(small_chain):
    s, o, x = small_chain
    gb = GBParams()
    E, dx, dq, dr = oracle.gb_grad(x, s.q, s.rho, s.screen, gb)
    # consistency with the full-energy routine
    terms = oracle.energy(o, x, s.q, gb, forces=False)[0]
    assert E == pytest.approx(terms[0], rel=1e-13)
    # Euler: E is homogeneous of degree 2 in q
    assert float(np.dot(s.q, dq)) == pytest.approx(2 * E, rel=1e-12)
    rng = np.random.default_rng(2)
    h = 1e-5
    for i in rng.choice(s.n, 6, replace=False):
        c = int(rng.integers(3))
        xp, xm = x.copy(), x.copy()
        xp[i, c] += h
        xm[i, c] -= h
        fd = (oracle.gb_grad(xp, s.q, s.rho, s.screen, gb)[0]
              - oracle.gb_grad(xm, s.q, s.rho, s.screen, gb)[0]) / (2 * h)
        assert dx[i, c] == pytest.approx(fd, rel=1e-6, abs=1e-7 * np.abs(dx).max())
        rp, rm = s.rho.copy(), s.rho.copy()
        rp[i] += h
        rm[i] -= h
        fd = (oracle.gb_grad(x, s.q, rp, s.screen, gb)[0]
              - oracle.gb_grad(x, s.q, rm, s.screen, gb)[0]) / (2 * h)
        assert dr[i] == pytest.approx(fd, rel=1e-6, abs=1e-7 * np.abs(dr).max())
        qp, qm = s.q.copy(), s.q.copy()
        qp[i] += h
        qm[i] -= h
        fd = (oracle.gb_grad(x, qp, s.rho, s.screen, gb)[0]
              - oracle.gb_grad(x, qm, s.rho, s.screen, gb)[0]) / (2 * h)
        assert dq[i] == pytest.approx(fd, rel=1e-7, abs=1e-8 * np.abs(dq).max())


# ---------------------------------------------------------------- salt screening

def test_salt_born_isolated_ion():
    """With salt the lone ion's Born energy is -1/2 k (1/eps_in - exp(-kappa R)/eps_out) q^2/R."""
    for kappa in (0.05, 0.3):
        gb = GBParams(kappa=kappa)
        q, rho = -0.8, 1.7
        s, o = _one_system(1, [[0.1, 0.2, -0.3]], [q], [rho])
        terms = oracle.energy(o, s.x, s.q, gb)[0]
        Rb = rho - gb.offset
        want = -0.5 * KCOUL * (1 / gb.eps_in - math.exp(-kappa * Rb) / gb.eps_out) * q * q / Rb
        assert terms[0] == pytest.approx(want, rel=1e-14)


def test_salt_far_pair_is_debye_huckel():
    """Far apart (f = r), Coulomb + the GB cross term leave the screened
    Debye-Hueckel interaction k q1 q2 exp(-kappa r) / (eps_out r)."""
    q1, q2 = 0.7, -0.9
    for kappa, r in ((0.1, 30.0), (0.1, 60.0), (0.02, 150.0)):
        gb = GBParams(kappa=kappa)
        s, o = _one_system(2, [[0, 0, 0], [r, 0, 0]], [q1, q2], [1.5, 1.7])
        terms, _, R, _ = oracle.energy(o, s.x, s.q, gb)
        self_e = sum(-0.5 * KCOUL * (1 / gb.eps_in - math.exp(-kappa * R[k]) / gb.eps_out) * qk * qk / R[k]
                     for k, qk in enumerate((q1, q2)))
        pair = terms[0] + terms[1] - self_e
        target = KCOUL * q1 * q2 * math.exp(-kappa * r) / (gb.eps_out * r)
        assert pair == pytest.approx(target, rel=1e-9)


def test_salt_vanishing_kappa_is_salt_free(small_chain):
    s, o, x = small_chain
    t0 = oracle.energy(o, x, s.q, GBParams(), forces=False)[0]
    t1 = oracle.energy(o, x, s.q, GBParams(kappa=1e-12), forces=False)[0]
    np.testing.assert_allclose(t1, t0, rtol=1e-10)


def test_salt_forces_and_gradient_match_central_differences(small_chain):
    s, o, x = small_chain
    gb = GBParams(kappa=0.15)
    terms, F, _, _ = oracle.energy(o, x, s.q, gb)
    E, dx, dq, dr = oracle.gb_grad(x, s.q, s.rho, s.screen, gb)
    assert E == pytest.approx(terms[0], rel=1e-13)
    assert float(np.dot(s.q, dq)) == pytest.approx(2 * E, rel=1e-12)  # still quadratic in q
    h = 1e-5
    rng = np.random.default_rng(5)
    for i in rng.choice(s.n, 6, replace=False):
        c = int(rng.integers(3))
        xp, xm = x.copy(), x.copy()
        xp[i, c] += h
        xm[i, c] -= h
        fd = -(oracle.energy(o, xp, s.q, gb, forces=False)[0][5]
               - oracle.energy(o, xm, s.q, gb, forces=False)[0][5]) / (2 * h)
        assert F[i, c] == pytest.approx(fd, rel=2e-6, abs=2e-6 * np.abs(F).max())
        rp, rm = s.rho.copy(), s.rho.copy()
        rp[i] += h
        rm[i] -= h
        fd = (oracle.gb_grad(x, s.q, rp, s.screen, gb)[0]
              - oracle.gb_grad(x, s.q, rm, s.screen, gb)[0]) / (2 * h)
        assert dr[i] == pytest.approx(fd, rel=1e-6, abs=1e-7 * np.abs(dr).max())


# ---------------------------------------------------------------- nonpolar surface term

def test_sa_term_isolated_atom():
    """ACE surface term of a lone atom (psi = 0, R = rho - offset):
    4 pi gamma (rho + probe)^2 (rho / R)^6 on top of the Born energy."""
    gb = GBParams(sa_gamma=0.005, sa_probe=1.4)
    q, rho = 0.5, 1.8
    s, o = _one_system(1, [[0.0, 0.0, 0.0]], [q], [rho])
    terms = oracle.energy(o, s.x, s.q, gb)[0]
    R = rho - gb.offset
    born = -0.5 * KCOUL * (1 / gb.eps_in - 1 / gb.eps_out) * q * q / R
    sa = 4 * math.pi * 0.005 * (rho + 1.4) ** 2 * (rho / R) ** 6
    assert terms[0] == pytest.approx(born + sa, rel=1e-14)


def test_sa_forces_and_gradient_match_central_differences(small_chain):
    s, o, x = small_chain
    gb = GBParams(sa_gamma=0.007, sa_probe=1.4)
    terms, F, _, _ = oracle.energy(o, x, s.q, gb)
    E, dx, dq, dr = oracle.gb_grad(x, s.q, s.rho, s.screen, gb)
    assert E == pytest.approx(terms[0], rel=1e-13)
    h = 1e-5
    rng = np.random.default_rng(8)
    for i in rng.choice(s.n, 6, replace=False):
        c = int(rng.integers(3))
        xp, xm = x.copy(), x.copy()
        xp[i, c] += h
        xm[i, c] -= h
        fd = -(oracle.energy(o, xp, s.q, gb, forces=False)[0][5]
               - oracle.energy(o, xm, s.q, gb, forces=False)[0][5]) / (2 * h)
        assert F[i, c] == pytest.approx(fd, rel=2e-6, abs=2e-6 * np.abs(F).max())
        fdx = (oracle.gb_grad(xp, s.q, s.rho, s.screen, gb)[0]
               - oracle.gb_grad(xm, s.q, s.rho, s.screen, gb)[0]) / (2 * h)
        assert dx[i, c] == pytest.approx(fdx, rel=1e-6, abs=1e-7 * np.abs(dx).max())
        rp, rm = s.rho.copy(), s.rho.copy()
        rp[i] += h
        rm[i] -= h
        fd = (oracle.gb_grad(x, s.q, rp, s.screen, gb)[0]
              - oracle.gb_grad(x, s.q, rm, s.screen, gb)[0]) / (2 * h)
        assert dr[i] == pytest.approx(fd, rel=1e-6, abs=1e-7 * np.abs(dr).max())



# ---------------------------------------------------------------- Born-radius cutoff

CUT_CASES = [
    # (r, rt, s, rc): sphere straddling the cutoff, wholly beyond it, wholly inside it
    (9.0, 1.4, 1.5, 10.0),
    (10.2, 1.4, 1.5, 10.0),
    (11.6, 1.4, 1.5, 10.0),
    (6.0, 1.4, 1.2, 10.0),
    (4.5, 1.2, 1.8, 5.0),
]


@pytest.mark.parametrize("r,rt,s,rc", CUT_CASES)
def test_hct_cutoff_matches_truncated_shell_quadrature(r, rt, s, rc):
    h = oracle.hct(r, rt, s, rc)
    ref = shell_integral(r, rt, s, rc)
    assert h == pytest.approx(ref, rel=1e-10, abs=1e-14)
    if r - s >= rc:
        assert h == 0.0
    if r + s <= rc:
        assert h == oracle.hct(r, rt, s)


@pytest.mark.parametrize("r,rt,s,rc", CUT_CASES[:2] + CUT_CASES[3:])
def test_hct_cutoff_derivatives_match_finite_differences(r, rt, s, rc):
    h = 1e-6
    H = lambda a, b, c: oracle.hct(a, b, c, rc)
    assert oracle.hct_dr(r, rt, s, rc) == pytest.approx((H(r + h, rt, s) - H(r - h, rt, s)) / (2 * h),
                                                        rel=1e-6, abs=1e-10)
    assert oracle.hct_drt(r, rt, s, rc) == pytest.approx((H(r, rt + h, s) - H(r, rt - h, s)) / (2 * h),
                                                         rel=1e-6, abs=1e-10)
    assert oracle.hct_ds(r, rt, s, rc) == pytest.approx((H(r, rt, s + h) - H(r, rt, s - h)) / (2 * h),
                                                        rel=1e-6, abs=1e-10)


def test_cutoff_forces_and_gradient_match_central_differences(small_chain):
    """A cutoff that cuts: the chain spans ~15 A, rgbmax = 6 A."""
    s, o, x = small_chain
    gb = GBParams(rgbmax=6.0)
    terms, F, R, _ = oracle.energy(o, x, s.q, gb)
    R0 = oracle.energy(o, x, s.q, GBParams())[2]
    assert (R < R0).any() and (R <= R0 + 1e-12).all()  # less descreening: no radius grows
    E, dx, dq, dr = oracle.gb_grad(x, s.q, s.rho, s.screen, gb)
    assert E == pytest.approx(terms[0], rel=1e-13)
    hh = 1e-5
    rng = np.random.default_rng(11)
    for i in rng.choice(s.n, 6, replace=False):
        c = int(rng.integers(3))
        xp, xm = x.copy(), x.copy()
        xp[i, c] += hh
        xm[i, c] -= hh
        fd = -(oracle.energy(o, xp, s.q, gb, forces=False)[0][5]
               - oracle.energy(o, xm, s.q, gb, forces=False)[0][5]) / (2 * hh)
        assert F[i, c] == pytest.approx(fd, rel=2e-6, abs=2e-6 * np.abs(F).max())
        rp, rm = s.rho.copy(), s.rho.copy()
        rp[i] += hh
        rm[i] -= hh
        fd = (oracle.gb_grad(x, s.q, rp, s.screen, gb)[0]
              - oracle.gb_grad(x, s.q, rm, s.screen, gb)[0]) / (2 * hh)
        assert dr[i] == pytest.approx(fd, rel=1e-6, abs=1e-7 * np.abs(dr).max())
