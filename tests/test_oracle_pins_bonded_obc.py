"""Pins of the oracle's harmonic bonded terms and of the OBC Born-radius map
against facts fixed outside the oracle's code.

Bonded terms (the paper's Implicit Solvent Calculations section runs AMBER
force fields; AMBER's harmonic terms carry no factor 1/2): a two-atom bond and
a three-atom angle are built at separations and angles known by construction,
so E_bond = k_b (r - r0)^2 and E_angle = k_t (theta - theta0)^2 are checked at
values of r and theta that the test sets, with the force on each atom fixed
by the geometry of the construction (magnitude and direction).  A factor-2
slip, a missing square or a radian/degree mix fails here.

OBC map R(psi) = 1 / (1/rt - tanh(alpha psi - beta psi^2 + gamma psi^3)/rho),
rt = rho - offset (the "igb=2" model the Implicit Solvent Calculations section
names).  Two limits pin where rho and rt enter:
  - small psi: one far neighbour j (r >> s_j) gives psi_i = rt_i s_j^3 / (3 r^4)
    from the point-volume form of the descreening integral, and
    R_i - rt_i -> alpha rt_i^2 psi_i / rho_i;
  - large psi (an atom inside several large spheres): tanh -> 1 and
    R_i -> rho_i rt_i / offset, the model's largest radius.
The higher-order coefficients (beta, gamma) are literature values with no
printed example to pin them against; they are checked only through these two
ends and monotonicity."""
import math

import numpy as np
import pytest

import oracle
from oracle import GBParams
from paper_1809_07726_gb300 import synth


def _system(x, rho=None, screen=None, bonds=None, bond_k=None, bond_r0=None, angles=None,
            angle_k=None, angle_t0=None):
    x = np.asarray(x, float)
    n = len(x)
    e2 = np.zeros((0, 2), np.int32)
    e3 = np.zeros((0, 3), np.int32)
    s = synth.System(x=x, mass=np.full(n, 12.0), q=np.zeros(n),
                     rho=np.full(n, 1.5) if rho is None else np.asarray(rho, float),
                     screen=np.full(n, 0.8) if screen is None else np.asarray(screen, float),
                     sigma=np.full(n, 2.0), eps=np.zeros(n),
                     bonds=e2 if bonds is None else np.asarray(bonds, np.int32),
                     bond_k=np.zeros(0) if bond_k is None else np.asarray(bond_k, float),
                     bond_r0=np.zeros(0) if bond_r0 is None else np.asarray(bond_r0, float),
                     angles=e3 if angles is None else np.asarray(angles, np.int32),
                     angle_k=np.zeros(0) if angle_k is None else np.asarray(angle_k, float),
                     angle_t0=np.zeros(0) if angle_t0 is None else np.asarray(angle_t0, float))
    return s, oracle.OSystem(s)


@pytest.mark.parametrize("r", [1.2, 1.5, 1.93])
def test_two_atom_bond_energy_and_force(r):
    """E_bond = k_b (r - r0)^2; each atom is pulled along the bond by
    2 k_b (r - r0) (toward its partner when stretched)."""
    kb, r0 = 300.0, 1.5
    u = np.array([2.0, -1.0, 2.0]) / 3.0  # unit bond direction
    x = [[0.4, 0.1, -0.3], list(np.array([0.4, 0.1, -0.3]) + r * u)]
    s, o = _system(x, bonds=[[0, 1]], bond_k=[kb], bond_r0=[r0])
    terms, F, _, _ = oracle.energy(o, s.x, s.q, GBParams())
    assert terms[0] == 0.0 and terms[1] == 0.0 and terms[2] == 0.0  # no charge, no LJ
    assert terms[3] == pytest.approx(kb * (r - r0) ** 2, rel=1e-13, abs=1e-13)
    assert terms[4] == 0.0
    mag = 2.0 * kb * (r - r0)
    np.testing.assert_allclose(F[0], mag * u, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(F[1], -mag * u, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("theta_deg", [80.0, 110.0, 152.5])
def test_three_atom_angle_energy_and_force(theta_deg):
    """Vertex j at the origin, i at distance a on the x axis, k at distance b
    at angle theta in the xy plane: E_angle = k_t (theta - theta0)^2.  The
    force on i lies in the plane, perpendicular to the j-i arm, of magnitude
    2 k_t |theta - theta0| / a, turning i toward theta0; likewise for k; the
    vertex takes minus their sum."""
    kt, t0 = 60.0, math.radians(110.0)
    th = math.radians(theta_deg)
    a, b = 1.4, 1.7
    xi = np.array([a, 0.0, 0.0])
    xk = np.array([b * math.cos(th), b * math.sin(th), 0.0])
    s, o = _system([xi, [0.0, 0.0, 0.0], xk], angles=[[0, 1, 2]], angle_k=[kt], angle_t0=[t0])
    terms, F, _, _ = oracle.energy(o, s.x, s.q, GBParams())
    assert terms[3] == 0.0
    assert terms[4] == pytest.approx(kt * (th - t0) ** 2, rel=1e-12, abs=1e-13)
    # direction in which theta grows, for each arm: i turns clockwise (-y),
    # k counterclockwise (away from i)
    grow_i = np.array([0.0, -1.0, 0.0])
    grow_k = np.array([-math.sin(th), math.cos(th), 0.0])
    dEdth = 2.0 * kt * (th - t0)
    np.testing.assert_allclose(F[0], -dEdth / a * grow_i, rtol=1e-11, atol=1e-11)
    np.testing.assert_allclose(F[2], -dEdth / b * grow_k, rtol=1e-11, atol=1e-11)
    np.testing.assert_allclose(F[1], -(F[0] + F[2]), rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("alpha,beta,gamma", [(0.8, 0.0, 2.909125), (1.0, 0.8, 4.85)])
def test_obc_radius_small_psi_slope(alpha, beta, gamma):
    """One far neighbour: psi_i from the point-volume limit of the descreening
    integral, and the first-order OBC radius rt + alpha rt^2 psi / rho."""
    gb = GBParams(alpha=alpha, beta=beta, gamma=gamma)
    rho_i, rho_j, scr_j, r = 1.5, 1.8, 0.85, 60.0
    s, o = _system([[0, 0, 0], [0, 0, r]], rho=[rho_i, rho_j], screen=[0.72, scr_j])
    psi, R = oracle.born(s.x, s.rho, s.screen, gb)
    rt_i = rho_i - gb.offset
    sj = scr_j * (rho_j - gb.offset)
    # point-volume limit, with its leading relative correction O(s^2 / r^2)
    psi_point = rt_i * sj ** 3 / (3.0 * r ** 4)
    assert psi[0] == pytest.approx(psi_point, rel=3 * (sj / r) ** 2)
    slope = (R[0] - rt_i) / psi[0]
    # R - rt = alpha rt^2 psi / rho (1 + O(psi)); rho and rt swapped would be off by 6 %
    assert slope == pytest.approx(alpha * rt_i ** 2 / rho_i, rel=1e-5)
    assert abs(slope - alpha * rho_i ** 2 / rt_i) > 0.1 * slope
    assert abs(slope - alpha * rt_i) > 0.05 * slope


@pytest.mark.parametrize("alpha,beta,gamma", [(0.8, 0.0, 2.909125), (1.0, 0.8, 4.85)])
def test_obc_radius_saturates_at_rho_rt_over_offset(alpha, beta, gamma):
    """An atom inside six large spheres: psi is several units, tanh = 1 to
    rounding, and R = rho rt / offset (1/R = 1/rt - 1/rho)."""
    gb = GBParams(alpha=alpha, beta=beta, gamma=gamma)
    rho_i = 1.5
    d = 0.6
    x = [[0, 0, 0], [d, 0, 0], [-d, 0, 0], [0, d, 0], [0, -d, 0], [0, 0, d], [0, 0, -d]]
    rho = [rho_i] + [12.0] * 6
    s, o = _system(x, rho=rho, screen=[0.8] + [1.0] * 6)
    psi, R = oracle.born(s.x, s.rho, s.screen, gb)
    assert psi[0] > 5.0
    rt = rho_i - gb.offset
    assert R[0] == pytest.approx(rho_i * rt / gb.offset, rel=1e-12)


def test_obc_radius_grows_with_burial():
    """R increases with psi and stays between rt and rho rt / offset: a probe
    atom approached by a growing number of neighbours."""
    gb = GBParams()
    rho_i = 1.6
    rt = rho_i - gb.offset
    dirs = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
            (1, 1, 1), (-1, -1, 1), (1, -1, -1), (-1, 1, -1)]
    last_psi, last_R = 0.0, rt
    for m in range(1, len(dirs) + 1):
        x = [[0, 0, 0]] + [list(3.0 * np.asarray(v, float) / np.linalg.norm(v)) for v in dirs[:m]]
        s, o = _system(x, rho=[rho_i] + [1.9] * m, screen=[0.8] + [0.85] * m)
        psi, R = oracle.born(s.x, s.rho, s.screen, gb)
        assert psi[0] > last_psi and R[0] > last_R
        assert rt < R[0] < rho_i * rt / gb.offset
        last_psi, last_R = psi[0], R[0]
