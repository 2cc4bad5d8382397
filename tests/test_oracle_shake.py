"""Pins of the oracle's SHAKE: the one-constraint case against its closed
form, constraint satisfaction and momentum conservation on a cluster, and
rigid X-H bonds through a scheduled run."""
import math

import numpy as np
import pytest

import oracle
from oracle.run import shake, shake_clusters
from paper_1809_07726_gb300 import synth


def test_single_constraint_matches_closed_form():
    """One bond: the displacement is g r_old (1/m_i, -1/m_j) with g the root of
    |r_new + g (1/m_i + 1/m_j) r_old|^2 = d^2 nearest zero."""
    rng = np.random.default_rng(0)
    m = np.array([12.01, 1.008])
    d0 = 1.09
    u = rng.normal(size=3)
    u /= np.linalg.norm(u)
    x_old = np.array([[0.0, 0.0, 0.0], d0 * u])
    x = x_old + rng.normal(0, 0.03, size=(2, 3))
    x_new = x.copy()
    v = np.zeros_like(x)
    shake(x_old, x, v, m, [(0, [(1, d0)])], 0.002, 1e-14)
    ro = x_old[0] - x_old[1]
    rn = x_new[0] - x_new[1]
    mu = 1 / m[0] + 1 / m[1]
    a, b, c = mu * mu * (ro @ ro), 2 * mu * (rn @ ro), rn @ rn - d0 * d0
    roots = np.roots([a, b, c])
    g = roots[np.argmin(np.abs(roots))].real
    want = x_new + np.array([g * ro / m[0], -g * ro / m[1]])
    np.testing.assert_allclose(x, want, atol=1e-12)
    np.testing.assert_allclose(v, (x - x_new) / 0.002, atol=1e-9)


def test_cluster_satisfies_constraints_and_conserves_momentum():
    rng = np.random.default_rng(1)
    m = np.array([14.01, 1.008, 1.008, 1.008, 1.008])
    d0 = [1.01, 1.02, 1.03, 1.04]
    x_old = np.zeros((5, 3))
    for k in range(4):
        u = rng.normal(size=3)
        x_old[k + 1] = d0[k] * u / np.linalg.norm(u)
    x = x_old + rng.normal(0, 0.04, size=(5, 3))
    x_new = x.copy()
    v = np.zeros_like(x)
    tol = 1e-12
    shake(x_old, x, v, m, [(0, [(k + 1, d0[k]) for k in range(4)])], 0.002, tol)
    for k in range(4):
        d = np.linalg.norm(x[0] - x[k + 1])
        assert abs(d * d - d0[k] ** 2) <= 2 * tol * d0[k] ** 2
    np.testing.assert_allclose((m[:, None] * (x - x_new)).sum(0), 0.0, atol=1e-13)
    # constraint forces act along the old bond vectors only
    dh = x[1:] - x_new[1:]
    rold = x_old[0] - x_old[1:]
    for k in range(4):
        assert np.linalg.norm(np.cross(dh[k], rold[k])) <= 1e-12 * max(1.0, np.linalg.norm(dh[k]))


def test_schedule_keeps_hydrogen_bonds_rigid():
    systems, grid = synth.config_h()
    s = systems[0]
    W = oracle.Walkers(systems, grid, seed=5, mc_ph=5, mc_redox=5, exchange_every=10,
                       shake=True, shake_tol=1e-10)
    oracle.run_schedule(W, 25)
    clusters = shake_clusters(s)
    assert sum(len(h) for _, h in clusters) == int((s.mass < 2).sum())
    for w in range(grid.n_slots):
        x = W.x[w]
        for heavy, hs in clusters:
            for h, d0 in hs:
                d = np.linalg.norm(x[heavy] - x[h])
                assert abs(d * d - d0 * d0) <= 2 * 1e-10 * d0 * d0 * (1 + 1e-9)
        assert np.isfinite(W.v[w]).all()
    # the constrained bonds carry no harmonic energy
    o = W.osys[0]
    hb = [k for k, (a, b) in enumerate(s.bonds) if s.mass[a] < 2 or s.mass[b] < 2]
    assert hb and all(o.bond_k[k] == 0.0 for k in hb)
