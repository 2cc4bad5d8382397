"""SHAKE on bonds to hydrogen (the paper's 2 fs runs constrain them) on the
GPU against the oracle: the FP64 whole schedule on a 246-atom system with
hydrogens, one FP32 step, rigid X-H bonds, launch-shape invariance, and the
set-up's refusals."""
import numpy as np
import pytest

import oracle
from oracle.run import shake_clusters
from paper_1809_07726_gb300 import cphremd, synth

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _xh_err(x, clusters):
    worst = 0.0
    for heavy, hs in clusters:
        for h, d0 in hs:
            d = np.linalg.norm(x[heavy] - x[h])
            worst = max(worst, abs(d * d - d0 * d0) / (d0 * d0))
    return worst


def test_fp64_schedule_with_shake_matches_oracle():
    systems, grid = synth.config_h()
    kw = dict(mc_ph_every=10, mc_redox_every=10, exchange_every=20)
    eng = cphremd.init_system(systems, grid, seed=6, precision=cphremd.PREC_FP64, shake=True,
                              shake_tol=TOL, **kw)
    W = oracle.Walkers(systems, grid, seed=6, mc_ph=10, mc_redox=10, exchange_every=20,
                       shake=True, shake_tol=TOL)
    n = 60
    eng.run(n)
    eng.status()
    oracle.run_schedule(W, n)
    x, v = eng.positions(), eng.velocities()
    cl = shake_clusters(systems[0])
    for w in range(grid.n_slots):
        sl = eng.walker_slice(w)
        np.testing.assert_allclose(x[sl], W.x[w], rtol=0, atol=1e-8)
        np.testing.assert_allclose(v[sl], W.v[w], rtol=0, atol=1e-5)
        assert _xh_err(x[sl], cl) <= 2 * TOL * (1 + 1e-6)
    np.testing.assert_array_equal(eng.condition_map(), W.slot_of)
    np.testing.assert_array_equal(eng.site_states(), np.concatenate(W.state))


def test_fp32_step_with_shake_matches_oracle():
    systems, grid = synth.config_h()
    eng = cphremd.init_system(systems, grid, seed=9, shake=True, shake_tol=TOL)
    eng.set_step(3)
    eng.step_replicas(1)
    eng.status()
    W = oracle.Walkers(systems, grid, seed=9, shake=True, shake_tol=TOL)
    W.t = 3
    oracle.run_schedule(W, 1, walkers=[0])
    s = systems[0]
    sl = eng.walker_slice(0)

    def rel_rms(a, b):
        return np.sqrt(((a - b) ** 2).mean()) / np.sqrt((b ** 2).mean())

    assert rel_rms(eng.velocities()[sl], W.v[0]) <= 1e-5
    assert rel_rms(eng.positions()[sl] - s.x, W.x[0] - s.x) <= 1e-5
    assert _xh_err(eng.positions()[sl], shake_clusters(s)) <= 2 * TOL * (1 + 1e-6)


def test_shake_runs_are_launch_shape_invariant():
    systems, grid = synth.config_h()
    a = cphremd.init_system(systems, grid, seed=4, shake=True, shake_tol=1e-8)
    b = cphremd.init_system(systems, grid, seed=4, shake=True, shake_tol=1e-8)
    b.set_launch_mode(cphremd.LAUNCH_PER_REPLICA)
    b.set_replica_streams(2)
    a.run(23)
    b.run(23)
    for get in ("positions", "velocities", "site_states", "condition_map"):
        np.testing.assert_array_equal(getattr(a, get)(), getattr(b, get)())


def test_shake_set_up_refusals():
    systems, grid = synth.config_h()
    with pytest.raises(cphremd.CphError):
        cphremd.init_system(systems, grid, seed=1, shake=True, shake_tol=0.0)
    s = systems[0]
    hs = np.flatnonzero(s.mass < 2.0)
    bad = synth.System(**{**s.__dict__, "bonds": np.vstack([s.bonds, [[hs[0], hs[1]]]]).astype(np.int32),
                          "bond_k": np.append(s.bond_k, 300.0), "bond_r0": np.append(s.bond_r0, 1.5)})
    with pytest.raises(cphremd.CphError):  # a bond between two hydrogens
        cphremd.init_system([bad], grid, seed=1, shake=True, shake_tol=1e-8)
    cphremd.init_system([bad], grid, seed=1)  # fine without SHAKE
