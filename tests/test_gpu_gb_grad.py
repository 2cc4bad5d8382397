"""GPU parity of the differentiable GB energy (cph_gb_energy and its adjoint)
against the oracle's analytic FP64 gradient (itself pinned by finite
differences in test_oracle_physics.py)."""
import numpy as np
import pytest

import errlog
import oracle
from paper_1809_07726_gb300 import build, cphremd, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()


def _batch(n_rep, n, seed):
    s, x, q, rho = synth.config_c5(n_rep=n_rep, n=n, seed=seed)
    return s, x, q, rho


def _torch(a, dtype):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda:0")


def _rel_rms(a, b):
    return np.sqrt(((a - b) ** 2).mean()) / np.sqrt((b ** 2).mean())


@pytest.mark.parametrize("n_rep,n", [(3, 300), (2, 129), (1, 7)])
def test_gb_energy_and_gradient_match_oracle(n_rep, n):
    import torch
    s, x, q, rho = _batch(n_rep, n, 60 + n)
    xt, qt, rt = _torch(x, torch.float32), _torch(q, torch.float32), _torch(rho, torch.float32)
    st = _torch(s.screen, torch.float32)
    E = cphremd.gb_energy(xt, qt, rt, st).cpu().numpy()
    up = np.linspace(0.5, 1.5, n_rep)
    dx, dq, dr = (t.cpu().numpy().astype(np.float64) for t in
                  cphremd.gb_energy_backward(xt, qt, rt, st, _torch(up, torch.float64)))
    for r in range(n_rep):
        xr, qr, rr = (a[r].astype(np.float32).astype(np.float64) for a in (x, q, rho))
        Eo, gx, gq, gr = oracle.gb_grad(xr, qr, rr, s.screen.astype(np.float32).astype(np.float64))
        assert abs(E[r] - Eo) <= 1e-6 * abs(Eo), (E[r], Eo)
        assert _rel_rms(dx[r], up[r] * gx) <= 1e-5
        assert _rel_rms(dq[r], up[r] * gq) <= 1e-5
        assert _rel_rms(dr[r], up[r] * gr) <= 1e-5


def test_autograd_function_uses_the_adjoint_kernel():
    import torch
    s, x, q, rho = _batch(2, 200, 7)
    xt = _torch(x, torch.float32).requires_grad_(True)
    qt = _torch(q, torch.float32).requires_grad_(True)
    rt = _torch(rho, torch.float32).requires_grad_(True)
    st = _torch(s.screen, torch.float32)
    E = cphremd.GBEnergy.apply(xt, qt, rt, st)
    (E * torch.tensor([1.0, -2.0], dtype=torch.float64, device="cuda:0")).sum().backward()
    dx, dq, dr = cphremd.gb_energy_backward(xt.detach(), qt.detach(), rt.detach(), st,
                                            torch.tensor([1.0, -2.0], device="cuda:0"))
    assert torch.equal(xt.grad, dx) and torch.equal(qt.grad, dq) and torch.equal(rt.grad, dr)


def test_full_size_batch_sampled_replica():
    """128 replicas of the 8000-atom system in one launch; replica 77 against
    the oracle (energy and gradient)."""
    import torch
    s, x, q, rho = _batch(128, 8000, 6)
    xt, qt, rt = _torch(x, torch.float32), _torch(q, torch.float32), _torch(rho, torch.float32)
    st = _torch(s.screen, torch.float32)
    E = cphremd.gb_energy(xt, qt, rt, st).cpu().numpy()
    dx, dq, dr = (t.cpu().numpy().astype(np.float64) for t in cphremd.gb_energy_backward(
        xt, qt, rt, st, torch.ones(128, dtype=torch.float64, device="cuda:0")))
    r = 77
    xr, qr, rr = (a[r].astype(np.float32).astype(np.float64) for a in (x, q, rho))
    Eo, gx, gq, gr = oracle.gb_grad(xr, qr, rr, s.screen.astype(np.float32).astype(np.float64))
    errlog.record("GB energy and gradient, 128 x 8000 (FP32)", replica=r, energy_rel=abs(E[r] - Eo) / abs(Eo),
                  dx_rms_rel=_rel_rms(dx[r], gx), dq_rms_rel=_rel_rms(dq[r], gq),
                  drho_rms_rel=_rel_rms(dr[r], gr))
    assert abs(E[r] - Eo) <= 1e-6 * abs(Eo)
    assert _rel_rms(dx[r], gx) <= 1e-5
    assert _rel_rms(dq[r], gq) <= 1e-5
    assert _rel_rms(dr[r], gr) <= 1e-5
    # every replica finite and distinct (each saw its own coordinates)
    assert np.isfinite(E).all() and len(np.unique(E)) == 128


def test_obc2_energy_and_gradient_match_oracle():
    """OBC model II ("igb=5": alpha 1.0, beta 0.8, gamma 4.85) through the same kernels."""
    import torch
    v = dict(eps_in=1.0, eps_out=78.5, offset=0.09, alpha=1.0, beta=0.8, gamma=4.85)
    gb = cphremd.GBParams(v["eps_in"], v["eps_out"], v["offset"], v["alpha"], v["beta"], v["gamma"])
    s, x, q, rho = _batch(2, 300, 71)
    xt, qt, rt = _torch(x, torch.float32), _torch(q, torch.float32), _torch(rho, torch.float32)
    st = _torch(s.screen, torch.float32)
    E = cphremd.gb_energy(xt, qt, rt, st, gb=gb).cpu().numpy()
    dx, dq, dr = (t.cpu().numpy().astype(np.float64) for t in cphremd.gb_energy_backward(
        xt, qt, rt, st, torch.ones(2, dtype=torch.float64, device="cuda:0"), gb=gb))
    for r in range(2):
        xr, qr, rr = (a[r].astype(np.float32).astype(np.float64) for a in (x, q, rho))
        Eo, gx, gq, gr = oracle.gb_grad(xr, qr, rr, s.screen.astype(np.float32).astype(np.float64),
                                        oracle.GBParams(**v))
        assert abs(E[r] - Eo) <= 1e-6 * abs(Eo), (E[r], Eo)
        assert _rel_rms(dx[r], gx) <= 1e-5
        assert _rel_rms(dq[r], gq) <= 1e-5
        assert _rel_rms(dr[r], gr) <= 1e-5


@pytest.mark.parametrize("rgbmax,n", [(9.0, 300), (14.0, 700)])
def test_cutoff_energy_and_gradient_match_oracle(rgbmax, n):
    """A Born-radius cutoff through the differentiable energy: the band-aware
    tiles' energy and gradient (including the capped-U terms of dH/dr, dH/ds
    and dH/drt) against the oracle's."""
    import torch
    gb = cphremd.default_gb()
    gb.rgbmax = rgbmax
    s, x, q, rho = _batch(2, n, 43)
    xt, qt, rt = _torch(x, torch.float32), _torch(q, torch.float32), _torch(rho, torch.float32)
    st = _torch(s.screen, torch.float32)
    E = cphremd.gb_energy(xt, qt, rt, st, gb=gb).cpu().numpy()
    dx, dq, dr = (t.cpu().numpy().astype(np.float64) for t in cphremd.gb_energy_backward(
        xt, qt, rt, st, torch.ones(2, dtype=torch.float64, device="cuda:0"), gb=gb))
    for r in range(2):
        xr, qr, rr = (a[r].astype(np.float32).astype(np.float64) for a in (x, q, rho))
        sc = s.screen.astype(np.float32).astype(np.float64)
        Eo, gx, gq, gr = oracle.gb_grad(xr, qr, rr, sc, oracle.GBParams(rgbmax=rgbmax))
        E_full = oracle.gb_grad(xr, qr, rr, sc, oracle.GBParams())[0]
        assert abs(Eo - E_full) > 1e-4 * abs(E_full)  # the cutoff matters here
        assert abs(E[r] - Eo) <= 1e-6 * abs(Eo), (E[r], Eo)
        assert _rel_rms(dx[r], gx) <= 1e-5
        assert _rel_rms(dq[r], gq) <= 1e-5
        assert _rel_rms(dr[r], gr) <= 1e-5


@pytest.mark.parametrize("kappa,extra", [(0.1, {}), (0.05, dict(sa_gamma=0.005, rgbmax=12.0))])
def test_salt_energy_and_gradient_match_oracle(kappa, extra):
    """Debye-Hueckel salt screening through the differentiable energy: every
    GB term carries tau(f) per pair (energy, dE/dq) and its f-derivative (dE/dx,
    dE/dR, hence dE/drho); alone and with the surface term and a cutoff."""
    import torch
    gb = cphremd.default_gb()
    gb.kappa = kappa
    gb.sa_gamma = extra.get("sa_gamma", 0.0)
    gb.rgbmax = extra.get("rgbmax", 0.0)
    s, x, q, rho = _batch(2, 300, 47)
    xt, qt, rt = _torch(x, torch.float32), _torch(q, torch.float32), _torch(rho, torch.float32)
    st = _torch(s.screen, torch.float32)
    E = cphremd.gb_energy(xt, qt, rt, st, gb=gb).cpu().numpy()
    dx, dq, dr = (t.cpu().numpy().astype(np.float64) for t in cphremd.gb_energy_backward(
        xt, qt, rt, st, torch.ones(2, dtype=torch.float64, device="cuda:0"), gb=gb))
    og = oracle.GBParams(kappa=kappa, sa_gamma=gb.sa_gamma, rgbmax=gb.rgbmax)
    for r in range(2):
        xr, qr, rr = (a[r].astype(np.float32).astype(np.float64) for a in (x, q, rho))
        sc = s.screen.astype(np.float32).astype(np.float64)
        Eo, gx, gq, gr = oracle.gb_grad(xr, qr, rr, sc, og)
        E0 = oracle.gb_grad(xr, qr, rr, sc, oracle.GBParams(sa_gamma=gb.sa_gamma, rgbmax=gb.rgbmax))[0]
        assert abs(Eo - E0) > 1e-4 * abs(E0)  # the salt matters here (100x the energy bar)
        assert abs(E[r] - Eo) <= 1e-6 * abs(Eo), (E[r], Eo)
        assert _rel_rms(dx[r], gx) <= 1e-5
        assert _rel_rms(dq[r], gq) <= 1e-5
        assert _rel_rms(dr[r], gr) <= 1e-5


def test_negative_salt_is_refused_by_the_differentiable_energy():
    import torch
    s, x, q, rho = _batch(1, 40, 3)
    xt, qt, rt = _torch(x, torch.float32), _torch(q, torch.float32), _torch(rho, torch.float32)
    st = _torch(s.screen, torch.float32)
    gb = cphremd.GBParams(1.0, 78.5, 0.09, 0.8, 0.0, 2.909125, -0.1)
    with pytest.raises(cphremd.CphError) as e:
        cphremd.gb_energy(xt, qt, rt, st, gb=gb)
    assert e.value.code == cphremd.E_INVALID


def test_surface_term_energy_and_gradient_match_oracle():
    """The ACE surface term through the differentiable energy (energy, and the
    gradient including the explicit rho dependence)."""
    import torch
    gb = cphremd.GBParams(1.0, 78.5, 0.09, 0.8, 0.0, 2.909125, 0.0, 0.006, 1.4)
    s, x, q, rho = _batch(2, 257, 31)
    xt, qt, rt = _torch(x, torch.float32), _torch(q, torch.float32), _torch(rho, torch.float32)
    st = _torch(s.screen, torch.float32)
    E = cphremd.gb_energy(xt, qt, rt, st, gb=gb).cpu().numpy()
    dx, dq, dr = (t.cpu().numpy().astype(np.float64) for t in cphremd.gb_energy_backward(
        xt, qt, rt, st, torch.ones(2, dtype=torch.float64, device="cuda:0"), gb=gb))
    for r in range(2):
        xr, qr, rr = (a[r].astype(np.float32).astype(np.float64) for a in (x, q, rho))
        Eo, gx, gq, gr = oracle.gb_grad(xr, qr, rr, s.screen.astype(np.float32).astype(np.float64),
                                        oracle.GBParams(sa_gamma=0.006, sa_probe=1.4))
        assert abs(E[r] - Eo) <= 1e-6 * abs(Eo), (E[r], Eo)
        assert _rel_rms(dx[r], gx) <= 1e-5
        assert _rel_rms(dq[r], gq) <= 1e-5
        assert _rel_rms(dr[r], gr) <= 1e-5
