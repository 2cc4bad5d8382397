"""Plain FP64 CPU oracle for the GB-OBC / C(pH,E)MD REMD hot path.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the CPU-baseline
leg of the benchmark are the only callers.  The oracle shares no code with the
CUDA engine; both are fed from the seeded input generator, which holds none of
the method's arithmetic.

Layout:
  cph_oracle.c  pair physics (Born radii, GB/Coulomb/LJ, bonded terms, forces,
                GB gradient), Philox4x32-10, the Langevin step;
  this module   ctypes bindings, 1-2/1-3 exclusions from the bond graph, the
                isolated-site reference energies, the C(pH,E)MD Monte-Carlo
                sweep, the Metropolis exchanges along E, pH and T, the step
                schedule, the closed forms of eqs (1), (2), (6)-(8), and
                the sampling observables (per-condition fractions, Hill fits
                of eqs (1) and (2); counters in run.py).

Readings of the paper where it is silent (it prints no GB formula, MC move set,
integrator or constant): the OBC "igb=2" model with HCT descreening, constants
below, leapfrog Langevin, one sweep over all sites of a kind per MC event with
a uniform proposal among the other states, and G(s) = U_el(s) - U_ref(s)
+ kT ln10 N_H(s) (pH - pKa_ref) + F N_e(s) (E - E0_ref).
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "liboracle.so")
SRC = os.path.join(HERE, "cph_oracle.c")

KCOUL = 332.0522173          # kcal A / (mol e^2)
KB = 0.0019872041            # kcal / (mol K)
FARADAY = 23.0605            # kcal / (mol V)
LN10 = math.log(10.0)

PURPOSE_LANGEVIN = 1
PURPOSE_MC_PH = 2
PURPOSE_MC_REDOX = 3
PURPOSE_EXCHANGE = 4
DIMS = {"E": 0, "pH": 1, "T": 2}

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle library with the host C compiler."""
    with _lock:
        if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
            tmp = LIB + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fno-fast-math",
                                   "-o", tmp, SRC, "-lm"])
            os.replace(tmp, LIB)
    return LIB


class OGB(C.Structure):
    _fields_ = [("eps_in", C.c_double), ("eps_out", C.c_double), ("offset", C.c_double),
                ("alpha", C.c_double), ("beta", C.c_double), ("gamma", C.c_double),
                ("kappa", C.c_double), ("sa_gamma", C.c_double), ("sa_probe", C.c_double),
                ("rgbmax", C.c_double)]


class OSYS(C.Structure):
    _fields_ = [("n", C.c_int),
                ("rho", C.c_void_p), ("screen", C.c_void_p), ("sigma", C.c_void_p),
                ("eps", C.c_void_p), ("excl", C.c_void_p),
                ("n_bonds", C.c_int), ("bonds", C.c_void_p), ("bond_k", C.c_void_p),
                ("bond_r0", C.c_void_p),
                ("n_angles", C.c_int), ("angles", C.c_void_p), ("angle_k", C.c_void_p),
                ("angle_t0", C.c_void_p)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        d, vp, i, u32, u64 = C.c_double, C.c_void_p, C.c_int, C.c_uint32, C.c_uint64
        L.o_hct.restype = d
        L.o_hct.argtypes = [d, d, d]
        for f in (L.o_hct_rc, L.o_hct_dr_rc, L.o_hct_drt_rc, L.o_hct_ds_rc):
            f.restype = d
            f.argtypes = [d, d, d, d]
        for f in (L.o_hct_dr, L.o_hct_drt, L.o_hct_ds):
            f.restype = d
            f.argtypes = [d, d, d]
        L.o_born.argtypes = [i, vp, vp, vp, C.POINTER(OGB), vp, vp]
        L.o_uel.restype = d
        L.o_uel.argtypes = [C.POINTER(OSYS), C.POINTER(OGB), vp, vp, vp]
        L.o_energy.argtypes = [C.POINTER(OSYS), C.POINTER(OGB), vp, vp, vp, vp, vp, vp]
        L.o_gb_grad.argtypes = [i, vp, vp, vp, vp, C.POINTER(OGB), vp, vp, vp, vp]
        L.o_philox.argtypes = [vp, vp, vp]
        L.o_uniforms.argtypes = [u64, u32, u32, u64, u32, vp]
        L.o_normals3.argtypes = [u64, u32, u32, u64, u32, vp]
        L.o_langevin.argtypes = [i, vp, vp, vp, vp, d, d, d, u64, u32, u64]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


@dataclass
class GBParams:
    """OBC model I ("igb=2") values: offset 0.09 A, (alpha, beta, gamma) =
    (0.8, 0.0, 2.909125); eps_in = 1, eps_out = 78.5; no salt (kappa = 0).
    With kappa > 0 every GB term -k q_i q_j tau / f takes tau(f) = 1/eps_in -
    exp(-kappa f)/eps_out (Debye-Hueckel screening of the reaction field).
    With sa_gamma > 0 the GB term also holds the nonpolar surface energy in the
    ACE approximation, sum_i 4 pi sa_gamma (rho_i + sa_probe)^2 (rho_i/R_i)^6."""
    eps_in: float = 1.0
    eps_out: float = 78.5
    offset: float = 0.09
    alpha: float = 0.8
    beta: float = 0.0
    gamma: float = 2.909125
    kappa: float = 0.0     # salt screening (Debye-Hueckel), 1/A; 0 = no salt
    sa_gamma: float = 0.0  # nonpolar surface term (ACE), kcal/mol/A^2; 0 = off
    sa_probe: float = 1.4  # solvent probe radius of the surface term, A
    rgbmax: float = 0.0    # Born-radius cutoff, A; 0 = none

    def c(self) -> OGB:
        return OGB(self.eps_in, self.eps_out, self.offset, self.alpha, self.beta, self.gamma,
                   self.kappa, self.sa_gamma, self.sa_probe, self.rgbmax)


def exclusion_matrix(n: int, bonds: np.ndarray, extra=None) -> np.ndarray:
    """1 for every pair one or two bonds apart in the bond graph (1-2 and 1-3),
    plus any extra listed pairs.  The diagonal stays 0 (self pairs are never
    part of the pair sums)."""
    nb = [set() for _ in range(n)]
    for a, b in np.asarray(bonds).reshape(-1, 2):
        nb[a].add(int(b))
        nb[b].add(int(a))
    ex = np.zeros((n, n), np.uint8)
    for i in range(n):
        for j in nb[i]:
            ex[i, j] = 1
            for k in nb[j]:
                if k != i:
                    ex[i, k] = 1
    if extra is not None:
        for a, b in np.asarray(extra).reshape(-1, 2):
            ex[a, b] = ex[b, a] = 1
    return ex


class OSystem:
    """One system's topology and parameters held in contiguous FP64 arrays."""

    def __init__(self, sysd, extra_excl=None):
        self._set(sysd.rho, sysd.screen, sysd.sigma, sysd.eps, sysd.mass,
                  exclusion_matrix(sysd.n, sysd.bonds, extra_excl),
                  sysd.bonds, sysd.bond_k, sysd.bond_r0,
                  sysd.angles, sysd.angle_k, sysd.angle_t0)

    def _set(self, rho, screen, sigma, eps, mass, excl, bonds, bond_k, bond_r0,
             angles, angle_k, angle_t0):
        f = lambda a: np.ascontiguousarray(a, np.float64)  # noqa: E731
        self.n = len(rho)
        self.rho, self.screen, self.sigma, self.eps, self.mass = map(f, (rho, screen, sigma,
                                                                        eps, mass))
        self.excl = np.ascontiguousarray(excl, np.uint8)
        self.bonds = np.ascontiguousarray(np.asarray(bonds).reshape(-1, 2), np.int32)
        self.angles = np.ascontiguousarray(np.asarray(angles).reshape(-1, 3), np.int32)
        self.bond_k, self.bond_r0, self.angle_k, self.angle_t0 = map(
            f, (bond_k, bond_r0, angle_k, angle_t0))
        self.c = OSYS(self.n, _p(self.rho).value, _p(self.screen).value, _p(self.sigma).value,
                      _p(self.eps).value, _p(self.excl).value,
                      len(self.bonds), _p(self.bonds).value, _p(self.bond_k).value,
                      _p(self.bond_r0).value,
                      len(self.angles), _p(self.angles).value, _p(self.angle_k).value,
                      _p(self.angle_t0).value)

    def subset(self, atoms):
        """The isolated group of ``atoms``: its own parameters and exclusions, no
        bonded terms."""
        a = np.asarray(atoms)
        o = OSystem.__new__(OSystem)
        o._set(self.rho[a], self.screen[a], self.sigma[a], self.eps[a], self.mass[a],
               self.excl[np.ix_(a, a)], np.zeros((0, 2)), [], [], np.zeros((0, 3)), [], [])
        return o


# ------------------------------------------------------------ pair physics

def hct(r, rt, s, rc=0.0):
    """Descreening integral H(r, rt, s); rc > 0 cuts it at that radius
    (Born-radius cutoff, AMBER's rgbmax)."""
    return lib().o_hct_rc(r, rt, s, rc)


def hct_dr(r, rt, s, rc=0.0):
    return lib().o_hct_dr_rc(r, rt, s, rc)


def hct_drt(r, rt, s, rc=0.0):
    return lib().o_hct_drt_rc(r, rt, s, rc)


def hct_ds(r, rt, s, rc=0.0):
    return lib().o_hct_ds_rc(r, rt, s, rc)


def born(x, rho, screen, gb: GBParams = GBParams()):
    """(psi, R) for one configuration x [N,3]."""
    x = np.ascontiguousarray(x, np.float64)
    rho = np.ascontiguousarray(rho, np.float64)
    screen = np.ascontiguousarray(screen, np.float64)
    n = len(rho)
    psi = np.zeros(n)
    R = np.zeros(n)
    g = gb.c()
    lib().o_born(n, _p(x), _p(rho), _p(screen), C.byref(g), _p(psi), _p(R))
    return psi, R


def energy(osys: OSystem, x, q, gb: GBParams = GBParams(), forces=True):
    """(terms, F, R, psi); terms = [E_GB, E_coul, E_LJ, E_bond, E_angle, total]."""
    x = np.ascontiguousarray(x, np.float64)
    q = np.ascontiguousarray(q, np.float64)
    terms = np.zeros(6)
    F = np.zeros((osys.n, 3)) if forces else None
    R = np.zeros(osys.n)
    psi = np.zeros(osys.n)
    g = gb.c()
    lib().o_energy(C.byref(osys.c), C.byref(g), _p(x), _p(q), _p(terms),
                   _p(F) if forces else None, _p(R), _p(psi))
    return terms, F, R, psi


def u_el(osys: OSystem, x, q, R, gb: GBParams = GBParams()) -> float:
    """E_coul + E_GB with fixed Born radii R."""
    x = np.ascontiguousarray(x, np.float64)
    q = np.ascontiguousarray(q, np.float64)
    R = np.ascontiguousarray(R, np.float64)
    g = gb.c()
    return lib().o_uel(C.byref(osys.c), C.byref(g), _p(x), _p(q), _p(R))


def gb_grad(x, q, rho, screen, gb: GBParams = GBParams()):
    """(E_GB, dE/dx [N,3], dE/dq [N], dE/drho [N]) for one configuration."""
    x = np.ascontiguousarray(x, np.float64)
    q = np.ascontiguousarray(q, np.float64)
    rho = np.ascontiguousarray(rho, np.float64)
    screen = np.ascontiguousarray(screen, np.float64)
    n = len(q)
    E = np.zeros(1)
    dx = np.zeros((n, 3))
    dq = np.zeros(n)
    dr = np.zeros(n)
    g = gb.c()
    lib().o_gb_grad(n, _p(x), _p(q), _p(rho), _p(screen), C.byref(g), _p(E), _p(dx),
                    _p(dq), _p(dr))
    return float(E[0]), dx, dq, dr


# ------------------------------------------------------------------ Philox

def philox(ctr, key):
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().o_philox(_p(c), _p(k), _p(out))
    return out


def uniforms(seed, index, stream, step, purpose):
    out = np.zeros(4)
    lib().o_uniforms(seed, index, stream, step, purpose, _p(out))
    return out


def normals3(seed, index, stream, step, purpose=PURPOSE_LANGEVIN):
    out = np.zeros(3)
    lib().o_normals3(seed, index, stream, step, purpose, _p(out))
    return out


def langevin(x, v, F, mass, dt, gamma, T, seed, walker, step):
    """One leapfrog Langevin step in place on x, v [N,3]."""
    assert x.flags.c_contiguous and v.flags.c_contiguous
    F = np.ascontiguousarray(F, np.float64)
    mass = np.ascontiguousarray(mass, np.float64)
    lib().o_langevin(len(mass), _p(x), _p(v), _p(F), _p(mass), dt, gamma, T, seed, walker,
                     step)


# ------------------------------------------------------ closed-form curves

def f_prot(pH, pKa, n_hill=1.0):
    """Eq (1): fraction protonated."""
    return 1.0 / (1.0 + np.exp(n_hill * LN10 * (np.asarray(pH) - pKa)))


def f_red(E, E0, T, v=1.0, n_hill=1.0):
    """Eq (2): fraction reduced."""
    return 1.0 / (1.0 + np.exp(n_hill * v * FARADAY / (KB * T) * (np.asarray(E) - E0)))


def eq6_delta_e0(pka_red, pka_oxi, T, v=1.0):
    """Eq (6): E0_prot - E0_deprot."""
    return KB * T * LN10 * np.sum(np.asarray(pka_red) - np.asarray(pka_oxi)) / (v * FARADAY)


def eq7_e0(pH, e0_prot, pka_red, pka_oxi, T, v=1.0):
    """Eq (7): pH-dependent standard redox potential."""
    s = 0.0
    for pr, po in zip(pka_red, pka_oxi):
        s += np.log((10.0 ** -pr + 10.0 ** -pH) / (10.0 ** -po + 10.0 ** -pH))
    return e0_prot + KB * T / (v * FARADAY) * s


def eq8_sum_pka(E, e0_prot, e0_deprot, pka_red, T, v=1.0):
    """Eq (8): redox-potential-dependent sum of pKa values (log base 10)."""
    b = FARADAY / (KB * T)
    num = np.exp(-v * b * e0_prot) + np.exp(-b * E)
    den = np.exp(-v * b * e0_deprot) + np.exp(-b * E)
    return np.sum(pka_red) + np.log10(num / den)


# ------------------------------------------------------ sampling observables

def site_fractions(W):
    """Per condition slot s, per site k of the walker sitting there: the
    sampled fraction protonated (pH site) or reduced (redox site), i.e. the
    mean over samples of (n(state) - n_min) / (n_max - n_min), n = protons or
    electrons of the state.  Returns a list over slots of arrays [n_sites]."""
    out = []
    for s, occ in enumerate(W.occ):
        sysd = W.systems[W.sys_of[s]]
        fr = np.zeros(len(sysd.sites))
        for k, st in enumerate(sysd.sites):
            n = np.asarray(st.n_prot if st.kind == "ph" else st.n_elec, np.float64)
            if n.max() > n.min():
                w = (n - n.min()) / (n.max() - n.min())
                fr[k] = sum(occ[k, t] * w[t] for t in range(len(n))) / W.n_obs
        out.append(fr)
    return out


def fit_hill(kind, x, f, T=300.0, v=1.0):
    """Least-squares fit of eq (1) (kind "pH": f = 1/(1 + 10^(n (pH - pKa))))
    or eq (2) (kind "redox": f = 1/(1 + exp(n v F (E - E0)/(kB T)))) to the
    fractions f at x.  Minimises the sum of squared fraction residuals with
    scipy's Levenberg-Marquardt, started from a straight-line fit of the Hill
    plot.  Returns (x0, n, rss)."""
    from scipy.optimize import least_squares

    x = np.asarray(x, np.float64)
    f = np.asarray(f, np.float64)

    def model(p):
        return f_prot(x, p[0], p[1]) if kind == "pH" else f_red(x, p[0], T, v, p[1])

    c = LN10 if kind == "pH" else v * FARADAY / (KB * T)
    inside = (f > 0) & (f < 1)
    fc = np.clip(f[inside], 1e-6, 1 - 1e-6)
    slope, icpt = np.polyfit(x[inside], np.log((1 - fc) / fc) / c, 1)
    res = least_squares(lambda p: f - model(p), [-icpt / slope, slope], method="lm",
                        xtol=1e-15, ftol=1e-15, gtol=1e-15)
    return float(res.x[0]), float(res.x[1]), float(np.sum(res.fun ** 2))


from .run import (Walkers, exchange_attempt, exchange_energy, exchange_exponent,  # noqa: E402,F401
                  mc_sweep, reference_energies, run_schedule)
