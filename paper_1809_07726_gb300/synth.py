"""Seeded synthetic inputs: heme-peptide-shaped chains with titratable sites.

This module produces inputs only. It holds none of the method's arithmetic (no
Born radii, no energies, no forces, no Monte Carlo and no exchange rule), so the
CUDA engine and the FP64 oracle can both be fed from it without sharing code.

The paper's own system (NAcMP8 + His peptide, 237 atoms, AMBER parameters;
"Parametrization" and "Implicit Solvent Calculations" sections) is not available,
so these systems take its shape instead:

* a compact self-avoiding heavy-atom chain grown inside a sphere of number
  density ~0.05 atoms/A^3 (bond 1.5 A, angle 110 deg, random dihedral, every
  pair three or more bonds apart kept >= 3.0 A apart);
* masses from {12.01, 14.01, 16.00, 32.06} amu, HCT screening factors from the
  matching element classes {0.72, 0.79, 0.85, 0.96};
* intrinsic radii rho ~ U[1.2, 2.0] A, LJ sigma ~ U[1.5, 3.5] A and
  epsilon ~ U[0.05, 0.2] kcal/mol;
* charges ~ N(0, 0.3) e shifted to a net charge of zero in the starting state;
* harmonic bonds (k_b = 300 kcal/mol/A^2, r0 = 1.5 A) and angles
  (k_theta = 60 kcal/mol/rad^2, theta0 = 110 deg) along the chain;
* titratable sites on disjoint contiguous atom blocks.  A pH site has one
  deprotonated state (0 protons) and n-1 protonated tautomers (1 proton each)
  whose charge deltas add +1 e; a redox site has an oxidised state (0
  electrons) and a reduced state (1 electron) whose delta adds -1 e.  Every
  site starts deprotonated / oxidised, as the paper's runs do.

Everything is a deterministic function of the seed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BOND_R0 = 1.5
BOND_K = 300.0
ANGLE_T0 = math.radians(110.0)
ANGLE_K = 60.0
MIN_NONBONDED = 3.0
DENSITY = 0.05

_MASSES = np.array([12.01, 14.01, 16.00, 32.06])
_SCREEN = np.array([0.72, 0.79, 0.85, 0.96])
_CLASS_P = np.array([0.6, 0.2, 0.15, 0.05])


@dataclass
class Site:
    kind: str                 # "ph" or "redox"
    atoms: np.ndarray         # int32 [n_atoms] atom indices
    q: np.ndarray             # float64 [n_states, n_atoms] charges per state
    n_prot: np.ndarray        # int32 [n_states]
    n_elec: np.ndarray        # int32 [n_states]
    ref: float                # pKa_ref (pH) or E0_ref in volts (redox)
    init_state: int = 0


@dataclass
class System:
    x: np.ndarray             # float64 [N, 3] A
    mass: np.ndarray          # float64 [N] amu
    q: np.ndarray             # float64 [N] e, starting-state charges (net 0)
    rho: np.ndarray           # float64 [N] intrinsic radii, A
    screen: np.ndarray        # float64 [N] HCT screening factors
    sigma: np.ndarray         # float64 [N] LJ sigma, A
    eps: np.ndarray           # float64 [N] LJ epsilon, kcal/mol
    bonds: np.ndarray         # int32 [nb, 2]
    bond_k: np.ndarray        # float64 [nb]
    bond_r0: np.ndarray       # float64 [nb]
    angles: np.ndarray        # int32 [na, 3]
    angle_k: np.ndarray       # float64 [na]
    angle_t0: np.ndarray      # float64 [na] radians
    sites: list = field(default_factory=list)
    seed: int = 0

    @property
    def n(self) -> int:
        return int(self.x.shape[0])


def _grow_chain(n: int, rng: np.random.Generator) -> np.ndarray:
    """Self-avoiding chain with fixed bond length and angle inside a sphere.

    Each new atom tries 48 random dihedrals and keeps a valid one: 70% of the
    time the one nearest the centre (to keep the globule compact), else a
    random one.  A
    valid position lies inside the sphere and >= MIN_NONBONDED from every atom
    three or more bonds back.  When none is valid the growth backs up a few
    atoms; every 20 failures without progress the sphere radius grows by 3%
    (soft confinement).  A cubic cell list keeps the distance checks local."""
    radius = (3.0 * n / (4.0 * math.pi * DENSITY)) ** (1.0 / 3.0)
    x = np.zeros((n, 3))
    if n == 1:
        return x
    d = rng.normal(size=3)
    x[1] = x[0] + BOND_R0 * d / np.linalg.norm(d)
    if n == 2:
        return x - x.mean(0)
    b = x[1] - x[0]
    b /= np.linalg.norm(b)
    p = np.cross(b, rng.normal(size=3))
    p /= np.linalg.norm(p)
    st = math.sin(math.pi - ANGLE_T0)
    ct = math.cos(math.pi - ANGLE_T0)
    x[2] = x[1] + BOND_R0 * (ct * b + st * p)
    cell = MIN_NONBONDED + BOND_R0
    cells: dict = {}

    def key(v):
        return (int(math.floor(v[0] / cell)), int(math.floor(v[1] / cell)),
                int(math.floor(v[2] / cell)))

    def add(i):
        cells.setdefault(key(x[i]), []).append(i)

    def remove(i):
        cells[key(x[i])].remove(i)

    for i in range(3):
        add(i)
    ntry = 48
    k = 3
    best = 3
    stall = 0
    while k < n:
        a, bb, c = x[k - 3], x[k - 2], x[k - 1]
        u = c - bb
        u /= np.linalg.norm(u)
        nrm = np.cross(bb - a, u)
        nn = np.linalg.norm(nrm)
        if nn < 1e-9:
            nrm = np.cross(u, rng.normal(size=3))
            nn = np.linalg.norm(nrm)
        nrm /= nn
        m = np.cross(nrm, u)
        phi = rng.uniform(0.0, 2.0 * math.pi, size=ntry)
        dirs = (ct * u[None, :]
                + st * (np.cos(phi)[:, None] * m[None, :] + np.sin(phi)[:, None] * nrm[None, :]))
        cand = c[None, :] + BOND_R0 * dirs
        ok = np.einsum("ij,ij->i", cand, cand) <= radius * radius
        kx, ky, kz = key(c)
        near = []
        for ix in (kx - 1, kx, kx + 1):
            for iy in (ky - 1, ky, ky + 1):
                for iz in (kz - 1, kz, kz + 1):
                    lst = cells.get((ix, iy, iz))
                    if lst:
                        near.extend(j for j in lst if j <= k - 3)
        if near:
            pn = x[np.array(near)]
            d2 = ((cand[:, None, :] - pn[None, :, :]) ** 2).sum(-1)
            ok &= (d2 >= MIN_NONBONDED ** 2).all(1)
        idx = np.flatnonzero(ok)
        if idx.size == 0:
            stall += 1
            if stall % 20 == 0:
                radius *= 1.03
            back = min(k - 3, 1 + int(rng.integers(0, 4)) + stall // 10)
            for _ in range(back):
                k -= 1
                remove(k)
            continue
        if rng.uniform() < 0.7:
            pick = idx[np.argmin(np.einsum("ij,ij->i", cand[idx], cand[idx]))]
        else:
            pick = idx[int(rng.integers(0, idx.size))]
        x[k] = cand[pick]
        add(k)
        k += 1
        if k > best:
            best = k
            stall = 0
    return x - x.mean(0)


def _site_deltas(n_atoms: int, total: float, rng: np.random.Generator) -> np.ndarray:
    w = rng.uniform(0.2, 1.0, size=n_atoms)
    return total * w / w.sum()


def make_system(n: int, seed: int, n_ph: int = 0, ph_states=(2, 2), ph_atoms=(6, 6),
                ph_pka=None, n_redox: int = 1, redox_atoms: int = 16,
                redox_e0: float = -0.2) -> System:
    """Build one seeded synthetic system.

    n_ph pH sites get 2..4 states (``ph_states`` range, inclusive) and 6..12 atoms
    (``ph_atoms`` range, inclusive); ``ph_pka`` is either a list of n_ph values or
    None for pKa_ref ~ U[3.5, 7].  Redox sites have 2 states and ``redox_atoms`` atoms."""
    rng = np.random.default_rng(seed)
    x = _grow_chain(n, rng)
    cls = rng.choice(4, size=n, p=_CLASS_P)
    mass = _MASSES[cls].copy()
    screen = _SCREEN[cls].copy()
    rho = rng.uniform(1.2, 2.0, size=n)
    sigma = rng.uniform(1.5, 3.5, size=n)
    eps = rng.uniform(0.05, 0.2, size=n)
    q = rng.normal(0.0, 0.3, size=n)
    q -= q.mean()
    bonds = np.stack([np.arange(n - 1), np.arange(1, n)], 1).astype(np.int32)
    angles = np.stack([np.arange(n - 2), np.arange(1, n - 1), np.arange(2, n)], 1).astype(np.int32)

    # disjoint contiguous blocks for the sites, spread along the chain
    sizes = []
    kinds = []
    for _ in range(n_redox):
        sizes.append(redox_atoms)
        kinds.append("redox")
    ph_n_states = []
    for _ in range(n_ph):
        sizes.append(int(rng.integers(ph_atoms[0], ph_atoms[1] + 1)))
        kinds.append("ph")
        ph_n_states.append(int(rng.integers(ph_states[0], ph_states[1] + 1)))
    total = sum(sizes)
    if total > n:
        raise ValueError("sites do not fit in the system")
    order = rng.permutation(len(sizes))
    gap = (n - total) // (len(sizes) + 1) if sizes else 0
    starts = {}
    pos = gap
    for o in order:
        starts[o] = pos
        pos += sizes[o] + gap
    sites = []
    iph = 0
    for s_idx, (kind, sz) in enumerate(zip(kinds, sizes)):
        atoms = np.arange(starts[s_idx], starts[s_idx] + sz, dtype=np.int32)
        base = q[atoms].copy()
        if kind == "redox":
            qs = np.stack([base, base + _site_deltas(sz, -1.0, rng)])
            sites.append(Site("redox", atoms, qs, np.zeros(2, np.int32),
                              np.array([0, 1], np.int32), float(redox_e0)))
        else:
            ns = ph_n_states[iph]
            rows = [base] + [base + _site_deltas(sz, 1.0, rng) for _ in range(ns - 1)]
            npr = np.array([0] + [1] * (ns - 1), np.int32)
            if ph_pka is not None:
                pka = float(ph_pka[iph])
            else:
                pka = float(rng.uniform(3.5, 7.0))
            sites.append(Site("ph", atoms, np.stack(rows), npr, np.zeros(ns, np.int32), pka))
            iph += 1
    # pH sites first in index order, then redox sites (the order MC sweeps them)
    sites = [s for s in sites if s.kind == "ph"] + [s for s in sites if s.kind == "redox"]
    return System(x=x, mass=mass, q=q, rho=rho, screen=screen, sigma=sigma, eps=eps,
                  bonds=bonds, bond_k=np.full(n - 1, BOND_K), bond_r0=np.full(n - 1, BOND_R0),
                  angles=angles, angle_k=np.full(n - 2, ANGLE_K),
                  angle_t0=np.full(n - 2, ANGLE_T0), sites=sites, seed=seed)


@dataclass
class Grid:
    E: np.ndarray                  # volts
    pH: np.ndarray
    T: np.ndarray                  # kelvin
    system_of_slot: np.ndarray     # int32 [nE*npH*nT]; slot = iE + nE*(ipH + npH*iT)
    order: tuple = ("E", "pH", "T")

    @property
    def n_slots(self) -> int:
        return len(self.E) * len(self.pH) * len(self.T)


def slot_index(iE: int, ipH: int, iT: int, nE: int, npH: int) -> int:
    return iE + nE * (ipH + npH * iT)


H_MASS, H_RHO, H_SCREEN, H_SIGMA, H_EPS, H_Q = 1.008, 1.2, 0.85, 1.07, 0.0157, 0.1
XH_K, XH_R0 = 340.0, 1.09                 # bond X-H
XXH_K, HXH_K, TETRA = 50.0, 35.0, math.acos(-1.0 / 3.0)


def add_hydrogens(s: System, frac: float, seed: int) -> System:
    """A copy of a heavy-atom system with hydrogens: a fraction ``frac`` of the
    chain atoms carry one or two hydrogens (chain ends three), each 1.09 A
    from its heavy atom, pointing away from the chain neighbours at
    tetrahedral angles, and placed only where it keeps >= 1.6 A from every
    other atom.  A hydrogen takes +0.1 e from its heavy atom (net charge
    unchanged).  Bonds X-H (k 340, r0 1.09) and angles X-X-H (k 50) and H-X-H
    (k 35) at the tetrahedral angle join the force field; hydrogens follow
    their heavy atom in the atom order, and site atoms keep their identity."""
    rng = np.random.default_rng(seed)
    n = s.n
    nbr = [[] for _ in range(n)]
    for a, b in s.bonds:
        nbr[int(a)].append(int(b))
        nbr[int(b)].append(int(a))
    placed = [list(r) for r in s.x]
    hs = [[] for _ in range(n)]
    carry = rng.uniform(size=n) < frac

    def clear(p, skip):
        d = np.linalg.norm(np.asarray(placed) - p, axis=1)
        d[skip] = np.inf
        return d.min() >= 1.6

    for i in range(n):
        if not carry[i] or not nbr[i]:
            continue
        u = [(s.x[j] - s.x[i]) / np.linalg.norm(s.x[j] - s.x[i]) for j in nbr[i]]
        away = -np.sum(u, axis=0)
        away /= np.linalg.norm(away)
        if len(u) == 1:  # chain end: three hydrogens around the bond axis
            ref = np.cross(away, rng.normal(size=3))
            ref /= np.linalg.norm(ref)
            oth = np.cross(away, ref)
            # tetrahedral: each X-H makes 109.47 deg with the X-neighbour bond
            cz, sz = -math.cos(TETRA), math.sin(TETRA)
            dirs = [cz * away + sz * (math.cos(t) * ref + math.sin(t) * oth)
                    for t in (0.0, 2.0943951, 4.1887902)]
        else:
            nrm = np.cross(u[0], u[1])
            nrm /= np.linalg.norm(nrm)
            h = 0.5 * TETRA
            two = [math.cos(h) * away + math.sin(h) * nrm, math.cos(h) * away - math.sin(h) * nrm]
            dirs = two if rng.uniform() < 0.5 else [away]
        for d in dirs:
            p = s.x[i] + XH_R0 * d / np.linalg.norm(d)
            if clear(p, [i]):
                placed.append(list(p))
                hs[i].append(p)
    # new order: each heavy atom followed by its hydrogens
    new_of = np.zeros(n, np.int64)
    xs, mass, q, rho, scr, sig, eps = [], [], [], [], [], [], []
    bonds, bk, br0, angles, ak, at0 = [], [], [], [], [], []
    k = 0
    h_idx = [[] for _ in range(n)]
    for i in range(n):
        new_of[i] = k
        xs.append(s.x[i]); mass.append(s.mass[i]); q.append(s.q[i] - H_Q * len(hs[i]))
        rho.append(s.rho[i]); scr.append(s.screen[i]); sig.append(s.sigma[i]); eps.append(s.eps[i])
        k += 1
        for p in hs[i]:
            h_idx[i].append(k)
            xs.append(p); mass.append(H_MASS); q.append(H_Q); rho.append(H_RHO); scr.append(H_SCREEN)
            sig.append(H_SIGMA); eps.append(H_EPS)
            k += 1
    for (a, b), kk, r0 in zip(s.bonds, s.bond_k, s.bond_r0):
        bonds.append((new_of[a], new_of[b])); bk.append(kk); br0.append(r0)
    for (a, b, c), kk, t0 in zip(s.angles, s.angle_k, s.angle_t0):
        angles.append((new_of[a], new_of[b], new_of[c])); ak.append(kk); at0.append(t0)
    for i in range(n):
        for hh in h_idx[i]:
            bonds.append((new_of[i], hh)); bk.append(XH_K); br0.append(XH_R0)
            for j in nbr[i]:
                angles.append((new_of[j], new_of[i], hh)); ak.append(XXH_K); at0.append(TETRA)
        for a_ in range(len(h_idx[i])):
            for b_ in range(a_ + 1, len(h_idx[i])):
                angles.append((h_idx[i][a_], new_of[i], h_idx[i][b_])); ak.append(HXH_K); at0.append(TETRA)
    sites = [Site(st.kind, new_of[st.atoms].astype(np.int32), st.q.copy(), st.n_prot.copy(),
                  st.n_elec.copy(), st.ref, st.init_state) for st in s.sites]
    return System(x=np.array(xs), mass=np.array(mass), q=np.array(q), rho=np.array(rho),
                  screen=np.array(scr), sigma=np.array(sig), eps=np.array(eps),
                  bonds=np.array(bonds, np.int32).reshape(-1, 2), bond_k=np.array(bk),
                  bond_r0=np.array(br0), angles=np.array(angles, np.int32).reshape(-1, 3),
                  angle_k=np.array(ak), angle_t0=np.array(at0), sites=sites, seed=s.seed)


def titratable_ion(kind: str, ref: float, rho: float = 1.6) -> System:
    """One atom that is a whole titratable site.  pH: state 0 protonated
    (q = 0, one proton), state 1 deprotonated (q = -1).  Redox: state 0
    oxidised (q = 0), state 1 reduced (q = -1, one electron).  A lone atom has
    no descreening partner, so its Born radius, and with it every state's
    electrostatic energy, is the same at any position."""
    z = np.zeros(1)
    q = np.array([[0.0], [-1.0]])
    if kind == "ph":
        site = Site("ph", np.zeros(1, np.int32), q, np.array([1, 0], np.int32),
                    np.zeros(2, np.int32), float(ref))
    else:
        site = Site("redox", np.zeros(1, np.int32), q, np.zeros(2, np.int32),
                    np.array([0, 1], np.int32), float(ref))
    return System(x=np.zeros((1, 3)), mass=np.array([16.0]), q=z.copy(), rho=np.array([rho]),
                  screen=np.array([0.85]), sigma=np.array([3.0]), eps=np.array([0.1]),
                  bonds=np.zeros((0, 2), np.int32), bond_k=z[:0].copy(), bond_r0=z[:0].copy(),
                  angles=np.zeros((0, 3), np.int32), angle_k=z[:0].copy(),
                  angle_t0=z[:0].copy(), sites=[site])


def config_h():
    """A 128-heavy-atom chain with hydrogens on about half its atoms (about 240
    atoms, the size of the paper's NAcMP8 + His peptide system), 2 pH sites
    and 1 redox site; 4 walkers along E at pH 7, 300 K.  For SHAKE."""
    s = add_hydrogens(make_system(128, 8, n_ph=2, ph_states=(2, 2), ph_atoms=(6, 6),
                                  ph_pka=[4.4, 4.85]), 0.55, 8)
    g = Grid(np.linspace(-0.26, -0.14, 4), np.array([7.0]), np.array([300.0]),
             np.zeros(4, np.int32), order=("E",))
    return [s], g


# ---------------------------------------------------------------------------
# The five workloads (systems + condition grids).  Seeds: 1 for the 160-atom
# system, 2 for 2400 atoms, 3/4/5 for 500/2000/8000 atoms, 6 for the 8000-atom
# differentiation system.

def config_c1():
    """160-atom chain, one replica: 1 redox site (16 atoms, E0 = -0.2 V) and
    2 pH sites (6 atoms, 2 states, pKa_ref 4.4 and 4.85); E = -0.2 V, pH 7, 300 K."""
    s = make_system(160, 1, n_ph=2, ph_states=(2, 2), ph_atoms=(6, 6), ph_pka=[4.4, 4.85])
    g = Grid(np.array([-0.2]), np.array([7.0]), np.array([300.0]), np.zeros(1, np.int32))
    return [s], g


def config_c2():
    """Same 160-atom system; 8 replicas at E = -0.35..-0.05 V, pH 7, 300 K."""
    s = config_c1()[0][0]
    g = Grid(np.linspace(-0.35, -0.05, 8), np.array([7.0]), np.array([300.0]),
             np.zeros(8, np.int32), order=("E",))
    return [s], g


def config_c3():
    """2400 atoms, 1 redox + 20 pH sites (2-4 states, 6-12 atoms); 8 E x 8 pH, 300 K."""
    s = make_system(2400, 2, n_ph=20, ph_states=(2, 4), ph_atoms=(6, 12))
    g = Grid(np.linspace(-0.35, -0.05, 8), np.arange(8) * 0.5 + 3.5, np.array([300.0]),
             np.zeros(64, np.int32), order=("E", "pH"))
    return [s], g


def c4_temperatures():
    return 300.0 * (4.0 / 3.0) ** (np.arange(6) / 5.0)


def config_c4(sizes=(500, 2000, 8000), seeds=(3, 4, 5), ph_sites=(4, 16, 64)):
    """8 E x 6 T x 8 pH = 384 replicas over three systems; the system of a slot is
    fixed by its T index: {0,1} -> first, {2,3} -> second, {4,5} -> third."""
    systems = [make_system(n, sd, n_ph=k, ph_states=(2, 4), ph_atoms=(6, 12))
               for n, sd, k in zip(sizes, seeds, ph_sites)]
    nE, npH, nT = 8, 8, 6
    sos = np.zeros(nE * npH * nT, np.int32)
    for iT in range(nT):
        for ipH in range(npH):
            for iE in range(nE):
                sos[slot_index(iE, ipH, iT, nE, npH)] = iT // 2
    g = Grid(np.linspace(-0.35, -0.05, nE), np.arange(npH) * 0.5 + 3.5, c4_temperatures(), sos,
             order=("E", "pH", "T"))
    return systems, g


def config_c5(n_rep: int = 128, n: int = 8000, seed: int = 6):
    """Differentiation workload: n_rep replicas of one seeded n-atom system, each
    with its own seeded coordinate jitter (0.05 A) and charges."""
    s = make_system(n, seed, n_ph=0, n_redox=0)
    rng = np.random.default_rng(seed + 1000)
    x = s.x[None, :, :] + rng.normal(0.0, 0.05, size=(n_rep, n, 3))
    q = s.q[None, :] + rng.normal(0.0, 0.02, size=(n_rep, n))
    rho = np.broadcast_to(s.rho, (n_rep, n)).copy()
    return s, x, q, rho
