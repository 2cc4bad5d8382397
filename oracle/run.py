"""Oracle REMD driver: walker state, C(pH,E)MD sweeps, exchanges, step schedule.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Schedule of global step t (x_t are the positions after t MD steps):
  1. Born radii at x_t;
  2. if t > 0 and t % mc_ph == 0: protonation sweep; then, if t > 0 and
     t % mc_redox == 0: redox sweep (protonation first when both fall on one
     step, as the C(pH,E)MD section of the paper requires);
  3. energies and forces at x_t with the current charges;
  4. if t > 0 and t % exchange_every == 0: one exchange attempt along the next
     dimension of the user order (one dimension per attempt, nearest
     neighbours that share the other two conditions; multidimensional REMD
     section);
  5. one sample of the observables: the state of every site of every walker
     is counted at the walker's current condition, and the walker's visit to
     that condition (the per-condition fractions that eqs (1) and (2) are
     fitted to in the results, and Figure 7's visitation counts);
  6. Langevin step to x_{t+1} at the walker's current temperature, followed,
     when SHAKE is on, by SHAKE on every bond that involves a hydrogen (an
     atom lighter than 2 amu): those bonds are held at their r0 and their
     harmonic terms are left out (the Implicit Solvent Calculations section
     runs SHAKE at 2 fs).
"""
from __future__ import annotations

import dataclasses
import math
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

from . import (DIMS, FARADAY, KB, LN10, PURPOSE_EXCHANGE, PURPOSE_MC_PH, PURPOSE_MC_REDOX,
               GBParams, OSystem, born, energy, langevin, u_el, uniforms)


def reference_energies(osys: OSystem, sysd, gb: GBParams):
    """U_ref[site][state]: U_el of the site's atoms alone, in the starting
    geometry, with their own Born radii (reference-energy reading of the
    Parametrization section: the reference compound is the isolated group)."""
    out = []
    for site in sysd.sites:
        sub = osys.subset(site.atoms)
        xs = np.ascontiguousarray(sysd.x[site.atoms])
        _, Rs = born(xs, sub.rho, sub.screen, gb)
        out.append(np.array([u_el(sub, xs, site.q[s], Rs, gb) for s in range(len(site.q))]))
    return out


@dataclass
class Walkers:
    systems: list                 # synth.System per system id
    grid: object                  # synth.Grid
    seed: int
    dt: float = 0.002
    gamma: float = 10.0
    mc_ph: int = 10
    mc_redox: int = 10
    exchange_every: int = 100
    gb: GBParams = field(default_factory=GBParams)
    t: int = 0
    shake: bool = False
    shake_tol: float = 1e-10
    # energy of eq (5): "potential" = U (total potential energy); "semigrand" =
    # U - sum_k U_ref,k(s_k) + sum_redox F N_e,k(s_k) (E - E0_ref,k), the part of
    # the C(pH,E)MD weight that scales with 1/kT
    t_energy: str = "potential"

    def __post_init__(self):
        if self.shake:
            self.clusters = [shake_clusters(s) for s in self.systems]
            self.osys = [OSystem(dataclasses.replace(s, bond_k=np.where(_h_bond(s), 0.0, s.bond_k)))
                         for s in self.systems]
        else:
            self.osys = [OSystem(s) for s in self.systems]
        self.uref = [reference_energies(o, s, self.gb) for o, s in zip(self.osys, self.systems)]
        ns = self.grid.n_slots
        self.sys_of = np.asarray(self.grid.system_of_slot, np.int64).copy()
        self.x = [np.ascontiguousarray(self.systems[s].x.copy()) for s in self.sys_of]
        self.v = [np.zeros_like(xx) for xx in self.x]
        self.state = [np.array([st.init_state for st in self.systems[s].sites], np.int64)
                      for s in self.sys_of]
        self.q = []
        for w in range(ns):
            sysd = self.systems[self.sys_of[w]]
            q = sysd.q.copy()
            for k, st in enumerate(sysd.sites):
                q[st.atoms] = st.q[self.state[w][k]]
            self.q.append(q)
        self.slot_of = np.arange(ns)
        self.walker_at = np.arange(ns)
        self.n_attempts = {d: 0 for d in self.grid.order}
        self.n_events = 0
        self.U = np.zeros(ns)
        self.terms = np.zeros((ns, 6))
        self.F = [None] * ns
        self.R = [None] * ns
        self.mc_log = []
        self.ex_log = []
        self.threads = 1
        # observables: occ[s][k, state] samples of site k at condition slot s,
        # visits[w, s] samples of walker w at slot s, n_obs samples taken
        self.occ = [np.zeros((len(self.systems[self.sys_of[s]].sites), 8), np.int64)
                    for s in range(ns)]
        self.visits = np.zeros((ns, ns), np.int64)
        self.n_obs = 0

    # -- conditions of a walker
    def cond(self, w):
        nE, npH = len(self.grid.E), len(self.grid.pH)
        s = int(self.slot_of[w])
        iE = s % nE
        ipH = (s // nE) % npH
        iT = s // (nE * npH)
        return self.grid.E[iE], self.grid.pH[ipH], self.grid.T[iT]

    def n_prot(self, w):
        sysd = self.systems[self.sys_of[w]]
        return int(sum(st.n_prot[self.state[w][k]] for k, st in enumerate(sysd.sites)))

    def n_elec(self, w):
        sysd = self.systems[self.sys_of[w]]
        return int(sum(st.n_elec[self.state[w][k]] for k, st in enumerate(sysd.sites)))

    def _map(self, fn, ws):
        if self.threads > 1:
            with ThreadPoolExecutor(self.threads) as ex:
                return list(ex.map(fn, ws))
        return [fn(w) for w in ws]


def mc_sweep(W: Walkers, w: int, kind: str, t: int, R=None):
    """One Monte-Carlo sweep over every site of ``kind`` ("ph" or "redox") of
    walker w, in site-index order, at positions x_t with Born radii R fixed.

    Proposal: b uniform over the other n-1 states, b = k if k < a else k + 1
    with k = floor(u0 (n-1)).  Acceptance: ln u1 < -(G(b) - G(a)) / kT with
    G(s) = U_el(s) - U_ref(s) + kT ln10 N_H(s)(pH - pKa_ref) + F N_e(s)(E - E0_ref).
    U_el(b) - U_el(a) is a full recomputation (the plain definition)."""
    o = W.osys[W.sys_of[w]]
    sysd = W.systems[W.sys_of[w]]
    x = W.x[w]
    if R is None:
        _, R = born(x, o.rho, o.screen, W.gb)
    E, pH, T = W.cond(w)
    kT = KB * T
    purpose = PURPOSE_MC_PH if kind == "ph" else PURPOSE_MC_REDOX
    q = W.q[w]
    for k, st in enumerate(sysd.sites):
        if st.kind != kind:
            continue
        u = uniforms(W.seed, k, w, t, purpose)
        a = int(W.state[w][k])
        n = len(st.q)
        j = int(math.floor(u[0] * (n - 1)))
        b = j if j < a else j + 1
        qb = q.copy()
        qb[st.atoms] = st.q[b]
        dU = u_el(o, x, qb, R, W.gb) - u_el(o, x, q, R, W.gb)
        ur = W.uref[W.sys_of[w]][k]
        dG = dU - (ur[b] - ur[a])
        if kind == "ph":
            dG += kT * LN10 * (st.n_prot[b] - st.n_prot[a]) * (pH - st.ref)
        else:
            dG += FARADAY * (st.n_elec[b] - st.n_elec[a]) * (E - st.ref)
        xexp = -dG / kT
        lnu = math.log(u[1])
        acc = lnu < xexp
        W.mc_log.append((w, k, a, b, dU, xexp, lnu, acc))
        if acc:
            q = qb
            W.state[w][k] = b
    W.q[w] = q


def _line_slots(W: Walkers, dim: str):
    """Every line of slots along ``dim`` (the other two condition indices fixed),
    ordered by the index along dim."""
    nE, npH, nT = len(W.grid.E), len(W.grid.pH), len(W.grid.T)

    def slot(iE, ipH, iT):
        return iE + nE * (ipH + npH * iT)

    lines = []
    if dim == "E":
        for iT in range(nT):
            for ipH in range(npH):
                lines.append([slot(i, ipH, iT) for i in range(nE)])
    elif dim == "pH":
        for iT in range(nT):
            for iE in range(nE):
                lines.append([slot(iE, i, iT) for i in range(npH)])
    else:
        for ipH in range(npH):
            for iE in range(nE):
                lines.append([slot(iE, ipH, i) for i in range(nT)])
    return lines


def exchange_energy(W: Walkers, w: int) -> float:
    """The energy eq (5) uses for walker w at its current condition.  The paper
    calls it "the energy of the system" (T-REMD section); "potential" takes
    the total potential energy U.  In C(pH,E)MD the sampled weight of a
    walker is exp(-(U - sum_k U_ref,k + F sum_redox N_e,k (E - E0_ref,k)) / kT)
    times 10^-(N_H (pH - pKa_ref)) (the state free energy G of the MC moves
    with U_el completed to U), so the part that scales with 1/kT is
    U - sum_k U_ref,k(s_k) + sum_redox F N_e,k(s_k) (E - E0_ref,k): "semigrand"
    takes that one.  The two differ when the pair's site states differ."""
    if W.t_energy == "potential":
        return float(W.U[w])
    if W.t_energy != "semigrand":
        raise ValueError(f"unknown T-exchange energy {W.t_energy!r}")
    sysd = W.systems[W.sys_of[w]]
    ur = W.uref[W.sys_of[w]]
    E = W.cond(w)[0]
    e = float(W.U[w])
    for k, st in enumerate(sysd.sites):
        b = int(W.state[w][k])
        e -= ur[k][b]
        if st.kind == "redox":
            e += FARADAY * st.n_elec[b] * (E - st.ref)
    return e


def exchange_exponent(dim, ci, cj, Ui, Uj, NHi, NHj, Nei, Nej):
    """Exponent x of min{1, e^x} for swapping walkers i and j with conditions
    ci, cj = (E, pH, T): eq (3) for pH, eq (4) for E, eq (5) for T."""
    Ei, pHi, Ti = ci
    Ej, pHj, Tj = cj
    if dim == "pH":
        return LN10 * (pHi - pHj) * (NHi - NHj)
    if dim == "E":
        return FARADAY / (KB * Ti) * (Ei - Ej) * (Nei - Nej)
    return (1.0 / (KB * Ti) - 1.0 / (KB * Tj)) * (Ui - Uj)


def exchange_attempt(W: Walkers, dim: str, t: int):
    """One exchange attempt along ``dim``: neighbours (m, m+1) with m of the
    attempt's parity, within each line, between walkers of the same system.

    Exponents (i = walker at slot m, j = walker at slot m+1):
      pH, eq (3): ln10 (pH_i - pH_j)(N_H,i - N_H,j)
      E,  eq (4): F/(kT) (E_i - E_j)(N_e,i - N_e,j)
      T,  eq (5): (1/kT_i - 1/kT_j)(U_i - U_j), U = exchange_energy (the
                  total potential energy by default)
    Accept iff ln u < x with u = Philox(slot m, dim, t, exchange).  On a T swap
    each walker's velocities are scaled by sqrt(T_new / T_old)."""
    par = W.n_attempts[dim] % 2
    W.n_attempts[dim] += 1
    di = DIMS[dim]
    for line in _line_slots(W, dim):
        for m in range(par, len(line) - 1, 2):
            s1, s2 = line[m], line[m + 1]
            wi, wj = int(W.walker_at[s1]), int(W.walker_at[s2])
            if W.sys_of[wi] != W.sys_of[wj]:
                continue
            Ei, pHi, Ti = W.cond(wi)
            Ej, pHj, Tj = W.cond(wj)
            Ui = exchange_energy(W, wi) if dim == "T" else 0.0
            Uj = exchange_energy(W, wj) if dim == "T" else 0.0
            x = exchange_exponent(dim, (Ei, pHi, Ti), (Ej, pHj, Tj), Ui, Uj,
                                  W.n_prot(wi), W.n_prot(wj), W.n_elec(wi), W.n_elec(wj))
            u = uniforms(W.seed, s1, di, t, PURPOSE_EXCHANGE)
            lnu = math.log(u[0])
            acc = lnu < x
            W.ex_log.append((dim, s1, s2, wi, wj, x, lnu, acc))
            if acc:
                W.walker_at[s1], W.walker_at[s2] = wj, wi
                W.slot_of[wi], W.slot_of[wj] = s2, s1
                if dim == "T":
                    W.v[wi] *= math.sqrt(Tj / Ti)
                    W.v[wj] *= math.sqrt(Ti / Tj)


def _h_bond(sysd):
    m = np.asarray(sysd.mass)
    b = np.asarray(sysd.bonds).reshape(-1, 2)
    return (m[b[:, 0]] < 2.0) | (m[b[:, 1]] < 2.0)


def shake_clusters(sysd):
    """The constrained bonds (those that involve an atom lighter than 2 amu)
    grouped by their heavy atom, in atom order: [(heavy, [(h, r0), ...]), ...],
    each group's hydrogens in bond-list order."""
    m = np.asarray(sysd.mass)
    groups = {}
    for (a, b), r0, hb in zip(np.asarray(sysd.bonds).reshape(-1, 2), sysd.bond_r0, _h_bond(sysd)):
        if not hb:
            continue
        heavy, h = (int(a), int(b)) if m[b] < 2.0 else (int(b), int(a))
        if m[heavy] < 2.0:
            raise ValueError("a bond between two hydrogens cannot be constrained")
        groups.setdefault(heavy, []).append((h, float(r0)))
    return sorted(groups.items())


def shake(x_old, x, v, mass, clusters, dt, tol, max_iter=1000):
    """SHAKE (Ryckaert, Ciccotti & Berendsen 1977) after a leapfrog step from
    x_old: each constraint in turn moves its two atoms along the old bond
    vector, in inverse proportion to their masses, until every constrained
    distance d satisfies |d0^2 - d^2| <= 2 tol d0^2; a cluster (one heavy atom
    and its hydrogens) is swept until none of its constraints moves.  The
    velocities take the same displacement divided by dt."""
    x_start = x.copy()
    for heavy, hs in clusters:
        for _ in range(max_iter):
            done = True
            for h, d0 in hs:
                rij = x[heavy] - x[h]
                diff = d0 * d0 - float(rij @ rij)
                if abs(diff) > 2.0 * tol * d0 * d0:
                    done = False
                    rold = x_old[heavy] - x_old[h]
                    g = diff / (2.0 * float(rold @ rij) * (1.0 / mass[heavy] + 1.0 / mass[h]))
                    x[heavy] += g * rold / mass[heavy]
                    x[h] -= g * rold / mass[h]
            if done:
                break
        else:
            raise RuntimeError("SHAKE did not converge")
    v += (x - x_start) / dt


def run_schedule(W: Walkers, n_steps: int, walkers=None):
    """Advance every walker (or the listed subset, for timing samples) by
    n_steps of the schedule in the module docstring."""
    ws = list(range(W.grid.n_slots)) if walkers is None else list(walkers)
    for _ in range(n_steps):
        t = W.t

        def radii(w):
            o = W.osys[W.sys_of[w]]
            return born(W.x[w], o.rho, o.screen, W.gb)[1]

        R = dict(zip(ws, W._map(radii, ws)))
        if t > 0 and W.mc_ph > 0 and t % W.mc_ph == 0:
            for w in ws:
                mc_sweep(W, w, "ph", t, R[w])
        if t > 0 and W.mc_redox > 0 and t % W.mc_redox == 0:
            for w in ws:
                mc_sweep(W, w, "redox", t, R[w])

        def ef(w):
            o = W.osys[W.sys_of[w]]
            return energy(o, W.x[w], W.q[w], W.gb)

        res = W._map(ef, ws)
        for w, (terms, F, Rw, _) in zip(ws, res):
            W.terms[w] = terms
            W.U[w] = terms[5]
            W.F[w] = F
            W.R[w] = Rw
        if t > 0 and W.exchange_every > 0 and t % W.exchange_every == 0 and walkers is None:
            dim = W.grid.order[W.n_events % len(W.grid.order)]
            W.n_events += 1
            exchange_attempt(W, dim, t)

        for w in ws:
            s = int(W.slot_of[w])
            W.visits[w, s] += 1
            for k, st in enumerate(W.state[w]):
                W.occ[s][k, st] += 1
        W.n_obs += 1

        def step(w):
            o = W.osys[W.sys_of[w]]
            T = W.cond(w)[2]
            x_old = W.x[w].copy() if W.shake else None
            langevin(W.x[w], W.v[w], W.F[w], o.mass, W.dt, W.gamma, T, W.seed, w, t)
            if W.shake:
                shake(x_old, W.x[w], W.v[w], o.mass, W.clusters[W.sys_of[w]], W.dt, W.shake_tol)

        W._map(step, ws)
        W.t += 1
