"""Thin Python binding of libcphremd.so (the C ABI in include/cphremd.h).

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  Function names follow the C calls without their ``cph_``
prefix.  The library must have been built (``paper_1809_07726_gb300.build``);
there is no fallback of any kind when it is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import LIB

# ---- constants mirrored from cphremd.h
OK, E_INVALID, E_CUDA, E_OOM, E_NONFINITE, E_TIMEOUT, E_STATE = 0, -1, -2, -3, -4, -5, -6
SITE_PH, SITE_REDOX = 0, 1
DIM_E, DIM_PH, DIM_T, DIM_NEXT = 0, 1, 2, -1
MC_PH, MC_REDOX, MC_BOTH = 1, 2, 3
PREC_FP64, PREC_FP32 = 0, 1
LAUNCH_BATCHED, LAUNCH_PER_REPLICA = 0, 1
TEX_POTENTIAL, TEX_SEMIGRAND = 0, 1
SHAPE_SYMMETRIC, SHAPE_WARP_PER_ATOM = 0, 1
NTERMS = 6
MAX_STATES = 8
FIT_PH, FIT_REDOX = 1, 2
TERMS = ("gb", "coul", "lj", "bond", "angle", "total")
DIM_NAMES = {"E": DIM_E, "pH": DIM_PH, "T": DIM_T}


class CphError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"cph error {code}: {msg}")
        self.code = code


class SiteDesc(C.Structure):
    _fields_ = [("kind", C.c_int), ("n_atoms", C.c_int), ("atoms", C.c_void_p),
                ("n_states", C.c_int), ("q", C.c_void_p), ("n_prot", C.c_void_p),
                ("n_elec", C.c_void_p), ("ref", C.c_double), ("init_state", C.c_int)]


class SystemDesc(C.Structure):
    _fields_ = [("n_atoms", C.c_int), ("x", C.c_void_p), ("v", C.c_void_p),
                ("mass", C.c_void_p), ("q", C.c_void_p), ("rho", C.c_void_p),
                ("screen", C.c_void_p), ("sigma", C.c_void_p), ("eps", C.c_void_p),
                ("n_bonds", C.c_int), ("bonds", C.c_void_p), ("bond_k", C.c_void_p),
                ("bond_r0", C.c_void_p), ("n_angles", C.c_int), ("angles", C.c_void_p),
                ("angle_k", C.c_void_p), ("angle_t0", C.c_void_p), ("n_excl", C.c_int),
                ("excl", C.c_void_p), ("n_sites", C.c_int), ("sites", C.c_void_p)]


class GridDesc(C.Structure):
    _fields_ = [("nE", C.c_int), ("npH", C.c_int), ("nT", C.c_int), ("E", C.c_void_p),
                ("pH", C.c_void_p), ("T", C.c_void_p), ("system_of_slot", C.c_void_p),
                ("n_order", C.c_int), ("order", C.c_int * 3)]


class GBParams(C.Structure):
    _fields_ = [("eps_in", C.c_double), ("eps_out", C.c_double), ("offset", C.c_double),
                ("alpha", C.c_double), ("beta", C.c_double), ("gamma", C.c_double),
                ("kappa", C.c_double), ("sa_gamma", C.c_double), ("sa_probe", C.c_double),
                ("rgbmax", C.c_double)]


class RunParams(C.Structure):
    _fields_ = [("gb", GBParams), ("dt", C.c_double), ("gamma_ln", C.c_double),
                ("precision", C.c_int), ("mc_ph_every", C.c_int), ("mc_redox_every", C.c_int),
                ("exchange_every", C.c_int), ("shake", C.c_int), ("shake_tol", C.c_double),
                ("t_exchange_energy", C.c_int)]


class MCRecord(C.Structure):
    _fields_ = [("walker", C.c_int), ("site", C.c_int), ("frm", C.c_int), ("to", C.c_int),
                ("accepted", C.c_int), ("pad_", C.c_int), ("dU", C.c_double),
                ("x", C.c_double), ("lnu", C.c_double)]


class ExchangeRow(C.Structure):
    _fields_ = [("walker", C.c_int), ("n_prot", C.c_int), ("n_elec", C.c_int), ("pad_", C.c_int),
                ("u_fix", C.c_int64), ("uref_sum", C.c_double), ("e0ref_ne_sum", C.c_double)]


ROW_DTYPE = np.dtype([("walker", np.int32), ("n_prot", np.int32), ("n_elec", np.int32),
                      ("pad_", np.int32), ("u_fix", np.int64), ("uref_sum", np.float64),
                      ("e0ref_ne_sum", np.float64)])


class ExRecord(C.Structure):
    _fields_ = [("dim", C.c_int), ("slot_lo", C.c_int), ("slot_hi", C.c_int),
                ("walker_lo", C.c_int), ("walker_hi", C.c_int), ("accepted", C.c_int),
                ("x", C.c_double), ("lnu", C.c_double)]


def default_gb() -> GBParams:
    """OBC "igb=2": offset 0.09, (alpha, beta, gamma) = (0.8, 0, 2.909125), eps 1 / 78.5, no salt,
    no surface term (probe 1.4 A when one is switched on), no Born-radius cutoff."""
    return GBParams(1.0, 78.5, 0.09, 0.8, 0.0, 2.909125, 0.0, 0.0, 1.4, 0.0)


_lib = None


def lib():
    """Load libcphremd.so; raises if it was not built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"{LIB} is missing: run paper_1809_07726_gb300.build.build() first")
        L = C.CDLL(LIB)
        vp, i, i64, d = C.c_void_p, C.c_int, C.c_int64, C.c_double
        sig = {
            "cph_init_system": ([vp, i, C.POINTER(GridDesc), C.POINTER(RunParams), C.c_uint64,
                                 C.POINTER(vp)], i),
            "cph_destroy": ([vp], None),
            "cph_last_error": ([vp], C.c_char_p),
            "cph_num_walkers": ([vp], i),
            "cph_total_atoms": ([vp], i),
            "cph_walker_offsets": ([vp, vp], i),
            "cph_site_offsets": ([vp, vp], i),
            "cph_set_launch_mode": ([vp, i], i),
            "cph_set_replica_streams": ([vp, i], i),
            "cph_evaluate": ([vp, vp], i),
            "cph_step_replicas": ([vp, i64, vp], i),
            "cph_mc_titrate": ([vp, i, vp], i),
            "cph_attempt_exchanges": ([vp, i, vp], i),
            "cph_run": ([vp, i64, vp], i),
            "cph_get_energies": ([vp, vp, vp], i),
            "cph_get_forces": ([vp, vp, vp], i),
            "cph_get_born_radii": ([vp, vp, vp], i),
            "cph_get_positions": ([vp, vp, vp], i),
            "cph_set_positions": ([vp, vp, vp], i),
            "cph_get_velocities": ([vp, vp, vp], i),
            "cph_set_velocities": ([vp, vp, vp], i),
            "cph_get_charges": ([vp, vp, vp], i),
            "cph_get_site_states": ([vp, vp, vp], i),
            "cph_set_site_states": ([vp, vp, vp], i),
            "cph_get_counts": ([vp, vp, vp, vp], i),
            "cph_get_condition_map": ([vp, vp, vp], i),
            "cph_set_condition_map": ([vp, vp, vp], i),
            "cph_get_accept_stats": ([vp, vp, vp], i),
            "cph_get_occupancy": ([vp, vp, vp, vp], i),
            "cph_get_visits": ([vp, vp, vp], i),
            "cph_get_fractions": ([vp, vp, vp], i),
            "cph_reset_observables": ([vp, vp], i),
            "cph_fit_hill": ([i, i, vp, vp, C.c_double, C.c_double, C.POINTER(C.c_double),
                              C.POINTER(C.c_double), C.POINTER(C.c_double)], i),
            "cph_predict_delta_e0": ([i, vp, vp, d, d, C.POINTER(C.c_double)], i),
            "cph_predict_e0": ([i, vp, d, i, vp, vp, d, d, vp], i),
            "cph_predict_sum_pka": ([i, vp, d, d, i, vp, d, d, vp], i),
            "cph_get_reference_energies": ([vp, vp], i),
            "cph_get_mc_records": ([vp, vp, i, vp, vp], i),
            "cph_get_exchange_records": ([vp, vp, i, vp, vp], i),
            "cph_get_step": ([vp], i64),
            "cph_set_step": ([vp, i64], i),
            "cph_state_bytes": ([vp], C.c_size_t),
            "cph_get_state": ([vp, vp, C.c_size_t, vp], i),
            "cph_set_state": ([vp, vp, C.c_size_t, vp], i),
            "cph_status": ([vp, vp], i),
            "cph_time_passes": ([vp, i, vp, vp], i),
            "cph_autotune": ([vp, vp, C.POINTER(C.c_int)], i),
            "cph_set_tile_shape": ([vp, i, i], i),
            "cph_set_local_walkers": ([vp, i, vp], i),
            "cph_exchange_rows": ([vp, vp, i, C.POINTER(C.c_int), vp], i),
            "cph_exchange_apply": ([vp, i, vp, i, vp], i),
            "cph_get_tile_shapes": ([vp, vp], i),
            "cph_probe_pipe_rates": ([C.POINTER(C.c_double), C.POINTER(C.c_double), vp], i),
            "cph_gb_workspace_bytes": ([i, i], C.c_size_t),
            "cph_gb_energy": ([i, i, vp, vp, vp, vp, C.POINTER(GBParams), vp, vp, C.c_size_t,
                               vp], i),
            "cph_gb_energy_backward": ([i, i, vp, vp, vp, vp, C.POINTER(GBParams), vp, vp, vp,
                                        vp, vp, C.c_size_t, vp], i),
            "cph_gb_energy_noalloc": ([i, i, vp, vp, vp, vp, C.POINTER(GBParams), vp, vp], i),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(rc, eng=None):
    if rc != OK:
        msg = lib().cph_last_error(eng)
        raise CphError(rc, msg.decode() if msg else "")


def _p(a):
    return C.c_void_p(a.ctypes.data) if a is not None else None


def _stream(stream):
    if stream is not None:
        return C.c_void_p(int(stream))
    try:
        import torch
        if torch.cuda.is_available():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:  # pragma: no cover
        pass
    return None


def _f64(a):
    return np.ascontiguousarray(a, np.float64)


def _i32(a):
    return np.ascontiguousarray(a, np.int32)


class _Keep:
    """Holds the numpy buffers a descriptor points into."""

    def __init__(self):
        self.refs = []

    def __call__(self, a):
        self.refs.append(a)
        return _p(a)


def system_desc(sysd, keep: _Keep, velocities=None) -> SystemDesc:
    """cph_system_desc for a ``synth.System``-like object."""
    n = sysd.n
    sites = (SiteDesc * max(1, len(sysd.sites)))()
    for k, st in enumerate(sysd.sites):
        sites[k] = SiteDesc(SITE_PH if st.kind == "ph" else SITE_REDOX, len(st.atoms),
                            keep(_i32(st.atoms)), st.q.shape[0], keep(_f64(st.q)),
                            keep(_i32(st.n_prot)), keep(_i32(st.n_elec)), float(st.ref),
                            int(st.init_state))
    keep.refs.append(sites)
    d = SystemDesc()
    d.n_atoms = n
    d.x = keep(_f64(sysd.x).reshape(-1))
    d.v = keep(_f64(velocities).reshape(-1)) if velocities is not None else None
    d.mass, d.q, d.rho, d.screen, d.sigma, d.eps = (keep(_f64(a)) for a in (
        sysd.mass, sysd.q, sysd.rho, sysd.screen, sysd.sigma, sysd.eps))
    d.n_bonds = len(sysd.bonds)
    d.bonds = keep(_i32(sysd.bonds).reshape(-1))
    d.bond_k = keep(_f64(sysd.bond_k))
    d.bond_r0 = keep(_f64(sysd.bond_r0))
    d.n_angles = len(sysd.angles)
    d.angles = keep(_i32(sysd.angles).reshape(-1))
    d.angle_k = keep(_f64(sysd.angle_k))
    d.angle_t0 = keep(_f64(sysd.angle_t0))
    d.n_excl = 0
    d.excl = None
    d.n_sites = len(sysd.sites)
    d.sites = C.cast(sites, C.c_void_p) if sysd.sites else None
    return d


class Engine:
    """Owns a cph_engine*.  Methods mirror the C calls."""

    def __init__(self, ptr, systems, grid):
        self.ptr = ptr
        self.systems = systems
        self.grid = grid
        L = lib()
        self.W = L.cph_num_walkers(ptr)
        self.total_atoms = L.cph_total_atoms(ptr)
        self.offsets = np.zeros(self.W + 1, np.int32)
        _check(L.cph_walker_offsets(ptr, _p(self.offsets)))
        self.site_offsets = np.zeros(self.W + 1, np.int32)
        _check(L.cph_site_offsets(ptr, _p(self.site_offsets)))

    def __del__(self):
        if getattr(self, "ptr", None):
            lib().cph_destroy(self.ptr)
            self.ptr = None

    close = __del__

    def _c(self, rc):
        _check(rc, self.ptr)

    # ---- hot path
    def set_launch_mode(self, mode):
        self._c(lib().cph_set_launch_mode(self.ptr, mode))

    def set_replica_streams(self, n):
        self._c(lib().cph_set_replica_streams(self.ptr, int(n)))

    def evaluate(self, stream=None):
        self._c(lib().cph_evaluate(self.ptr, _stream(stream)))

    def step_replicas(self, n_steps, stream=None):
        self._c(lib().cph_step_replicas(self.ptr, int(n_steps), _stream(stream)))

    def mc_titrate(self, kind=MC_BOTH, stream=None):
        self._c(lib().cph_mc_titrate(self.ptr, kind, _stream(stream)))

    def attempt_exchanges(self, dim=DIM_NEXT, stream=None):
        self._c(lib().cph_attempt_exchanges(self.ptr, dim, _stream(stream)))

    def run(self, n_steps, stream=None):
        self._c(lib().cph_run(self.ptr, int(n_steps), _stream(stream)))

    # ---- getters / setters
    def _get(self, fn, shape, dtype=np.float64, stream=None):
        out = np.zeros(shape, dtype)
        self._c(fn(self.ptr, _p(out), _stream(stream)))
        return out

    def energies(self, stream=None):
        return self._get(lib().cph_get_energies, (self.W, NTERMS), stream=stream)

    def forces(self, stream=None):
        return self._get(lib().cph_get_forces, (self.total_atoms, 3), stream=stream)

    def born_radii(self, stream=None):
        return self._get(lib().cph_get_born_radii, (self.total_atoms,), stream=stream)

    def positions(self, stream=None):
        return self._get(lib().cph_get_positions, (self.total_atoms, 3), stream=stream)

    def velocities(self, stream=None):
        return self._get(lib().cph_get_velocities, (self.total_atoms, 3), stream=stream)

    def charges(self, stream=None):
        return self._get(lib().cph_get_charges, (self.total_atoms,), stream=stream)

    def site_states(self, stream=None):
        return self._get(lib().cph_get_site_states, (int(self.site_offsets[-1]),), np.int32,
                         stream=stream)

    def condition_map(self, stream=None):
        return self._get(lib().cph_get_condition_map, (self.W,), np.int32, stream=stream)

    def accept_stats(self, stream=None):
        return self._get(lib().cph_get_accept_stats, (10,), np.int64, stream=stream)

    # ---- sampling observables
    def occupancy(self, stream=None):
        """(counts [site rows, MAX_STATES] int64, samples): row
        site_offsets[s] + k is site k of the walker at condition slot s."""
        out = np.zeros((int(self.site_offsets[-1]), MAX_STATES), np.int64)
        n = C.c_int64(0)
        self._c(lib().cph_get_occupancy(self.ptr, _p(out), C.byref(n), _stream(stream)))
        return out, int(n.value)

    def visits(self, stream=None):
        return self._get(lib().cph_get_visits, (self.W, self.W), np.int64, stream=stream)

    def fractions(self, stream=None):
        return self._get(lib().cph_get_fractions, (int(self.site_offsets[-1]),), stream=stream)

    def reset_observables(self, stream=None):
        self._c(lib().cph_reset_observables(self.ptr, _stream(stream)))

    def set_positions(self, x, stream=None):
        self._c(lib().cph_set_positions(self.ptr, _p(_f64(x).reshape(-1)), _stream(stream)))

    def set_velocities(self, v, stream=None):
        self._c(lib().cph_set_velocities(self.ptr, _p(_f64(v).reshape(-1)), _stream(stream)))

    def set_site_states(self, s, stream=None):
        self._c(lib().cph_set_site_states(self.ptr, _p(_i32(s)), _stream(stream)))

    def set_condition_map(self, m, stream=None):
        self._c(lib().cph_set_condition_map(self.ptr, _p(_i32(m)), _stream(stream)))

    def counts(self, stream=None):
        npr = np.zeros(self.W, np.int32)
        nel = np.zeros(self.W, np.int32)
        self._c(lib().cph_get_counts(self.ptr, _p(npr), _p(nel), _stream(stream)))
        return npr, nel

    def reference_energies(self):
        n = sum(sum(len(st.q) for st in s.sites) for s in self.systems)
        out = np.zeros(max(1, n))
        self._c(lib().cph_get_reference_energies(self.ptr, _p(out)))
        return out[:n]

    def mc_records(self, stream=None):
        n = int(self.site_offsets[-1])
        buf = (MCRecord * max(1, n))()
        got = C.c_int(0)
        self._c(lib().cph_get_mc_records(self.ptr, C.cast(buf, C.c_void_p), n, C.byref(got),
                                         _stream(stream)))
        return [buf[i] for i in range(got.value)]

    def exchange_records(self, stream=None):
        buf = (ExRecord * max(1, self.W))()
        got = C.c_int(0)
        self._c(lib().cph_get_exchange_records(self.ptr, C.cast(buf, C.c_void_p), self.W,
                                               C.byref(got), _stream(stream)))
        return [buf[i] for i in range(got.value)]

    def get_state(self, stream=None):
        """Checkpoint as a uint8 array (see cph_get_state)."""
        buf = np.zeros(lib().cph_state_bytes(self.ptr), np.uint8)
        self._c(lib().cph_get_state(self.ptr, _p(buf), buf.size, _stream(stream)))
        return buf

    def set_state(self, buf, stream=None):
        buf = np.ascontiguousarray(buf, np.uint8)
        self._c(lib().cph_set_state(self.ptr, _p(buf), buf.size, _stream(stream)))

    def get_step(self):
        return int(lib().cph_get_step(self.ptr))

    def set_step(self, t):
        self._c(lib().cph_set_step(self.ptr, int(t)))

    def time_passes(self, reps=3, stream=None):
        """Mean CUDA-event durations (ms) of the Born, GB/Coulomb/LJ and chain passes."""
        ms = np.zeros(3)
        self._c(lib().cph_time_passes(self.ptr, int(reps), _p(ms), _stream(stream)))
        return ms

    def autotune(self, stream=None):
        """cph_autotune: pick the fastest work-item size; returns it."""
        c = C.c_int(0)
        self._c(lib().cph_autotune(self.ptr, _stream(stream), C.byref(c)))
        return c.value

    # ---- one grid sharded over several engines
    def set_local_walkers(self, walkers):
        w = _i32(walkers).reshape(-1)
        self._c(lib().cph_set_local_walkers(self.ptr, w.size, _p(w)))

    def exchange_rows(self, stream=None):
        """Energies at the current state, then one row per local walker
        (a structured array of ROW_DTYPE)."""
        out = np.zeros(self.W, ROW_DTYPE)
        n = C.c_int(0)
        self._c(lib().cph_exchange_rows(self.ptr, _p(out), self.W, C.byref(n), _stream(stream)))
        return out[:n.value].copy()

    def exchange_apply(self, dim, rows, stream=None):
        r = np.ascontiguousarray(rows, ROW_DTYPE)
        self._c(lib().cph_exchange_apply(self.ptr, int(dim), _p(r), r.size, _stream(stream)))

    def set_tile_shape(self, system, shape):
        self._c(lib().cph_set_tile_shape(self.ptr, int(system), int(shape)))

    def tile_shapes(self):
        out = np.zeros(len(self.systems), np.int32)
        self._c(lib().cph_get_tile_shapes(self.ptr, _p(out)))
        return out

    def status(self, stream=None):
        self._c(lib().cph_status(self.ptr, _stream(stream)))

    def walker_slice(self, w):
        return slice(int(self.offsets[w]), int(self.offsets[w + 1]))


def probe_pipe_rates(stream=None):
    """(FP32 lane ops/s, MUFU ops/s) measured on the current device."""
    a, b = C.c_double(), C.c_double()
    _check(lib().cph_probe_pipe_rates(C.byref(a), C.byref(b), _stream(stream)))
    return a.value, b.value


def fit_hill(kind, x, f, T=300.0, v=1.0):
    """Least-squares fit of eq (1) (kind FIT_PH) or eq (2) (FIT_REDOX) to the
    fractions f at x: returns (x0, n_hill, rss)."""
    x, f = _f64(x).reshape(-1), _f64(f).reshape(-1)
    if x.size != f.size:
        raise ValueError("x and f differ in length")
    x0, n, rss = C.c_double(), C.c_double(), C.c_double()
    _check(lib().cph_fit_hill(kind, x.size, _p(x), _p(f), float(T), float(v), C.byref(x0),
                              C.byref(n), C.byref(rss)))
    return x0.value, n.value, rss.value


def predict_delta_e0(pka_red, pka_oxi, T, v=1.0):
    """Eq (6): E0_prot - E0_deprot (V) from the per-site pKa_red, pKa_oxi."""
    a, b = _f64(pka_red).reshape(-1), _f64(pka_oxi).reshape(-1)
    if a.size != b.size:
        raise ValueError("pka_red and pka_oxi differ in length")
    out = C.c_double()
    _check(lib().cph_predict_delta_e0(a.size, _p(a), _p(b), float(T), float(v), C.byref(out)))
    return out.value


def predict_e0(pH, e0_prot, pka_red, pka_oxi, T, v=1.0):
    """Eq (7): the pH-dependent E0 (V) at every pH."""
    x = _f64(pH).reshape(-1)
    a, b = _f64(pka_red).reshape(-1), _f64(pka_oxi).reshape(-1)
    if a.size != b.size:
        raise ValueError("pka_red and pka_oxi differ in length")
    out = np.zeros(x.size)
    _check(lib().cph_predict_e0(x.size, _p(x), float(e0_prot), a.size, _p(a), _p(b), float(T),
                                float(v), _p(out)))
    return out


def predict_sum_pka(E, e0_prot, e0_deprot, pka_red, T, v=1.0):
    """Eq (8): the sum of the pH sites' pKa values at every redox potential E (V)."""
    x = _f64(E).reshape(-1)
    a = _f64(pka_red).reshape(-1)
    out = np.zeros(x.size)
    _check(lib().cph_predict_sum_pka(x.size, _p(x), float(e0_prot), float(e0_deprot), a.size,
                                     _p(a), float(T), float(v), _p(out)))
    return out


def init_system(systems, grid, seed, precision=PREC_FP32, dt=0.002, gamma_ln=10.0,
                mc_ph_every=10, mc_redox_every=10, exchange_every=100, gb=None,
                velocities=None, shake=False, shake_tol=1e-10,
                t_exchange_energy=TEX_POTENTIAL) -> Engine:
    """cph_init_system for a list of ``synth.System`` and a ``synth.Grid``."""
    keep = _Keep()
    descs = (SystemDesc * len(systems))()
    for k, s in enumerate(systems):
        descs[k] = system_desc(s, keep, None if velocities is None else velocities[k])
    g = GridDesc()
    g.nE, g.npH, g.nT = len(grid.E), len(grid.pH), len(grid.T)
    g.E, g.pH, g.T = keep(_f64(grid.E)), keep(_f64(grid.pH)), keep(_f64(grid.T))
    g.system_of_slot = keep(_i32(grid.system_of_slot))
    g.n_order = len(grid.order)
    for k, name in enumerate(grid.order):
        g.order[k] = DIM_NAMES[name]
    p = RunParams(gb or default_gb(), dt, gamma_ln, precision, mc_ph_every, mc_redox_every,
                  exchange_every, 1 if shake else 0, shake_tol, int(t_exchange_energy))
    out = C.c_void_p()
    rc = lib().cph_init_system(C.cast(descs, C.c_void_p), len(systems), C.byref(g), C.byref(p),
                               C.c_uint64(seed), C.byref(out))
    _check(rc, None)
    return Engine(out, systems, grid)


# ---------------------------------------------------- differentiable GB energy

def gb_workspace_bytes(n_rep, n):
    return int(lib().cph_gb_workspace_bytes(n_rep, n))


def _dptr(t):
    return C.c_void_p(t.data_ptr())


def gb_energy(x, q, rho, screen, gb=None, workspace=None, stream=None):
    """E_GB [n_rep] (float64 CUDA tensor) for x [n_rep, n, 3], q and rho [n_rep, n]
    (float32 CUDA tensors) and screen [n]."""
    import torch
    n_rep, n = q.shape
    x, q, rho, screen = (t.contiguous() for t in (x, q, rho, screen))
    E = torch.empty(n_rep, dtype=torch.float64, device=q.device)
    ws = workspace if workspace is not None else _workspace(n_rep, n, q.device)
    g = gb or default_gb()
    _check(lib().cph_gb_energy(n_rep, n, _dptr(x), _dptr(q), _dptr(rho), _dptr(screen),
                               C.byref(g), _dptr(E), _dptr(ws), ws.numel(), _stream(stream)))
    return E


def gb_energy_backward(x, q, rho, screen, dE, gb=None, workspace=None, stream=None):
    import torch
    n_rep, n = q.shape
    x, q, rho, screen = (t.contiguous() for t in (x, q, rho, screen))
    dE = dE.to(torch.float64).contiguous()
    dx = torch.empty_like(x)
    dq = torch.empty_like(q)
    drho = torch.empty_like(rho)
    ws = workspace if workspace is not None else _workspace(n_rep, n, q.device)
    g = gb or default_gb()
    _check(lib().cph_gb_energy_backward(n_rep, n, _dptr(x), _dptr(q), _dptr(rho), _dptr(screen),
                                        C.byref(g), _dptr(dE), _dptr(dx), _dptr(dq),
                                        _dptr(drho), _dptr(ws), ws.numel(), _stream(stream)))
    return dx, dq, drho


def gb_energy_noalloc(x, q, rho, screen, gb=None, stream=None):
    """E_GB like gb_energy, without a workspace: the library's fixed scratch
    array is used (see cph_gb_energy_noalloc in cphremd.h for its size limit and
    the rule that overlapping calls race)."""
    import torch
    n_rep, n = q.shape
    x, q, rho, screen = (t.contiguous() for t in (x, q, rho, screen))
    E = torch.empty(n_rep, dtype=torch.float64, device=q.device)
    g = gb or default_gb()
    _check(lib().cph_gb_energy_noalloc(n_rep, n, _dptr(x), _dptr(q), _dptr(rho), _dptr(screen),
                                       C.byref(g), _dptr(E), _stream(stream)))
    return E


def _workspace(n_rep, n, device):
    import torch
    nb = gb_workspace_bytes(n_rep, n)
    return torch.empty(nb, dtype=torch.uint8, device=device)  # caching allocator: 512-B aligned


def _gb_function():
    import torch

    class GBEnergy(torch.autograd.Function):
        """E_GB with the hand-written adjoint kernel as its backward."""

        @staticmethod
        def forward(ctx, x, q, rho, screen):
            ctx.save_for_backward(x, q, rho, screen)
            return gb_energy(x, q, rho, screen)

        @staticmethod
        def backward(ctx, gE):
            x, q, rho, screen = ctx.saved_tensors
            dx, dq, drho = gb_energy_backward(x, q, rho, screen, gE)
            return dx, dq, drho, None

    return GBEnergy


def __getattr__(name):
    if name == "GBEnergy":
        return _gb_function()
    raise AttributeError(name)
