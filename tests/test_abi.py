"""Host-side tests of the C ABI (no GPU needed): the library builds, exports
every function include/cphremd.h declares, and rejects invalid descriptors
before touching the device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1809_07726_gb300 import build, cphremd, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cphremd.h")


@pytest.fixture(scope="module")
def L():
    build.build()
    return cphremd.lib()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cph_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary_calls():
    names = declared_functions()
    for core in ("cph_init_system", "cph_step_replicas", "cph_mc_titrate",
                 "cph_attempt_exchanges", "cph_run", "cph_gb_energy", "cph_gb_energy_backward"):
        assert core in names


def test_library_exports_every_declared_symbol(L):
    for name in declared_functions():
        assert hasattr(L, name), name


def _descs(systems, grid, keep):
    descs = (cphremd.SystemDesc * len(systems))()
    for k, s in enumerate(systems):
        descs[k] = cphremd.system_desc(s, keep)
    g = cphremd.GridDesc()
    g.nE, g.npH, g.nT = len(grid.E), len(grid.pH), len(grid.T)
    g.E, g.pH, g.T = keep(np.asarray(grid.E, float)), keep(np.asarray(grid.pH, float)), keep(
        np.asarray(grid.T, float))
    g.system_of_slot = keep(np.asarray(grid.system_of_slot, np.int32))
    g.n_order = len(grid.order)
    for k, nm in enumerate(grid.order):
        g.order[k] = cphremd.DIM_NAMES[nm]
    return descs, g


def _init(L, systems, grid, **kw):
    keep = cphremd._Keep()
    descs, g = _descs(systems, grid, keep)
    gb = cphremd.default_gb()
    gb.rgbmax = kw.get("rgbmax", 0.0)
    p = cphremd.RunParams(gb, kw.get("dt", 0.002), 10.0,
                          kw.get("precision", cphremd.PREC_FP32), 10, 10, 100)
    out = C.c_void_p()
    rc = L.cph_init_system(C.cast(descs, C.c_void_p), len(systems), C.byref(g), C.byref(p), 1,
                           C.byref(out))
    return rc, out, L.cph_last_error(None).decode()


@pytest.fixture(scope="module")
def small():
    return synth.make_system(30, 2, n_ph=1, ph_atoms=(6, 6), redox_atoms=6)


def test_rejects_bad_system_index(L, small):
    grid = synth.Grid(np.array([0.0]), np.array([7.0]), np.array([300.0]),
                      np.array([1], np.int32))
    rc, out, msg = _init(L, [small], grid)
    assert rc == cphremd.E_INVALID and not out.value and "system_of_slot" in msg


def test_rejects_shared_site_atoms(L, small):
    import copy
    s = copy.deepcopy(small)
    s.sites[1].atoms = s.sites[0].atoms.copy()
    grid = synth.Grid(np.array([0.0]), np.array([7.0]), np.array([300.0]), np.zeros(1, np.int32))
    rc, out, msg = _init(L, [s], grid)
    assert rc == cphremd.E_INVALID and "shared" in msg


def test_rejects_radius_below_offset(L, small):
    import copy
    s = copy.deepcopy(small)
    s.rho[3] = 0.05
    grid = synth.Grid(np.array([0.0]), np.array([7.0]), np.array([300.0]), np.zeros(1, np.int32))
    rc, _, msg = _init(L, [s], grid)
    assert rc == cphremd.E_INVALID and "rho" in msg


def test_rejects_nonfinite_positions(L, small):
    import copy
    s = copy.deepcopy(small)
    s.x[4, 1] = np.nan
    grid = synth.Grid(np.array([0.0]), np.array([7.0]), np.array([300.0]), np.zeros(1, np.int32))
    rc, _, msg = _init(L, [s], grid)
    assert rc == cphremd.E_INVALID and "non-finite" in msg


def test_rejects_bad_precision_and_timestep(L, small):
    grid = synth.Grid(np.array([0.0]), np.array([7.0]), np.array([300.0]), np.zeros(1, np.int32))
    rc, _, _ = _init(L, [small], grid, precision=7)
    assert rc == cphremd.E_INVALID
    rc, _, _ = _init(L, [small], grid, dt=0.0)
    assert rc == cphremd.E_INVALID


def test_rejects_site_beyond_64_atoms(L):
    s = synth.make_system(200, 43, n_ph=1, ph_atoms=(65, 65), n_redox=0)
    grid = synth.Grid(np.array([0.0]), np.array([7.0]), np.array([300.0]), np.zeros(1, np.int32))
    rc, out, msg = _init(L, [s], grid)
    assert rc == cphremd.E_INVALID and not out.value and "n_atoms must be 1..64" in msg
    s64 = synth.make_system(200, 43, n_ph=1, ph_atoms=(64, 64), n_redox=0)
    rc, out, _ = _init(L, [s64], grid)
    assert rc != cphremd.E_INVALID  # the limit itself is accepted (no GPU here: a CUDA error)


@pytest.mark.parametrize("rgbmax", [-1.0, float("nan"), float("inf")])
def test_rejects_bad_born_radius_cutoff(L, small, rgbmax):
    grid = synth.Grid(np.array([0.0]), np.array([7.0]), np.array([300.0]), np.zeros(1, np.int32))
    rc, out, msg = _init(L, [small], grid, rgbmax=rgbmax)
    assert rc == cphremd.E_INVALID and not out.value and "rgbmax" in msg


def test_gb_energy_rejects_bad_arguments(L):
    g = cphremd.default_gb()
    rc = L.cph_gb_energy(0, 10, None, None, None, None, C.byref(g), None, None, 0, None)
    assert rc == cphremd.E_INVALID
    assert L.cph_gb_workspace_bytes(0, 5) == 0
    # misaligned workspace is refused before any launch
    rc = L.cph_gb_energy(1, 10, C.c_void_p(16), C.c_void_p(16), C.c_void_p(16), C.c_void_p(16),
                         C.byref(g), C.c_void_p(16), C.c_void_p(8), 1 << 20, None)
    assert rc == cphremd.E_INVALID
    assert "aligned" in L.cph_last_error(None).decode()


def test_tile_shape_calls_refuse_a_missing_engine(L):
    assert L.cph_set_tile_shape(None, 0, cphremd.SHAPE_SYMMETRIC) == cphremd.E_INVALID
    shapes = np.zeros(1, np.int32)
    assert L.cph_get_tile_shapes(None, shapes.ctypes.data) == cphremd.E_INVALID
